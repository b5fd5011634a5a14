/*
 * cs.h — C ABI of the GB300 (sm_103a) implementation of the component-splitting implicit
 * LU-SGS scheme for multicomponent reacting flows (Zhang, Cai & Pan, arXiv:2403.03440).
 *
 * One pseudo-time iteration (Sec. 2.2-2.3 of the paper): explicit residual R(Q) (Eq.
 * (iterate): MUSCL + Roe inviscid flux, central viscous and diffusive fluxes, finite-rate
 * chemistry), then either the split (CS) operator — flow block with the flow spectral radius
 * plus ns scalar species equations with their own radius and the chemical source diagonal
 * (Sec. 2.3.1-2.3.2) — or the coupled (CI) (4+N)-block operator, both solved by LU-SGS
 * forward/backward sweeps (Sec. 2.2), then the consistency corrections and the update
 * (Sec. 2.3.3).
 *
 * Conventions
 *  - Every function returns a cs_status; none aborts, exits or traps.  On error the grid keeps
 *    a message (cs_last_error) and, for device-detected errors, the offending cell index.
 *  - Units SI; 2D grids have unit depth.  FP64 throughout.
 *  - Cells are numbered c = i + ni*(j + nj*k) (i fastest); arrays are struct-of-arrays
 *    [var][cell].  Conserved state Q: var = rho_1..rho_ns, rho*u_1..rho*u_d, rho*E,
 *    [rho*e_v] (two-temperature models), nq = ns + d + 1 (+1).
 *  - Split increments dQ: (rho, rho*u_1..d, rho*E, [rho*e_v], rho_1..rho_ns), nsplit = nF + ns
 *    with nF = d + 2 (+1).  Coupled increments: (rho, rho*u, rho*E, [rho*e_v],
 *    rho_2..rho_ns), nci = nF + ns - 1: the first species (N2 in air, the most abundant) is
 *    eliminated as rho - sum of the others (Sec. 2.3.3 eliminates one species; eliminating
 *    the electron, last in the list, would leave the coupled blocks singular).
 *  - Pointers marked "host or device" may be either (the library copies with
 *    cudaMemcpyDefault); they are borrowed for the duration of the call and owned by the
 *    caller.  The grid owns all of its device work arrays.
 *  - All device work is enqueued on the CUDA stream given at creation; functions that return
 *    host values synchronise that stream.
 */
#ifndef CS_H
#define CS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CS_OK = 0,
  CS_ERR_ARG = 1,          /* invalid argument (size, pointer, option) */
  CS_ERR_OOM = 2,          /* device allocation failed */
  CS_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  CS_ERR_NONPHYSICAL = 4,  /* negative density / non-positive mixture sum / singular block */
  CS_ERR_NEWTON = 5,       /* temperature solve did not converge */
  CS_ERR_TIMEOUT = 6,      /* a bounded device wait gave up */
  CS_ERR_STATE = 7         /* call order: e.g. operator before residual */
} cs_status;

enum { CS_BC_PERIODIC = 0, CS_BC_WALL = 1, CS_BC_FARFIELD = 2, CS_BC_OUTFLOW = 3, CS_BC_AXIS = 4 };
/* Gas models: single-species perfect diatomic gas (tests), 5-species air with one
 * temperature and 5 reactions, 11-species ionised air with two temperatures and 21
 * reactions (Sec. 3.2 / 3.3 of the paper: Park's model). */
enum { CS_MECH_PERFECT = 0, CS_MECH_AIR5 = 1, CS_MECH_AIR11 = 2 };
enum { CS_SCHEME_SPLIT = 0, CS_SCHEME_COUPLED = 1 };
/* Precision of the implicit operator: CS_FP64 everywhere, or CS_MIXED = the LU-SGS sweeps of
 * the split operator compute in FP32 (from FP64 spectral radii, diagonals and right-hand side,
 * into FP64 increments) while the residual, the corrections and the update stay FP64. */
enum { CS_FP64 = 0, CS_MIXED = 1 };

typedef struct cs_grid_s *cs_grid;

typedef struct {
  int ndim;          /* 2 or 3 */
  int ni, nj, nk;    /* cells per direction (nk ignored for 2D) */
  int bc[6];         /* imin, imax, jmin, jmax, kmin, kmax: CS_BC_*; a periodic pair must
                        be periodic on both sides */
  int mech;          /* CS_MECH_* */
  int limiter;       /* 0 first order, 1 minmod (paper), 2 van Albada */
  double entropy_fix;/* Harten coefficient eps (delta = eps (|u_n| + c)); 0.1 typical */
  int reacting;      /* 1: chemical and vibrational sources on, 0: off */
} cs_grid_desc;

typedef struct {
  double T, Tv, p, mach;   /* K, K, Pa, - ; Tv ignored by one-temperature models */
  double Y[16];            /* mass fractions in the model's species order */
  double dir[3];           /* flow direction (normalised by the library) */
} cs_freestream;

typedef struct {
  double Tw;               /* isothermal wall temperature, K */
  int catalytic;           /* must be 0 (non-catalytic) */
} cs_wall;

typedef struct {
  int scheme;              /* CS_SCHEME_SPLIT | CS_SCHEME_COUPLED */
  int correction;          /* 1 (CS-1) or 2 (CS-2); ignored by the coupled scheme */
  int clip;                /* 1: negative densities set to 0 and counted */
  double cfl;              /* target CFL */
  double cfl_start;        /* first CFL of the geometric ramp */
  int ramp_iters;          /* ramp length in iterations (0: no ramp) */
  int precision;           /* CS_FP64 or CS_MIXED (split scheme) */
  int iters;               /* iterations to run */
} cs_step_opts;

typedef struct {
  int iters_done;
  double r_species, r_energy;   /* L2 over cells of R/V, species and energy (last residual) */
  double q_stag;                /* stagnation wall heat flux, W/m^2 */
  int nclip;                    /* clipped values in the last correction */
  int status_cell;              /* cell of the last device-detected error, or -1 */
} cs_step_stats;

/* Create a grid on the current CUDA device.  nodes_host: node coordinates, host memory,
 * SoA [d][(nk+1)][(nj+1)][(ni+1)] (2D: [d][(nj+1)][(ni+1)]).  cuda_stream: cudaStream_t or
 * NULL for the legacy default stream.  Geometry (a1: face area vectors S = xi_x/J, volumes
 * V = 1/J, centroids; Sec. 2.2) is computed on the device.  Errors: CS_ERR_ARG (sizes, bc,
 * mech), CS_ERR_OOM, CS_ERR_CUDA. */
cs_status cs_grid_create(const cs_grid_desc *desc, const double *nodes_host, void *cuda_stream,
                         cs_grid *out);
cs_status cs_grid_destroy(cs_grid g);

/* Sizes: out[0] = ncell, [1] = nq, [2] = nsplit, [3] = nci, [4] = ns, [5] = ntemp,
 * [6] = nF, [7] = stagnation cell (-1 before cs_set_boundary). */
cs_status cs_grid_dims(cs_grid g, int out[8]);

/* Freestream and wall data (far-field ghost states, wall temperature, stagnation cell). */
cs_status cs_set_boundary(cs_grid g, const cs_freestream *fs, const cs_wall *wall);

/* Q (host or device, [nq][ncell]): set the conserved state.  Resets the iteration counter
 * and the temperature warm starts. */
cs_status cs_set_state(cs_grid g, const double *Q);
/* Q (host or device, [nq][ncell]): replace the conserved state and continue the run: unlike
 * cs_set_state, the iteration counter (and with it the CFL ramp) and the temperature warm
 * starts are kept.  For a caller that holds the state in its own memory between iterations of
 * one run.  The copy is enqueued on the grid's stream (a host Q must stay valid until the next
 * call that synchronises it).  Errors: CS_ERR_ARG (null), CS_ERR_CUDA. */
cs_status cs_load_state(cs_grid g, const double *Q);
/* Fill Q with the uniform freestream (after cs_set_boundary). */
cs_status cs_init_freestream(cs_grid g);
/* Q_out (host or device, [nq][ncell]). */
cs_status cs_get_state(cs_grid g, double *Q_out);

/* Residual R(Q) (Sec. 2.2 Eq. (iterate)): R = sum_faces (F_inv + F_vis).S_out - V S(Q).
 * R_out (host or device, [nq][ncell], nullable).  norms_host[3] (nullable): r_species,
 * r_energy, q_stag.  Errors: CS_ERR_NONPHYSICAL / CS_ERR_NEWTON from the primitive recovery. */
cs_status cs_residual(cs_grid g, double *R_out, double norms_host[3]);

/* Split operator (Sec. 2.3.1-2.3.2) solved by LU-SGS (Sec. 2.2) with the local time step of
 * the given CFL; uses R of the last cs_residual.  dQ_out (host or device,
 * [nsplit][ncell], nullable).  precision: CS_FP64 or CS_MIXED.  Errors: CS_ERR_STATE (no
 * residual); CS_ERR_TIMEOUT (a bounded wait of the 2D point-to-point sweep for a neighbouring
 * CTA's increments gave up; the increments are then not valid). */
cs_status cs_lusgs_split(cs_grid g, double cfl, int precision, double *dQ_out);

/* Coupled (CI) operator: unified spectral radius, dense diagonal blocks with the source
 * Jacobian, LU-SGS.  dQ_out (host or device, [nci][ncell], nullable).  The first call
 * allocates library-owned work arrays: the LU factors, pivots and inverse of every cell's
 * diagonal block (2 nci^2 doubles + nci ints per cell) and, on 2D grids of at most 256 rows
 * in j, the four neighbour coupling blocks of the one-launch sweep (4 nci nP + nP doubles per
 * cell, nP = nci rounded up to even, plus 2 nci nP per row j; without them the sweep applies
 * the products matrix-free).
 * Errors: CS_ERR_STATE (no residual), CS_ERR_OOM (the factors could not be allocated). */
cs_status cs_lusgs_coupled(cs_grid g, double cfl, double *dQ_out);

/* Consistency correction and update (Sec. 2.3.3): mode 1 = CS-1 (increment normalisation),
 * 2 = CS-2 (mass-fraction normalisation), 0 = coupled update.  dQ (host or device, nullable:
 * NULL uses the increments of the last cs_lusgs_split / cs_lusgs_coupled); layout split for
 * modes 1-2, coupled for mode 0.  nclip_out (nullable): clipped values. */
cs_status cs_correct(cs_grid g, int mode, int clip, const double *dQ, int *nclip_out);

/* opts->iters pseudo-time iterations: residual, operator, correction + update.  Errors: those
 * of cs_residual, cs_lusgs_split / cs_lusgs_coupled and cs_correct. */
cs_status cs_step(cs_grid g, const cs_step_opts *opts, cs_step_stats *stats);

/* Per-cell auxiliary fields for tests and monitors: name in {"T", "Tv", "p", "c", "rho",
 * "mu", "lamF", "lamC", "lamCI", "DF", "DFev", "Ds", "omega", "dom", "V", "xc"}; out (host or
 * device) must hold the returned count of doubles; *count_out = number written. */
cs_status cs_get_field(cs_grid g, const char *name, double *out, int *count_out);

/* Library's gas-model constants (host, no device work): M[ns] kg/kmol, hf[ns] J/kg,
 * dims[3] = ns, nreactions, ntemp. */
cs_status cs_gas_info(int mech, double *M, double *hf, int dims[3]);

/* Per-phase device timing of cs_step with CUDA events on the grid's stream (not part of the
 * method; a measurement aid).  Phases: 0 primitives (the temperature solves; with the
 * chemistry where the second stream below could not be made), 1 gradients, 2 face fluxes, up
 * to the end of the chemistry, which cs_step runs on a second library-owned stream beside
 * phases 1 and 2 (forked from and joined back into the grid's stream), 3 residual assembly +
 * norms, 4 spectral radii / diagonals (+ coupled blocks), 5 forward sweep, 6 backward sweep, 7
 * correction + update.  ms_out[8] and launches_out[8] (host,
 * nullable) receive the totals accumulated since the last call; the call then resets them
 * and enables (enable = 1) or disables timing. */
cs_status cs_profile(cs_grid g, int enable, double *ms_out, long *launches_out);

/* FP64 fused multiply-add throughput of the current device in GFLOP/s (a measurement aid, not
 * part of the method): independent DFMA chains on every SM, timed with CUDA events on
 * cuda_stream (NULL: legacy default stream), best of three launches after a warm-up (~0.1 s in
 * all).  The FP64-bound kernels of the residual are compared with this rate.  Errors:
 * CS_ERR_ARG (null), CS_ERR_CUDA. */
cs_status cs_measure_fp64_rate(void *cuda_stream, double *gflops_out);

/* Which kernel ran the last split sweep of g (a measurement aid, not part of the method):
 * out[0] in the numbering of the "cluster_sweep" option below (0 one launch per hyperplane,
 * 1 direct loads, 2 wavefront records, 4 one CTA per component, 5 assembled couplings exchanged
 * point to point, 6 assembled couplings with a cluster barrier; -1 before the first sweep),
 * out[1] its CTAs per cluster (0 for one launch per hyperplane).  Host only, no device work.
 * Errors: CS_ERR_ARG (null). */
cs_status cs_sweep_info(cs_grid g, int out[2]);

/* Implementation options (not part of the method): "cluster_sweep" = 3 (default) runs the 2D
 * split sweeps in one launch, choosing per precision: 5 where its records can be allocated and
 * its ring fits, else for the FP32 operator 4 where it applies, else 2, and for FP64 6, else 1.
 * 1 is a thread-block-cluster kernel reading the cell arrays directly, 2 a cluster kernel over
 * hyperplane-ordered cell records, 4 the FP32 operator's sweeps with one CTA per component
 * holding every row (nj <= 384; __syncthreads between hyperplanes; FP64 and larger grids fall
 * back to 2), 5 the sweeps over neighbour couplings assembled beforehand: D^-1 times the split
 * Jacobian blocks, formed by one parallel launch into library-owned records (FP64, or FP32,
 * formed in FP32, for the FP32 operator) of 4 nF nP + 4 elements per cell and 2 nF nP + 4 per row j, nP =
 * nF rounded up to a whole 16-byte load; then a cluster kernel with 8 threads per row whose
 * CTAs exchange the rows at their boundaries point to point (st.async into the next CTA's
 * shared memory, one mbarrier per hyperplane) and each thread copies its step inputs six steps
 * ahead with cp.async into a ring in shared memory ((ni + nj - 1) x (8 x element size + 8)
 * bytes plus 7 x threads x (2 nP x element size + 16) bytes per CTA, at most 200 KiB; single
 * grids only), 6 the FP64 couplings with one cluster barrier per hyperplane (the FP32 operator
 * falls back to 4, else 2); 7 (a retired form that swept the couplings with systolic warps)
 * runs as 5; 0 runs one launch per hyperplane.
 * All give the same arithmetic up to rounding.  cs_batch_tune reports 4 as kind 3 with C = 1.
 * "cluster_size" = C in {1, 2, 4, 8, 16} fixes the CTAs per component of the 2D cluster
 * sweeps (0, the default: the largest that fits; a C that does not fit the grid or the device
 * falls back to one launch per hyperplane); cs_batch_tune sets it.
 * Method option: "h_correction" = 1 (default) widens the entropy fix of every face's Roe flux
 * to at least twice the face's multidimensional H-correction (Sanders, Morano and Druguet,
 * J. Comput. Phys. 145, 1998; the paper names Roe's scheme, Sec. 3.2, but not its entropy
 * fix), which keeps the bow shock of a blunt body free of the carbuncle instability; 0 keeps
 * only the one-dimensional fix entropy_fix (|u_n| + c).
 * Method option: "update_limit" = f >= 0 (default 0 = off; not in the paper) scales each
 * cell's whole increment before the consistency corrections of cs_correct / cs_step by
 * alpha = min(1, f rho / |d rho|), halved (at most 30 times) while the corrected state is
 * non-physical or its specific translational(-rotational) thermal energy leaves a factor
 * 1 + f of the old one, or (2T) its specific pool energy gains more than f times the old
 * specific thermal plus pool energy.  alpha is 1 once increments are small, so the converged
 * solution does not change; it only carries an impulsively started hypersonic flow through
 * its start-up transient at large CFL.
 * Method option: "ci_splitting" = 0 (default) splits the coupled operator's flux Jacobian
 * spectrally, A+- = (A +- lambda I)/2 (the paper's choice, Sec. 2.3); 1 uses the eigenvalue
 * splitting A+- = (A +- |A|)/2 with |A| = R |Lambda| R^-1 (the acoustic waves U_n +- c and
 * U_n for the rest), the viscous radius staying a scalar: the diagonal block becomes
 * (V/dtau + sum 2 lambda_vis) I + sum_d |A(S_d)| - V dS/dQ and the neighbours couple with
 * -(A + |A| + 2 lambda_vis)/2 and (A - |A| - 2 lambda_vis)/2.  The split operator is not
 * affected.
 * Method option: "transport" = 0 (default): Sutherland viscosity, conductivities from constant
 * Prandtl number 0.72, one diffusion coefficient rho D = mu / 0.5 for every species; 1: the
 * species model (air only; Sec. 2.1 defers transport data to its references and diffuses each
 * species with its own effective coefficient D_s): Blottner viscosity fits (Blottner, Johnson
 * & Ellis 1971; the ions take the fit of NO+), Eucken conductivities (two temperatures:
 * trans-rotational and vibrational-electronic parts), Wilke's mixing rule, hard-sphere binary
 * diffusion coefficients (first Chapman-Enskog approximation, diameters from the Blottner
 * viscosities) combined by Blanc's law into D_s, electrons diffusing with the ions (no net
 * charge flux) and a correction velocity so that the diffusive mass fluxes sum to zero; the
 * species radius takes max_s D_s (Eq. (vislambda)).  One more kernel per iteration.
 * Method option: "dtau_source" = 0 (default): V/dtau = sum_d (lambda_inv,d + lambda_vis,d) / CFL,
 * the source entering only through the diagonals (V max(0, -d omega_s/d rho_s) on the species,
 * the relaxation rate on the flow block's vibrational row); 1: the local time step of Sec. 2.2
 * with its source radius, V/dtau = (sum_d (lambda_inv,d + lambda_vis,d) + V lambda_S) / CFL,
 * lambda_S read as the largest magnitude on the source Jacobian's diagonal (max over species
 * of |d omega_s / d rho_s| and, 2T, the vibrational relaxation rate).  Both schemes; no effect
 * on a non-reacting grid.  The converged solution does not change.
 * Errors: CS_ERR_ARG for an unknown name, a negative / NaN update_limit, a ci_splitting,
 * transport or dtau_source other than 0 or 1, or the species model for a perfect gas. */
cs_status cs_set_option(cs_grid g, const char *name, double value);

/* Dual time stepping for unsteady flow (Sec. 2.3, the dual-time form of the implicit scheme).
 * With a physical step dt > 0 every residual (cs_residual, cs_step, batches) becomes
 *   R + V [(1+theta)(Q - Q^n) - theta (Q^n - Q^{n-1})] / dt
 * (its monitors too: the pseudo-time iterations converge it to zero) and (1+theta) V / dt is
 * added to every diagonal of both operators, where Q^n and Q^{n-1} are the last two physical
 * time levels.  theta = 0 is the implicit Euler step, theta = 1/2 the second-order three-level
 * backward difference (theta = 2, which the paper names for second order, is first order by
 * Taylor expansion).  cs_set_dual allocates the two levels on first use (2 x nq x ncell
 * doubles, library-owned), discards any stored levels and leaves the scheme steady until
 * cs_dual_advance begins the first physical step; dt = 0 switches dual time stepping off.
 * cs_dual_advance begins a physical step from the current state (Q^{n-1} <- Q^n, Q^n <- Q,
 * enqueued on the grid's stream); the first step after cs_set_dual uses theta = 0 (no
 * Q^{n-1} exists yet), the following ones theta.  A user loop: cs_set_dual once, then per
 * physical step cs_dual_advance and cs_step until the inner residual has dropped.
 * Errors: CS_ERR_ARG for a negative or non-finite dt or theta; CS_ERR_OOM if the levels cannot
 * be allocated; cs_dual_advance: CS_ERR_STATE while dual time stepping is off. */
cs_status cs_set_dual(cs_grid g, double dt, double theta);
cs_status cs_dual_advance(cs_grid g);

/* Residual monitors without device allocation (no counterpart in the paper: a service for
 * callers that cannot allocate device memory, e.g. an application whose memory pool already
 * holds the device, or monitoring code that must not let cudaMalloc / cudaFree synchronise the
 * device).  Computes norms_host[0] = r_species and norms_host[1] = r_energy exactly as
 * cs_residual does, from a residual R_dev (device, [nq][ncell], species rows first, energy row
 * nspecies + ndim) and cell volumes V_dev (device, [ncell]) owned by the caller.  Its scratch is
 * a static device array of CS_NORMS_STATIC_MAX_BLOCKS x 2 doubles (256 KiB) that every GPU
 * loading the library keeps until exit; ncell above CS_NORMS_STATIC_MAX_CELLS is rejected with
 * CS_ERR_ARG.  It allocates nothing: every call looks up the array's address in the current
 * context (cudaGetSymbolAddress); the first call in a context may load the library's device
 * code, so make that first call before any stream capture.  All calls share the array, so
 * calls that overlap on the GPU race; the call synchronises cuda_stream (NULL: legacy default
 * stream) before returning.  Errors: CS_ERR_ARG (null pointer, size, nspecies, ndim),
 * CS_ERR_CUDA. */
#define CS_NORMS_STATIC_MAX_BLOCKS 16384
#define CS_NORMS_STATIC_MAX_CELLS (CS_NORMS_STATIC_MAX_BLOCKS * 256)
cs_status cs_residual_norms_static(const double *R_dev, const double *V_dev, int ncell,
                                   int nspecies, int ndim, void *cuda_stream,
                                   double norms_host[2]);

const char *cs_last_error(cs_grid g);

/* ---- Batches of independent cases (no counterpart in the paper: many cases of uneven size
 * stepped together on one GPU) ----
 * A batch refers to grids the caller created and set up (cs_set_boundary done); it does not
 * own them, and they must outlive it.  cs_batch_step captures iters_per_graph iterations of
 * every case (each with its own cs_step_opts; the CFL ramp of each case is evaluated on the
 * device from the case's iteration count) into one CUDA graph, each case on a stream of the
 * batch, and replays the graph iters / iters_per_graph times; the cases run concurrently.  The
 * graph is kept and reused while the options and iters_per_graph stay the same.  Work the
 * caller queued on a grid's own stream completes before the batch runs, and the batch's work
 * has completed when a batch call returns.  Results are those of cs_step with the same options
 * (up to the rounding of the device-evaluated CFL ramp).
 * Errors: CS_ERR_ARG (null pointers, ncases < 1, a grid without boundary conditions, invalid
 * options, iters not a multiple of iters_per_graph), CS_ERR_CUDA (stream capture, graph
 * instantiation or launch failed), CS_ERR_OOM; after the run, the first case that ended in a
 * non-physical state or failed temperature solve gives CS_ERR_NONPHYSICAL / CS_ERR_NEWTON,
 * the per-case status being in stats[c].status_cell (-1: fine) and iters_done (0: failed). */
typedef struct cs_batch_s *cs_batch;
cs_status cs_batch_create(int ncases, const cs_grid *grids, cs_batch *out);
cs_status cs_batch_destroy(cs_batch b);
/* Autotuner: for every 2D case of the batch, time trials applications of the split sweep
 * operator (on the operator inputs of the current state; the state is not changed) for each
 * cluster kernel (1: direct loads, 2: hyperplane-ordered records) and each cluster size C in
 * {1, 2, 4, 8, 16} that fits the grid and the device, and keep the fastest (a smaller C wins
 * unless the larger one is more than 3 % faster).  choice_out (host [2 * ncases], nullable)
 * receives (kind, C) per case, (0, 0) where no cluster sweep applies (3D or periodic j). */
cs_status cs_batch_tune(cs_batch b, int precision, int trials, int *choice_out);
cs_status cs_batch_step(cs_batch b, const cs_step_opts *opts, int iters, int iters_per_graph,
                        cs_step_stats *stats);
/* ---- Chemistry surrogate network (no counterpart in the paper: it stands in for the
 * Arrhenius source and Jacobian-diagonal evaluation of Sec. 2.1 / Sec. 2.3.2 inside the
 * implicit operator only; the residual keeps the exact chemistry) ----
 * A 14-128-128-128-22 multilayer perceptron with SiLU hidden activations.  Parameters are one
 * FP32 vector of CS_MLP_NPARAM values in the order W1 [128][14], b1 [128], W2 [128][128], b2,
 * W3 [128][128], b3, W4 [22][128], b4 [22] (W row-major [out][in]); matrix products run on
 * the tensor cores with bfloat16 weights, inputs and activations and FP32 accumulation.
 * Inputs X are FP32 [n][14] and targets / outputs FP32 [n][22], device pointers, 1 <= n <=
 * max_batch.  Loss = mean over rows and outputs of (y - t)^2; training is Adam (beta1 0.9,
 * beta2 0.999, eps 1e-8) on the FP32 master parameters.
 * Errors: CS_ERR_ARG, CS_ERR_OOM, CS_ERR_CUDA, CS_ERR_TIMEOUT (a tensor-core completion wait
 * ran out; the network is then unusable). */
#define CS_MLP_IN 14
#define CS_MLP_HIDDEN 128
#define CS_MLP_OUT 22
#define CS_MLP_NPARAM 37782
typedef struct cs_mlp_s *cs_mlp;
cs_status cs_mlp_create(int max_batch, const float *params_host, cs_mlp *out);
cs_status cs_mlp_destroy(cs_mlp m);
cs_status cs_mlp_get_params(cs_mlp m, float *params_host);
cs_status cs_mlp_forward(cs_mlp m, const float *X_dev, int n, float *Y_dev);
/* loss and gradient (host [CS_MLP_NPARAM], nullable) of one batch, no update */
cs_status cs_mlp_grad(cs_mlp m, const float *X_dev, const float *T_dev, int n, float *grad_host,
                      double *loss_out);
/* one Adam step on one batch; loss_out (nullable) receives the loss before the step */
cs_status cs_mlp_train_step(cs_mlp m, const float *X_dev, const float *T_dev, int n, float lr,
                            double *loss_out);
const char *cs_mlp_last_error(cs_mlp m);

/* Solver coupling.  cs_surrogate_sample writes, for every cell of g, the raw features
 * [log10 rho, log10 T, log10 Tv, log10(Y_1 + 1e-10) .. log10(Y_11 + 1e-10)] (X_dev, FP32
 * [N][14]; -10 beyond the model's species) and the raw targets
 * [asinh(omega_s), asinh(max(0, -d omega_s / d rho_s))] (T_dev, FP32 [N][22]; SI units, the
 * derivative at fixed other conserved variables as in the operator, of which the operator uses
 * only this stiffness part; zero beyond the model's species) of the last primitive evaluation
 * (after cs_residual or cs_step).
 * cs_surrogate_attach makes every later iteration of g take the species Jacobian diagonal of
 * the split operator from the network instead of the exact chemistry (whose Jacobian is then
 * not evaluated; the residual keeps the exact source): inputs are standardised as
 * (raw - mean) / std with norm_host = [mean[14], std[14], target mean[22], target std[22]],
 * outputs de-standardised, held to [max(0, mean - 8 std), mean + 8 std] and passed through
 * sinh to give d omega_s / d rho_s = -sinh(t).  The network must hold at least N rows
 * (max_batch) and must not serve two grids that run at the same time.  cs_surrogate_detach
 * returns to the exact chemistry.  Errors: CS_ERR_ARG (null, too small a network, a std <= 0),
 * CS_ERR_OOM. */
cs_status cs_surrogate_sample(cs_grid g, float *X_dev, float *T_dev);
cs_status cs_surrogate_attach(cs_grid g, cs_mlp m, const double *norm_host);
cs_status cs_surrogate_detach(cs_grid g);

/* The batch's own stream (cudaStream_t): every graph launch of cs_batch_step is issued on it,
 * so CUDA events recorded on it before and after a cs_batch_step call bracket the batch's
 * device work.  The stream stays owned by the batch. */
cs_status cs_batch_stream(cs_batch b, void **stream_out);
const char *cs_batch_last_error(cs_batch b);

/* ---------------------------------------------------------------------------------------
 * Species-count scaling test (Sec. 3.1): one implicit step of the split (CS) or coupled (CI)
 * operator for a uniform, non-reacting flow of ns species in a Cartesian box, any ns.
 * Species s is calorically perfect: molar mass M_host[s] (kg/kmol), dof_host[s] translational-
 * rotational degrees of freedom (c_v,s = dof/2 R_u/M_s), mass fraction Y_host[s]; the flow
 * has temperature T (K), pressure p (Pa) and velocity u_host[3] (m/s); the box has
 * ni x nj x nk cells over size_host[3] (m), far field on every side (boundary neighbours add
 * nothing to the sweeps).  Radii are inviscid (the flow is uniform): lambda_F = |u.S| + c|S|,
 * lambda_C = |u.S|, V/dtau = sum lambda_F / cfl.
 * cs_species_box_step: rhs_dev = device [ns + 4][ncell] in the conserved layout (rho_1 ..
 * rho_ns, m_x, m_y, m_z, rho E); dQ_dev = device, split: [5 + ns][ncell] (rho, m, rho E,
 * rho_1 .. rho_ns), coupled: [4 + ns][ncell] (rho, m, rho E, rho_2 .. rho_ns).  The coupled
 * operator assembles and LU-factorises a dense (ns+4)^2 diagonal block per cell (library-owned,
 * allocated on first use; refused with CS_ERR_ARG above 32 GiB).  Synchronises the box's stream.
 * cs_species_box_time: the same step `reps` times on the box's stream, each bracketed by CUDA
 * events and preceded (outside the events) by a write of flush_bytes to flush_dev (a device
 * buffer larger than L2, or null with flush_bytes 0); ms_out receives the mean device time per
 * step.  It does not check the coupled factorisation: run cs_species_box_step first.
 * cs_species_box_state copies the box's conserved state into Q_dev ([ns + 4][ncell]).
 * Errors: CS_ERR_ARG (sizes, ns outside 1..65536, non-positive T, p, M, dof, negative Y, host
 * pointers where device ones are required), CS_ERR_OOM, CS_ERR_CUDA, CS_ERR_NONPHYSICAL (a
 * singular coupled block). */
typedef struct cs_species_box_s *cs_species_box;
cs_status cs_species_box_create(int ns, int ni, int nj, int nk, const double *size_host,
                                const double *M_host, const double *dof_host, const double *Y_host,
                                double T, double p, const double *u_host, cs_species_box *out);
cs_status cs_species_box_destroy(cs_species_box b);
cs_status cs_species_box_state(cs_species_box b, double *Q_dev);
cs_status cs_species_box_step(cs_species_box b, int scheme, double cfl, const double *rhs_dev,
                              double *dQ_dev);
cs_status cs_species_box_time(cs_species_box b, int scheme, double cfl, const double *rhs_dev,
                              double *dQ_dev, int reps, void *flush_dev, size_t flush_bytes,
                              double *ms_out);
const char *cs_species_box_last_error(cs_species_box b);

#ifdef __cplusplus
}
#endif
#endif /* CS_H */
