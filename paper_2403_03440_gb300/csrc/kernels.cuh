// CUDA kernels of one pseudo-time iteration of the component-splitting (CS) and coupled (CI)
// implicit LU-SGS scheme (arXiv:2403.03440, Sec. 2.2-2.3), FP64, for sm_103a.
//
// Data layout (HBM): cell c = i + ni*(j + nj*k); every per-cell array is struct-of-arrays
// [var][cell] so that a warp reads consecutive cells of one variable (coalesced).  Face arrays
// are [var][face] per direction.  The per-cell auxiliary array W holds everything the
// transcendental work produces (temperatures, transport, chemistry) so that the face kernels
// and the sweeps are purely algebraic: on GB300 the FP64 pipe, not HBM, bounds this path.
#pragma once
#include <cstdint>
#include <utility>

#include "gas.cuh"

namespace cs {

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_FARFIELD = 2, BC_OUTFLOW = 3, BC_AXIS = 4 };
enum { ST_OK = 0, ST_NONPHYSICAL = 4, ST_NEWTON = 5, ST_TIMEOUT = 6 };

// Per-cell auxiliary layout (offsets in units of N).
template <class G, int ND>
struct Aux {
  static constexpr int NS = G::NS;
  static constexpr int RHO = 0, U = 1, T = U + ND, TV = T + 1, P = TV + 1, C = P + 1,
                       BETA = C + 1, GAM = BETA + 1, EV = GAM + 1, H = EV + 1, CVTR = H + 1,
                       CVVE = CVTR + 1, CV = CVVE + 1, MU = CV + 1, KT = MU + 1, KV = KT + 1,
                       RHOD = KV + 1, PREV = RHOD + 1, RELAX = PREV + 1, OMV = RELAX + 1,
                       PY = OMV + 1, Y = PY + 1, PRS = Y + NS, HS = PRS + NS, EVE = HS + NS,
                       OM = EVE + NS, DOM = OM + NS, EMP = DOM + NS, RHODS = EMP + NS,
                       COUNT = RHODS + NS;
  static constexpr int NQ = NS + ND + 1 + (G::NTEMP == 2);
  static constexpr int NF = 1 + ND + 1 + (G::NTEMP == 2);
  static constexpr int NCI = NF + NS - 1;
  static constexpr int NG = ND + 1 + (G::NTEMP == 2) + NS;      // gradient variables
  static constexpr int NRC = NS + ND + 3 + (G::NTEMP == 2);      // reconstructed variables
};

struct DevGrid {
  int nd, ni, nj, nk, N;
  int bc[6];
  int limiter, react, hcorr, nojac;
  int cisplit;            // coupled operator: 0 spectral splitting, 1 eigenvalue splitting
  int transport;          // 0 Sutherland, constant Pr and Sc; 1 species model (k_transport)
  int dtau_src;           // 1: the source radius lambda_S joins the local time step (Sec. 2.2)
  double efix, Tw, ulim;
  int nf[3];
  const double* S[3];
  const double* fc[3];
  const double* V;
  const double* xc;       // [3][N]
  double* Q;              // [nq][N]
  double* W;              // [aux][N]
  double* fsW;            // freestream aux record [aux]
  double* grad;           // [ng*3][N]
  double* F[3];           // [nq][nf]
  double* eta[3];         // [nf] H-correction eta of every face (k_eta)
  double* R;              // [nq][N]
  double* lamF;           // [3][N]
  double* lamC;
  double* lamCI;
  double* DF;
  double* DFev;
  double* Ds;             // [ns][N]
  double* DLU;            // [N][nci*nci]
  int* piv;               // [N][nci]
  double* DINV;           // [N][nci*nci] inverse of the coupled diagonal block (row-major)
  double* CIM;            // 2D coupled neighbour blocks of k_ci_mat (cell and row records) or null
  double* dQs;            // [nsplit][N]
  double* dQ;
  double* dQcs;           // [nci][N]
  double* dQc;
  double* red;            // reduction scratch
  double* Vdt;            // [N] V / dtau
  double* invD;           // [2 + ns][N]: 1/D_F, 1/D_F,ev, 1/D_s
  double* rhsF;           // [nF][N]: -(sum_s R_s, R_m, R_E, [R_ev])
  double* SMC;            // 2D split-sweep couplings of k_sweep_mat (cell and row records) or null
  // 2D wavefront sweep: per-cell sweep records in hyperplane order (w = woff[h] + j - jlo(h))
  const int* woff;        // [H + 2]
  void* wrec;             // flow records [N][kRecF] (compute type)
  void* wrecs;            // species-group records [groups][N][kRecS]
  void* wbase;            // forward results in hyperplane order: flow [N][8], species [groups][N][4]
  int* status;            // [0] code, [1] cell, [2] clip count
  const double* params;   // [0] cfl, [1] (1+theta)/dt, [2] theta/dt (dual time; 0: steady)
  const double* Qn;       // dual time stepping: physical levels Q^n, Q^{n-1} [nq][N] (or null)
  const double* Qnm1;
};

__device__ __forceinline__ void set_status(const DevGrid& g, int code, int cell) {
  if (atomicCAS(&g.status[0], 0, code) == 0) g.status[1] = cell;
}

__device__ __forceinline__ void cell_ijk(const DevGrid& g, int c, int& i, int& j, int& k) {
  i = c % g.ni;
  j = (c / g.ni) % g.nj;
  k = c / (g.ni * g.nj);
}
__device__ __forceinline__ int cell_of(const DevGrid& g, int i, int j, int k) {
  return i + g.ni * (j + g.nj * k);
}
// face index along direction d of the face at the low side of (i,j,k) (+1 on d for high side)
__device__ __forceinline__ int face_of(const DevGrid& g, int d, int i, int j, int k) {
  const int fi = g.ni + (d == 0), fj = g.nj + (d == 1);
  return i + fi * (j + fj * k);
}
__device__ __forceinline__ int coord(int d, int i, int j, int k) {
  return d == 0 ? i : (d == 1 ? j : k);
}
__device__ __forceinline__ int extent(const DevGrid& g, int d) {
  return d == 0 ? g.ni : (d == 1 ? g.nj : g.nk);
}

// Neighbour across side s (-1/+1) of direction d; -1 at a non-periodic boundary.
// lower = neighbour precedes the cell in h = i+j+k order.
__device__ __forceinline__ int neighbour(const DevGrid& g, int i, int j, int k, int d, int s,
                                         bool& lower) {
  int p[3] = {i, j, k};
  const int n = extent(g, d);
  int q = p[d] + s;
  if (q < 0 || q >= n) {
    if (g.bc[2 * d + (s > 0)] != BC_PERIODIC) return -1;
    q = (q + n) % n;
  }
  lower = q < p[d];
  p[d] = q;
  return cell_of(g, p[0], p[1], p[2]);
}

__device__ __forceinline__ const double* face_vec(const DevGrid& g, int d, int i, int j, int k,
                                                  int s) {
  int p[3] = {i, j, k};
  if (s > 0) p[d]++;
  return g.S[d] + 3 * (size_t)face_of(g, d, p[0], p[1], p[2]);
}

// ---------------------------------------------------------------------------------------
// Thermodynamic state of one cell (Sec. 2.1)
// ---------------------------------------------------------------------------------------

// Mixture energy in the one-temperature model: e(T) and c_v(T) per unit mass.
template <class G>
__device__ __forceinline__ void mix_e1(const double* Y, double T, double& e, double& cv) {
  e = 0.0;
  cv = 0.0;
  const double iT = 1.0 / T;
#pragma unroll
  for (int s = 0; s < G::NS; ++s) {
    double ev, cvv, em;
    vib_it<G>(s, iT, ev, cvv, em);
    e += Y[s] * (cvtr<G>(s) * T + ev + hf<G>(s));
    cv += Y[s] * (cvtr<G>(s) + cvv);
  }
}
// Vibrational-electronic pool energy (2T) and its heat capacity.
template <class G>
__device__ __forceinline__ void mix_pool(const double* Y, double Tv, double& e, double& cv) {
  e = 0.0;
  cv = 0.0;
  const double iTv = 1.0 / Tv;
#pragma unroll
  for (int s = 0; s < G::NS; ++s) {
    if (G::sp(s).kind == ELECTRON) {
      e += Y[s] * 1.5 * Rs<G>(s) * Tv;
      cv += Y[s] * 1.5 * Rs<G>(s);
    } else {
      double ev, cvv, em;
      vib_it<G>(s, iTv, ev, cvv, em);
      e += Y[s] * ev;
      cv += Y[s] * cvv;
    }
  }
}

// Mixture energy (1T: e(T), POOL: the vibrational-electronic pool e_v(Tv)) and its heat
// capacity in FP32: the predictor of the temperature solves.
template <class G, bool POOL>
__device__ __forceinline__ void mix_f32(const float* Y, float T, float& e, float& cv) {
  e = 0.0f;
  cv = 0.0f;
  const float iT = 1.0f / T;
#pragma unroll
  for (int s = 0; s < G::NS; ++s) {
    const SpeciesData& d = G::sp(s);
    const float R = c_gas.Rsf[s];
    float ev = 0.0f, cvv = 0.0f;
    if (d.kind == ELECTRON && POOL) {
      ev = 1.5f * R * T;
      cvv = 1.5f * R;
    } else if (d.kind == DIATOMIC && d.thv > 0.0) {
      const float x = c_gas.thvf[s] * iT, em = __expf(-x), r = 1.0f / (1.0f - em);
      ev = R * c_gas.thvf[s] * em * r;
      cvv = R * x * x * em * r * r;
    }
    if (POOL) {
      e += Y[s] * ev;
      cv += Y[s] * cvv;
    } else {
      const float ct = d.kind == DIATOMIC ? 2.5f * R : 1.5f * R;
      e += Y[s] * (ct * T + ev + c_gas.hff[s]);
      cv += Y[s] * (ct + cvv);
    }
  }
}

// Safeguarded Newton for a monotone energy: returns 0 on convergence, 1 otherwise.  The
// energies at the bracket ends [kTmin, kTmax] are evaluated only when a Newton step leaves the
// bracket (a state below / above them is clamped to the end, as in a plain bracketed solve).
// An FP32 Newton predictor first brings the guess to ~1e-6 relative (where the warm start is
// not already that close); the FP64 iteration then stops when a Newton step is at most 1e-8 T
// (quadratic convergence puts the new iterate within ~1e-16 T, the accuracy the bracketed
// solve's own test |dT| <= 1e-12 T gives one iteration later) or a bisection step is at most
// 1e-12 T.  Fewer FP64 iterations, and fewer lanes of a warp idling while others iterate.
template <class G, bool POOL>
__device__ int solve_temperature(const double* Y, double target, double guess, double& Tout) {
  double lo = kTmin, hi = kTmax, e, cv;
  // (the loop below counts the bracket-end evaluations as passes: 200 Newton / bisection
  // steps plus at most two end checks)
  bool lo_checked = false, hi_checked = false;
  double T = (guess > lo && guess < hi) ? guess : 1000.0;
  {
    float Yf[G::NS];
#pragma unroll
    for (int s = 0; s < G::NS; ++s) Yf[s] = (float)Y[s];
    const float tf = (float)target;
    float Tf = (float)T;
    bool ok = true;
#pragma unroll 1
    for (int it = 0; it < 12; ++it) {
      float ef, cf;
      mix_f32<G, POOL>(Yf, Tf, ef, cf);
      const float dT = (tf - ef) / cf;
      const float Tn = Tf + dT;
      if (!(Tn > (float)kTmin && Tn < (float)kTmax)) { ok = false; break; }
      Tf = Tn;
      if (fabsf(dT) <= 3e-6f * Tf) break;
    }
    if (ok && fabs((double)Tf - T) > 3e-6 * T) T = (double)Tf;
  }
  // One energy evaluation per pass of the loop: at the Newton iterate, or (check = 1 / 2) at a
  // bracket end the iterate has stepped past, evaluated once each.
  int check = 0;
#pragma unroll 1
  for (int it = 0; it < 202; ++it) {
    const double Te = check == 1 ? kTmin : (check == 2 ? kTmax : T);
    if (POOL) mix_pool<G>(Y, Te, e, cv); else mix_e1<G>(Y, Te, e, cv);
    double Tn;
    bool newton;
    if (check) {
      if (check == 1) {
        lo_checked = true;
        if (e >= target) { Tout = kTmin; return 0; }
      } else {
        hi_checked = true;
        if (e <= target) { Tout = kTmax; return 1; }
      }
      check = 0;
      Tn = 0.5 * (lo + hi);
      newton = false;
    } else {
      const double f = e - target;
      if (f > 0) hi = T; else lo = T;
      Tn = (cv > 0) ? T - f / cv : 0.5 * (lo + hi);
      newton = cv > 0;
      // A Newton step of at most 1e-8 T has converged even where it lands on, or by rounding
      // just past, the bracket end that T itself has just become: at the exact root (f == 0,
      // e.g. the warm start of an unchanged cell) T becomes the lower end and Tn == T, which
      // the open-bracket test below would send into a bisection towards kTmax and a dozen
      // more passes back.
      if (newton && fabs(Tn - T) <= 1e-8 * T) {
        Tout = fmin(fmax(Tn, kTmin), kTmax);
        return 0;
      }
      if (!(Tn > lo && Tn < hi)) {
        if (Tn <= lo && lo == kTmin && !lo_checked) { check = 1; continue; }
        if (Tn >= hi && hi == kTmax && !hi_checked) { check = 2; continue; }
        Tn = 0.5 * (lo + hi);
        newton = false;
      }
    }
    const double step = fabs(Tn - T);
    if (step <= 1e-12 * T || (newton && step <= 1e-8 * T)) { Tout = Tn; return 0; }
    T = Tn;
  }
  Tout = T;
  return 1;
}

// Register-resident primitive record.
template <class G, int ND>
struct Prim {
  double rhos[G::NS], Y[G::NS], rho, u[ND], T, Tv, p, c, beta, rhoE, rhoev, ev, H, Gam;
  double prs[G::NS], prev, cvtr, cvve, cv, mu, kt, kv, rhoD, hs[G::NS], eve[G::NS];
  double emP[G::NS];   // exp(-theta_v/T) at the vibrational temperature (Tv, or T in 1T)
};

// Conserved -> primitive.  Returns ST_OK, ST_NONPHYSICAL or ST_NEWTON.  With STORE the
// per-species results (Y, prs, hs, eve, emP) are also written to the auxiliary array as they
// are produced (Wc = &W[cell], stride N), so that they need not stay in registers until the
// record is stored; the caller then stores the scalars (store_prim_scalars).
template <class G, int ND, bool STORE = false>
__device__ int primitive(const double* q, double Tguess, double Tvguess, Prim<G, ND>& w,
                         double* Wc = nullptr, size_t N = 0) {
  using A = Aux<G, ND>;
  constexpr int NS = G::NS;
  double rho = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    w.rhos[s] = q[s];
    if (q[s] < 0.0) return ST_NONPHYSICAL;
    rho += q[s];
  }
  if (!(rho > 0.0)) return ST_NONPHYSICAL;
  w.rho = rho;
  const double irho = 1.0 / rho;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    w.Y[s] = w.rhos[s] * irho;
    if (STORE) Wc[(A::Y + s) * N] = w.Y[s];
  }
  double ke = 0.0;
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    w.u[d] = q[NS + d] * irho;
    ke += 0.5 * w.u[d] * w.u[d];
  }
  w.rhoE = q[NS + ND];
  const double rhoe = w.rhoE - rho * ke;
  int st;
  if (G::NTEMP == 1) {
    double T;
    st = solve_temperature<G, false>(w.Y, rhoe * irho, Tguess, T);
    w.T = w.Tv = T;
    w.rhoev = 0.0;
    w.ev = 0.0;
  } else {
    w.rhoev = q[NS + ND + 1];
    w.ev = w.rhoev * irho;
    double Tv;
    st = solve_temperature<G, true>(w.Y, w.ev, Tvguess > 0 ? Tvguess : Tguess, Tv);
    w.Tv = Tv;
    double etr = rhoe - w.rhoev, ct = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      etr -= w.rhos[s] * hf<G>(s);
      ct += w.rhos[s] * cvtr<G>(s);
    }
    w.T = etr / ct;
    if (!(w.T > kTmin)) w.T = kTmin;   // floor, as the temperature solves
  }
  if (st) return ST_NEWTON;
  const double T = w.T, Tv = w.Tv;
  const double iTp = 1.0 / (G::NTEMP == 2 ? Tv : T);
  double p = 0.0, Rh = 0.0, cvt = 0.0, cvve = 0.0, cv = 0.0, pe = 0.0;
  double evs[NS], cvvs[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const bool elec = G::sp(s).kind == ELECTRON;
    const double R = Rs<G>(s);
    if (G::NTEMP == 2 && elec) {
      p += w.rhos[s] * R * Tv;
      pe += w.rhos[s] * R;
      evs[s] = 1.5 * R * Tv;
      cvvs[s] = 1.5 * R;
      w.emP[s] = 0.0;
    } else {
      p += w.rhos[s] * R * T;
      Rh += w.Y[s] * R;
      vib_it<G>(s, iTp, evs[s], cvvs[s], w.emP[s]);
    }
    if (STORE) Wc[(A::EMP + s) * N] = w.emP[s];
    cvt += w.Y[s] * cvtr<G>(s);
    if (G::NTEMP == 2) cvve += w.Y[s] * cvvs[s];
    else cv += w.Y[s] * (cvtr<G>(s) + cvvs[s]);
  }
  w.p = p;
  w.cvtr = cvt;
  w.cvve = cvve;
  w.cv = cv;
  const double beta = (G::NTEMP == 2) ? Rh / cvt : Rh / cv;
  w.beta = beta;
  double pefac = 0.0;
  if (G::NTEMP == 2) {
    pefac = (cvve > 0.0) ? pe / (rho * cvve) : 0.0;
    w.prev = -beta + pefac;
  } else {
    w.prev = 0.0;
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const bool elec = G::sp(s).kind == ELECTRON;
    const double R = Rs<G>(s);
    if (G::NTEMP == 1) {
      const double es = cvtr<G>(s) * T + evs[s] + hf<G>(s);
      w.prs[s] = R * T + beta * (ke - es);
      w.hs[s] = es + R * T;
      w.eve[s] = 0.0;
    } else {
      w.prs[s] = beta * (ke - hf<G>(s) - cvtr<G>(s) * T) - pefac * evs[s] +
                 (elec ? R * Tv : R * T);
      const double es = cvtr<G>(s) * T + evs[s] + hf<G>(s);
      w.hs[s] = es + R * (elec ? Tv : T);
      w.eve[s] = elec ? 2.5 * R * Tv : evs[s];
    }
    if (STORE) {
      Wc[(A::PRS + s) * N] = w.prs[s];
      Wc[(A::HS + s) * N] = w.hs[s];
      Wc[(A::EVE + s) * N] = w.eve[s];
    }
  }
  w.c = sqrt((1.0 + beta) * p * irho);
  w.H = (w.rhoE + p) * irho;
  w.Gam = rhoe / p;
  w.mu = kSuthMu * T * sqrt(T) / (T + kSuthT);
  if (G::NTEMP == 2) {
    w.kt = w.mu * (cvt + Rh) * kInvPr;
    w.kv = w.mu * cvve * kInvPr;
  } else {
    w.kt = w.mu * (cv + Rh) * kInvPr;
    w.kv = 0.0;
  }
  w.rhoD = w.mu * kInvSc;
  return ST_OK;
}

// the scalar fields of the record (the per-species ones: primitive<G, ND, true>)
template <class G, int ND>
__device__ __forceinline__ void store_prim_scalars(const DevGrid& g, int c, const Prim<G, ND>& w) {
  using A = Aux<G, ND>;
  double* W = g.W;
  const size_t N = g.N;
  W[A::RHO * N + c] = w.rho;
#pragma unroll
  for (int d = 0; d < ND; ++d) W[(A::U + d) * N + c] = w.u[d];
  W[A::T * N + c] = w.T;
  W[A::TV * N + c] = w.Tv;
  W[A::P * N + c] = w.p;
  W[A::C * N + c] = w.c;
  W[A::BETA * N + c] = w.beta;
  W[A::GAM * N + c] = w.Gam;
  W[A::EV * N + c] = w.ev;
  W[A::H * N + c] = w.H;
  W[A::CVTR * N + c] = w.cvtr;
  W[A::CVVE * N + c] = w.cvve;
  W[A::CV * N + c] = w.cv;
  W[A::MU * N + c] = w.mu;
  W[A::KT * N + c] = w.kt;
  W[A::KV * N + c] = w.kv;
  W[A::RHOD * N + c] = w.rhoD;
  W[A::PREV * N + c] = w.prev;
}

template <class G, int ND>
__device__ __forceinline__ void store_prim(const DevGrid& g, int c, const Prim<G, ND>& w) {
  using A = Aux<G, ND>;
  double* W = g.W;
  const size_t N = g.N;
  W[A::RHO * N + c] = w.rho;
#pragma unroll
  for (int d = 0; d < ND; ++d) W[(A::U + d) * N + c] = w.u[d];
  W[A::T * N + c] = w.T;
  W[A::TV * N + c] = w.Tv;
  W[A::P * N + c] = w.p;
  W[A::C * N + c] = w.c;
  W[A::BETA * N + c] = w.beta;
  W[A::GAM * N + c] = w.Gam;
  W[A::EV * N + c] = w.ev;
  W[A::H * N + c] = w.H;
  W[A::CVTR * N + c] = w.cvtr;
  W[A::CVVE * N + c] = w.cvve;
  W[A::CV * N + c] = w.cv;
  W[A::MU * N + c] = w.mu;
  W[A::KT * N + c] = w.kt;
  W[A::KV * N + c] = w.kv;
  W[A::RHOD * N + c] = w.rhoD;
  W[A::PREV * N + c] = w.prev;
#pragma unroll
  for (int s = 0; s < G::NS; ++s) {
    W[(A::Y + s) * N + c] = w.Y[s];
    W[(A::PRS + s) * N + c] = w.prs[s];
    W[(A::HS + s) * N + c] = w.hs[s];
    W[(A::EVE + s) * N + c] = w.eve[s];
    W[(A::EMP + s) * N + c] = w.emP[s];
  }
}

// ---------------------------------------------------------------------------------------
// Chemistry (Sec. 2.1 source; Park air).  k_b = k_f(T_b)/K_c(T_b) in log space, K_c from the
// species' RRHO Gibbs energies.  Derivatives: d omega/d rho at fixed T, Tv and d omega/dT,
// d omega/dTv, giving the conserved-variable source Jacobian A_S of Sec. 2.2.
// ---------------------------------------------------------------------------------------

// g_s/(R_u T) and H_s/(R_u T) at the standard pressure, simplified form (translational,
// rotational and vibrational enthalpy terms cancel between H/RT and S/R); em = exp(-theta_v/T)
// and r = 1/(1 - em) are supplied by the caller, iT = 1/T.
template <class G>
__device__ __forceinline__ void gibbs(int s, double iT, double lnT, double em, double r,
                                      double& gRT, double& hRT) {
  const SpeciesData& d = G::sp(s);
  const double hr = d.h0 * iT * kInvRu;
  double g = hr - 2.5 * lnT + c_gas.gc0[s];
  double h = 2.5 + hr;
  if (d.kind == DIATOMIC) {
    g -= lnT;
    h += 1.0;
    if (d.thv > 0.0) {
      const double x = d.thv * iT;
      g += log_tab(1.0 - em);
      h += x * em * r;
    }
  }
  gRT = g;
  hRT = h;
}

// exp(-theta_v/T) of every diatomic species (0 for the others)
template <class G>
__device__ __forceinline__ void vib_exp(double iT, double* em) {
#pragma unroll
  for (int s = 0; s < G::NS; ++s) {
    const SpeciesData& d = G::sp(s);
    em[s] = (d.kind == DIATOMIC && d.thv > 0.0) ? exp_tab(-d.thv * iT) : 0.0;
  }
}
// 1/(1 - em) of every species
template <class G>
__device__ __forceinline__ void vib_rcp(const double* em, double* r) {
#pragma unroll
  for (int s = 0; s < G::NS; ++s) {
    const SpeciesData& d = G::sp(s);
    r[s] = (d.kind == DIATOMIC && d.thv > 0.0) ? 1.0 / (1.0 - em[s]) : 1.0;
  }
}
// harmonic-oscillator energy and heat capacity from em = exp(-theta/T) and r = 1/(1 - em)
template <class G>
__device__ __forceinline__ void vib_em(int s, double iT, double em, double r, double& e, double& cv) {
  const SpeciesData& d = G::sp(s);
  if (d.kind != DIATOMIC || d.thv <= 0.0) { e = 0.0; cv = 0.0; return; }
  const double x = d.thv * iT, Rem = c_gas.Rs[s] * em * r;
  e = Rem * d.thv;
  cv = Rem * x * x * r;
}

__device__ __forceinline__ double rate_temp(int kind, double T, double Tv) {
  return kind == TK_A ? sqrt(T * Tv) : (kind == TK_V ? Tv : T);
}

// omega[s]; optionally the fixed-T Jacobian diagonal jd[s] = d omega_s/d rho_s, the full
// fixed-T Jacobian J[s*NS+r] and the temperature derivatives wT[s], wTv[s].
// Working set of the chemistry evaluation (registers after inlining).
template <class G, bool FULL>
struct ChemCtx {
  static constexpr int NS = G::NS;
  double X[NS], gT[NS], hT[NS], gV[NS], hV[NS];
  double omega[NS], jd[NS], wT[NS], wTv[NS];
  double J[FULL ? NS * NS : 1];
  double lnT, lnTv, lnTa, iT, iTv, iTa, lnPT, lnPTv, T, Tv, Ta;
};

template <int K>
__device__ __forceinline__ void pick_temp(double T, double Tv, double Ta, double lnT, double lnTv,
                                          double lnTa, double iT, double iTv, double iTa,
                                          double& Tk, double& lnTk, double& iTk) {
  if (K == TK_T) { Tk = T; lnTk = lnT; iTk = iT; }
  else if (K == TK_V) { Tk = Tv; lnTk = lnTv; iTk = iTv; }
  else { Tk = Ta; lnTk = lnTa; iTk = iTa; }
}

struct RxTerms {
  double kf, kb, M, Pf, Pb, net, dRT, dRV;
};

// d(product of the concentrations of a species list)/dX_q, repeats handled
template <int RI>
__device__ __forceinline__ double dprod_f(const double* X, int q) {
  constexpr RxShape x = rx_shape(RI);
  double v = 0.0;
  if (x.r0 == q) v += (x.nr > 1) ? X[x.r1] : 1.0;
  if (x.nr > 1 && x.r1 == q) v += X[x.r0];
  return v;
}
template <int RI>
__device__ __forceinline__ double dprod_b(const double* X, int q) {
  constexpr RxShape x = rx_shape(RI);
  double v = 0.0;
  if (x.p0 == q) v += (x.np > 1 ? X[x.p1] : 1.0) * (x.np > 2 ? X[x.p2] : 1.0);
  if (x.np > 1 && x.p1 == q) v += X[x.p0] * (x.np > 2 ? X[x.p2] : 1.0);
  if (x.np > 2 && x.p2 == q) v += X[x.p0] * X[x.p1];
  return v;
}

// contribution of reaction RI to species S (nothing when S does not change in RI); JAC =
// false: the source only, no derivatives
template <class G, bool FULL, bool JAC, int RI, int S>
__device__ __forceinline__ void species_term(ChemCtx<G, FULL>& c, const RxTerms& t) {
  constexpr int nu = rx_nu(RI, S);
  if constexpr (nu != 0) {
    constexpr int NS = G::NS;
    constexpr RxShape x = rx_shape(RI);
    const ReactionData& d = c_reactions[RI];
    const double Ms = G::sp(S).M;
    c.omega[S] += Ms * nu * t.net;
    if constexpr (!JAC) return;
    c.wT[S] += Ms * nu * t.dRT;
    c.wTv[S] += Ms * nu * t.dRV;
    if (FULL) {
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        const double e = x.third ? d.eff[q] : 0.0;
        const double dRf = t.kf * (dprod_f<RI>(c.X, q) * t.M + t.Pf * e);
        const double dRb = t.kb * (dprod_b<RI>(c.X, q) * t.M + t.Pb * e);
        c.J[S * NS + q] += Ms * nu * (dRf - dRb) * c_gas.invM[q];
      }
    } else {
      const double e = x.third ? d.eff[S] : 0.0;
      c.jd[S] += nu * (t.kf * (dprod_f<RI>(c.X, S) * t.M + t.Pf * e) -
                       t.kb * (dprod_b<RI>(c.X, S) * t.M + t.Pb * e));
    }
  }
}
template <class G, bool FULL, bool JAC, int RI, int... S>
__device__ __forceinline__ void species_terms(ChemCtx<G, FULL>& c, const RxTerms& t,
                                              std::integer_sequence<int, S...>) {
  (species_term<G, FULL, JAC, RI, S>(c, t), ...);
}

// One reaction, unrolled at compile time (species indices are constants).
template <class G, bool FULL, bool JAC, int RI>
__device__ __forceinline__ void reaction(ChemCtx<G, FULL>& c) {
  constexpr RxShape x = rx_shape(RI);
  constexpr int NS = G::NS;
  const ReactionData& d = c_reactions[RI];
  constexpr bool bv = x.tb == TK_V;
  double sg = 0.0, sh = 0.0;
  int dn = 0;
  // products minus reactants of nu g/RT and nu h/RT at the backward temperature
  const double* gB = bv ? c.gV : c.gT;
  const double* hB = bv ? c.hV : c.hT;
  sg += gB[x.p0]; sh += hB[x.p0]; ++dn;
  if (x.np > 1) { sg += gB[x.p1]; sh += hB[x.p1]; ++dn; }
  if (x.np > 2) { sg += gB[x.p2]; sh += hB[x.p2]; ++dn; }
  sg -= gB[x.r0]; sh -= hB[x.r0]; --dn;
  if (x.nr > 1) { sg -= gB[x.r1]; sh -= hB[x.r1]; --dn; }
  const double lnKc = -sg + dn * (bv ? c.lnPTv : c.lnPT);
  double Tf, lnTf, iTf, Tb, lnTb, iTb;
  pick_temp<x.tf>(c.T, c.Tv, c.Ta, c.lnT, c.lnTv, c.lnTa, c.iT, c.iTv, c.iTa, Tf, lnTf, iTf);
  pick_temp<x.tb>(c.T, c.Tv, c.Ta, c.lnT, c.lnTv, c.lnTa, c.iT, c.iTv, c.iTa, Tb, lnTb, iTb);
  const double kf = exp_tab(d.lnA + d.n * lnTf - d.theta * iTf);
  const double kb = exp_tab(d.lnA + d.n * lnTb - d.theta * iTb - lnKc);
  double M = 1.0;
  if (x.third) {
    M = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) M += d.eff[s] * c.X[s];
  }
  double Pf = c.X[x.r0];
  if (x.nr > 1) Pf *= c.X[x.r1];
  double Pb = c.X[x.p0];
  if (x.np > 1) Pb *= c.X[x.p1];
  if (x.np > 2) Pb *= c.X[x.p2];
  const double Rf = kf * Pf * M, Rb = kb * Pb * M;
  if constexpr (!JAC) {
    species_terms<G, FULL, JAC, RI>(c, RxTerms{kf, kb, M, Pf, Pb, Rf - Rb, 0.0, 0.0},
                                    std::make_integer_sequence<int, NS>{});
    return;
  }
  const double dlf = (d.n + d.theta * iTf) * iTf;
  const double dlb = (d.n + d.theta * iTb - (sh - dn)) * iTb;
  constexpr bool fA = x.tf == TK_A, bA = x.tb == TK_A;
  const double fT = x.tf == TK_T ? 1.0 : (fA ? 0.5 * Tf * c.iT : 0.0);
  const double fV = x.tf == TK_V ? 1.0 : (fA ? 0.5 * Tf * c.iTv : 0.0);
  const double bT = x.tb == TK_T ? 1.0 : (bA ? 0.5 * Tb * c.iT : 0.0);
  const double bVv = x.tb == TK_V ? 1.0 : (bA ? 0.5 * Tb * c.iTv : 0.0);
  const double dRT = Rf * dlf * fT - Rb * dlb * bT;
  const double dRV = Rf * dlf * fV - Rb * dlb * bVv;
  const double net = Rf - Rb;
  species_terms<G, FULL, JAC, RI>(c, RxTerms{kf, kb, M, Pf, Pb, net, dRT, dRV},
                                  std::make_integer_sequence<int, NS>{});
}

template <class G, bool FULL, bool JAC, int... RI>
__device__ __forceinline__ void all_reactions(ChemCtx<G, FULL>& c, std::integer_sequence<int, RI...>) {
  (reaction<G, FULL, JAC, RI>(c), ...);
}

// omega[s]; the fixed-T Jacobian diagonal jd[s] = d omega_s/d rho_s (or the full fixed-T
// Jacobian J[s*NS+r] when FULL) and the temperature derivatives wT[s], wTv[s] (all zero when
// JAC is false: the source alone).
// emT/emTv: exp(-theta_v/T) and exp(-theta_v/Tv) of every species (vib_exp), rT/rV their
// 1/(1 - em) (vib_rcp).
template <class G, bool FULL, bool JAC = true>
__device__ __forceinline__ void chemistry(const double* rhos, double T, double Tv, const double* emT,
                                          const double* emTv, const double* rT, const double* rV,
                                          double* omega, double* jd, double* J, double* wT,
                                          double* wTv) {
  constexpr int NS = G::NS;
  ChemCtx<G, FULL> c;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    c.X[s] = rhos[s] * c_gas.invM[s];
    c.omega[s] = 0.0;
    c.jd[s] = 0.0;
    c.wT[s] = 0.0;
    c.wTv[s] = 0.0;
  }
  if (FULL)
#pragma unroll
    for (int k = 0; k < NS * NS; ++k) c.J[k] = 0.0;
  c.T = T;
  c.Tv = Tv;
  c.lnT = log_tab(T);
  c.lnTv = (G::NTEMP == 2) ? log_tab(Tv) : c.lnT;
  c.iT = 1.0 / T;
  c.iTv = (G::NTEMP == 2) ? 1.0 / Tv : c.iT;
  c.lnTa = 0.5 * (c.lnT + c.lnTv);
  c.Ta = (G::NTEMP == 2) ? sqrt(T * Tv) : T;
  c.iTa = (G::NTEMP == 2) ? 1.0 / c.Ta : c.iT;
  c.lnPT = c_gas.lnPRu - c.lnT;
  c.lnPTv = c_gas.lnPRu - c.lnTv;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    gibbs<G>(s, c.iT, c.lnT, emT[s], rT[s], c.gT[s], c.hT[s]);
    if (G::NTEMP == 2) gibbs<G>(s, c.iTv, c.lnTv, emTv[s], rV[s], c.gV[s], c.hV[s]);
    else { c.gV[s] = c.gT[s]; c.hV[s] = c.hT[s]; }
  }
  all_reactions<G, FULL, JAC>(c, std::make_integer_sequence<int, G::NR>{});
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    omega[s] = c.omega[s];
    wT[s] = c.wT[s];
    wTv[s] = c.wTv[s];
    jd[s] = FULL ? c.J[s * NS + s] : c.jd[s];
  }
  if (FULL)
#pragma unroll
    for (int k = 0; k < NS * NS; ++k) J[k] = c.J[k];
}

// Derivatives of T and Tv with respect to rho_s at fixed other conserved variables; irc =
// 1/(rho c_v) (1T) or 1/(rho c_v,tr) (2T), ircv = 1/(rho c_v,ve) (0 without a pool).
template <class G, int ND>
__device__ __forceinline__ void dT_drho_r(const Prim<G, ND>& w, int s, double evs, double irc,
                                          double ircv, double& dT, double& dTv) {
  double ke = 0.0;
#pragma unroll
  for (int d = 0; d < ND; ++d) ke += 0.5 * w.u[d] * w.u[d];
  if (G::NTEMP == 1) {
    const double es = cvtr<G>(s) * w.T + evs + hf<G>(s);
    dT = (ke - es) * irc;
    dTv = dT;
  } else {
    dT = (ke - hf<G>(s) - cvtr<G>(s) * w.T) * irc;
    dTv = -evs * ircv;
  }
}
template <class G, int ND>
__device__ __forceinline__ void dT_drho_recips(const Prim<G, ND>& w, double& irc, double& ircv) {
  irc = 1.0 / (w.rho * (G::NTEMP == 1 ? w.cv : w.cvtr));
  ircv = (G::NTEMP == 2 && w.cvve > 0.0) ? 1.0 / (w.rho * w.cvve) : 0.0;
}
template <class G, int ND>
__device__ __forceinline__ void dT_drho(const Prim<G, ND>& w, int s, double evs, double& dT,
                                        double& dTv) {
  double irc, ircv;
  dT_drho_recips<G, ND>(w, irc, ircv);
  dT_drho_r<G, ND>(w, s, evs, irc, ircv, dT, dTv);
}

// Millikan-White + Park vibrational relaxation (2T): the Landau-Teller part of the vibrational
// source (lt) and the relaxation diagonal (relax).  The chemistry-vibration coupling
// sum_s omega_s e_p,s is added by vib_coupling once the species sources are known.
// emT/emTv: exp(-theta_v/T), exp(-theta_v/Tv) per species; rT/rV: their 1/(1 - em).
template <class G, int ND>
__device__ void vib_relax(const Prim<G, ND>& w, const double* emT, const double* emTv,
                          const double* rT, const double* rV, double& lt_out, double& relax) {
  constexpr int NS = G::NS;
  double X[NS], xs = 0.0, ph = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    X[s] = 0.0;
    if (G::sp(s).kind == ELECTRON) continue;
    X[s] = w.rhos[s] * c_gas.invM[s];
    xs += X[s];
    ph += w.rhos[s] * Rs<G>(s) * w.T;
  }
  const double patm = ph * kInvPref, nden = xs * kNa, T13 = rcbrt(w.T);
  const double iT = 1.0 / w.T, iTv = 1.0 / w.Tv, sqT = sqrt(w.T);
  const double sv = 1e-21 * (50000.0 * iT) * (50000.0 * iT);
  // Park's collision-limited time 1/(n sigma cbar): cbar = cbk_s sqrt(T)
  const double ipark = 1.0 / (nden * sv * sqT);
  double lt = 0.0, rc = 0.0, rcT = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const SpeciesData& d = G::sp(s);
    if (d.kind == DIATOMIC && d.thv > 0.0) {
      // 1/tau_MW = sum_q X_q / tau_sq / sum_q X_q, tau_sq = exp(A T^-1/3 - AB) / p_atm
      double num = 0.0, den = 0.0;
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        if (G::sp(q).kind == ELECTRON) continue;
        num += X[q];
        den += X[q] * exp_tab(c_gas.mwAB[s][q] - c_gas.mwA[s][q] * T13);
      }
      den *= patm;
      const double tau = num / den + ipark * c_gas.icbk[s];
      const double itau = 1.0 / tau;
      double eT, cT, eV, cV;
      vib_em<G>(s, iT, emT[s], rT[s], eT, cT);
      vib_em<G>(s, iTv, emTv[s], rV[s], eV, cV);
      lt += w.rhos[s] * (eT - eV) * itau;
      rc += w.rhos[s] * cV * itau;
      rcT += w.rhos[s] * cT * itau;
    }
  }
  lt_out = lt;
  // -d(Landau-Teller)/d(rho e_v) at fixed rho_s, momentum and rho E: Tv rises with rho e_v
  // and T falls (the total energy being fixed); tau's temperature dependence is left out
  relax = ((w.cvve > 0.0) ? rc / (w.rho * w.cvve) : 0.0) +
          ((w.cvtr > 0.0) ? rcT / (w.rho * w.cvtr) : 0.0);
}
// Vibrational energy carried by species created or destroyed (2T): sum_s omega_s e_p,s with the
// pool energy e_p of each species (electrons: 3/2 R_e Tv).
template <class G, int ND>
__device__ __forceinline__ double vib_coupling(const Prim<G, ND>& w, const double* omega) {
  double lt = 0.0;
#pragma unroll
  for (int s = 0; s < G::NS; ++s) {
    const double ep = (G::sp(s).kind == ELECTRON) ? 1.5 * Rs<G>(s) * w.Tv : w.eve[s];
    lt += omega[s] * ep;
  }
  return lt;
}

// ---------------------------------------------------------------------------------------
// K1: primitives and transport (per cell): the temperature solves and everything that follows
// from the state alone.
// ---------------------------------------------------------------------------------------
// 64 threads x 10 CTAs per SM (at most 96 registers): 20 warps resident per SM instead of 12
// at the unconstrained 149 registers, for a kernel whose warps wait on dependent FP64 results
// (measured at 384 x 256: 2-5 % less time than 128 x 3; bitwise the same results)
#ifndef CS_PRIM_THREADS
#define CS_PRIM_THREADS 64     // threads per CTA
#endif
#ifndef CS_PRIM_MIN_BLOCKS
#define CS_PRIM_MIN_BLOCKS 10  // resident CTAs per SM the register allocation must allow
#endif
template <class G, int ND>
__global__ void __launch_bounds__(CS_PRIM_THREADS, CS_PRIM_MIN_BLOCKS) k_primitive(DevGrid g) {
  using A = Aux<G, ND>;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  const size_t N = g.N;
  double q[A::NQ];
#pragma unroll
  for (int v = 0; v < A::NQ; ++v) q[v] = g.Q[v * N + c];
  Prim<G, ND> w;
  const int st = primitive<G, ND, true>(q, g.W[A::T * N + c], g.W[A::TV * N + c], w, g.W + c, N);
  if (st != ST_OK) {
    set_status(g, st, c);
    return;
  }
  store_prim_scalars<G, ND>(g, c, w);
}

// ---------------------------------------------------------------------------------------
// K1b: chemistry, species Jacobian diagonal and vibrational source (per cell), from the state
// and the primitives of K1 (a separate kernel: the chemistry's working set and the temperature
// solves' iteration counts do not share one thread's registers and lanes).  A cell whose
// primitive recovery failed has its status set; the iteration is then rejected as a whole.
// ---------------------------------------------------------------------------------------
#ifndef CS_CHEM_MIN_BLOCKS
#define CS_CHEM_MIN_BLOCKS 2   // resident CTAs per SM the register allocation must allow
#endif
template <class G, int ND>
__global__ void __launch_bounds__(128, CS_CHEM_MIN_BLOCKS) k_chem(DevGrid g) {
  using A = Aux<G, ND>;
  constexpr int NS = G::NS;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  const size_t N = g.N;
  double om[NS], jd[NS], wT[NS], wTv[NS];
  double omv = 0.0, relax = 0.0;
  if (g.react && G::NR > 0) {
    const double* W = g.W;
    Prim<G, ND> w;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      w.rhos[s] = g.Q[s * N + c];
      w.eve[s] = W[(A::EVE + s) * N + c];
    }
    w.rho = W[A::RHO * N + c];
#pragma unroll
    for (int d = 0; d < ND; ++d) w.u[d] = W[(A::U + d) * N + c];
    w.T = W[A::T * N + c];
    w.Tv = W[A::TV * N + c];
    w.cv = W[A::CV * N + c];
    w.cvtr = W[A::CVTR * N + c];
    w.cvve = W[A::CVVE * N + c];
    // exp(-theta_v/T) at the vibrational temperature comes from the primitive recovery;
    // with two temperatures the trans-rotational one needs its own
    double emT[NS], emTv[NS], rT[NS], rV[NS];
    const double iT = 1.0 / w.T;
#pragma unroll
    for (int s = 0; s < NS; ++s) emTv[s] = W[(A::EMP + s) * N + c];
    if (G::NTEMP == 2) vib_exp<G>(iT, emT);
    else for (int s = 0; s < NS; ++s) emT[s] = emTv[s];
    vib_rcp<G>(emT, rT);
    if (G::NTEMP == 2) vib_rcp<G>(emTv, rV);
    else for (int s = 0; s < NS; ++s) rV[s] = rT[s];
    // the parts that need exp(-theta_v/T) and 1/(1 - em) come first, so that these arrays
    // are dead once the chemistry has formed its Gibbs energies
    double evT[NS];
    if (G::NTEMP == 1) {
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        double cvv;
        vib_em<G>(s, iT, emT[s], rT[s], evT[s], cvv);
      }
    }
    if (G::NTEMP == 2) vib_relax<G, ND>(w, emT, emTv, rT, rV, omv, relax);
    if (g.nojac) {
      // the species Jacobian diagonal comes from the surrogate network: source only
      chemistry<G, false, false>(w.rhos, w.T, w.Tv, emT, emTv, rT, rV, om, jd, nullptr, wT, wTv);
    } else {
      chemistry<G, false>(w.rhos, w.T, w.Tv, emT, emTv, rT, rV, om, jd, nullptr, wT, wTv);
      double irc, ircv;
      dT_drho_recips<G, ND>(w, irc, ircv);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const double ev = G::NTEMP == 1 ? evT[s]
                          : ((G::sp(s).kind == ELECTRON) ? 1.5 * Rs<G>(s) * w.Tv : w.eve[s]);
        double dT, dTv;
        dT_drho_r<G, ND>(w, s, ev, irc, ircv, dT, dTv);
        jd[s] += wT[s] * dT + wTv[s] * dTv;
      }
    }
    if (G::NTEMP == 2) omv += vib_coupling<G, ND>(w, om);
  } else {
#pragma unroll
    for (int s = 0; s < NS; ++s) { om[s] = 0.0; jd[s] = 0.0; }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    g.W[(A::OM + s) * N + c] = om[s];
    g.W[(A::DOM + s) * N + c] = jd[s];
  }
  g.W[A::OMV * N + c] = omv;
  g.W[A::RELAX * N + c] = relax;
}

// ---------------------------------------------------------------------------------------
// K1c (option transport = 1): species transport model replacing the Sutherland / constant
// Pr, Sc values of K1 (Sec. 2.1 defers the transport data to its references).  Blottner
// viscosity fits (heavy species at T, electrons at Tv), Eucken conductivities (2T: k_tr,s =
// mu_s (5/2 c_v,t + c_v,r), k_ve,s = mu_s c_v,v(Tv), electrons 5/2 mu_e c_v,t in the pool),
// Wilke's mixing rule; hard-sphere binary diffusion coefficients in the first Chapman-Enskog
// approximation with each species' diameter from its viscosity; Blanc's law for the effective
// coefficient of each heavy species (self-diffusion where a species is (nearly) alone); the
// electrons' flux follows the ions' in the face flux.  RHOD holds the largest rho D_s.
// ---------------------------------------------------------------------------------------
template <class G, int ND>
__global__ void __launch_bounds__(128) k_transport(DevGrid g) {
  using A = Aux<G, ND>;
  constexpr int NS = G::NS;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  const size_t N = g.N;
  double* W = g.W;
  const double T = W[A::T * N + c], Tv = W[A::TV * N + c], rho = W[A::RHO * N + c];
  const double lnT = log_tab(T), lnTv = G::NTEMP == 2 ? log_tab(Tv) : lnT;
  const double iTp = 1.0 / (G::NTEMP == 2 ? Tv : T);
  const double sqT = sqrt(T), sqTv = G::NTEMP == 2 ? sqrt(Tv) : sqT;
  double X[NS], mus[NS], ktr[NS], kve[NS], sig[NS];
  double xs = 0.0, n = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const SpeciesData& d = G::sp(s);
    const bool elec = d.kind == ELECTRON;
    const double l = elec ? lnTv : lnT;
    mus[s] = 0.1 * exp_tab((c_gas.blA[s] * l + c_gas.blB[s]) * l + c_gas.blC[s]);
    const double R = Rs<G>(s), cvt = 1.5 * R, cvr = d.kind == DIATOMIC ? R : 0.0;
    double cvv = 0.0;
    if (d.kind == DIATOMIC && d.thv > 0.0) {
      const double em = W[(A::EMP + s) * N + c], x = d.thv * iTp, r = 1.0 / (1.0 - em);
      cvv = R * x * x * em * r * r;
    }
    if (elec) {
      ktr[s] = 0.0;
      kve[s] = mus[s] * 2.5 * cvt;
    } else if (G::NTEMP == 2) {
      ktr[s] = mus[s] * (2.5 * cvt + cvr);
      kve[s] = mus[s] * cvv;
    } else {
      ktr[s] = mus[s] * (2.5 * cvt + cvr + cvv);
      kve[s] = 0.0;
    }
    const double Y = W[(A::Y + s) * N + c];
    X[s] = Y * c_gas.invM[s];
    xs += X[s];
    n += rho * Y * c_gas.ipm[s];
    sig[s] = sqrt(c_gas.hsd[s] * (elec ? sqTv : sqT) / mus[s]);
  }
  const double ixs = 1.0 / xs;
#pragma unroll
  for (int s = 0; s < NS; ++s) X[s] *= ixs;
  // Wilke: phi_s = sum_r X_r (1 + sqrt(mu_s / mu_r) (M_r/M_s)^(1/4))^2 / sqrt(8 (1 + M_s/M_r))
  double sq[NS], isq[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    sq[s] = sqrt(mus[s]);
    isq[s] = 1.0 / sq[s];
  }
  double mu = 0.0, kt = 0.0, kv = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double phi = 0.0;
#pragma unroll
    for (int r = 0; r < NS; ++r) {
      const double a = 1.0 + sq[s] * isq[r] * c_gas.wm[s][r];
      phi += X[r] * a * a * c_gas.wd[s][r];
    }
    const double w = X[s] / phi;
    mu += w * mus[s];
    kt += w * ktr[s];
    kv += w * kve[s];
  }
  W[A::MU * N + c] = mu;
  W[A::KT * N + c] = kt;
  W[A::KV * N + c] = G::NTEMP == 2 ? kv : 0.0;
  // Blanc: D_s = (1 - X_s) / sum_{r != s, heavy} X_r / D_sr, D_sr = dsr sqrt(T) / (n sigma_sr^2)
  const double sTn = sqT / n;   // D_sr = dsr sTn / sigma_sr^2
  double rDmax = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double rD = 0.0;
    if (G::sp(s).kind != ELECTRON) {
      double den = 0.0, Dss = 0.0;
#pragma unroll
      for (int r = 0; r < NS; ++r) {
        if (G::sp(r).kind == ELECTRON) continue;
        const double sr = 0.5 * (sig[s] + sig[r]);
        if (r == s) Dss = c_gas.dsr[s][r] * sTn / (sr * sr);
        else den += X[r] * sr * sr / (c_gas.dsr[s][r] * sTn);
      }
      const double D = (1.0 - X[s] > 1e-12 && den > 0.0) ? (1.0 - X[s]) / den : Dss;
      rD = rho * D;
    }
    W[(A::RHODS + s) * N + c] = rD;
    rDmax = rD > rDmax ? rD : rDmax;
  }
  W[A::RHOD * N + c] = rDmax;
}

// ---------------------------------------------------------------------------------------
// Boundary ghost values (reading: far-field in/out by the freestream's normal velocity; wall
// no-slip mirror for limiter slopes; outflow/axis copy).
// ---------------------------------------------------------------------------------------

// reconstructed variables of a cell: (rho_s, u, p, Gam, beta, [ev])
template <class G, int ND>
__device__ __forceinline__ void recon_load(const double* W, size_t N, int c, double* v) {
  using A = Aux<G, ND>;
#pragma unroll
  for (int s = 0; s < G::NS; ++s) v[s] = W[(A::Y + s) * N + c] * W[A::RHO * N + c];
#pragma unroll
  for (int d = 0; d < ND; ++d) v[G::NS + d] = W[(A::U + d) * N + c];
  v[G::NS + ND] = W[A::P * N + c];
  v[G::NS + ND + 1] = W[A::GAM * N + c];
  v[G::NS + ND + 2] = W[A::BETA * N + c];
  if (G::NTEMP == 2) v[G::NS + ND + 3] = W[A::EV * N + c];
}

// Is the far-field boundary on side (d, s) an inflow face for the freestream?
template <int ND>
__device__ __forceinline__ bool farfield_inflow(const DevGrid& g, const double* fsu, const double* Sf,
                                                int s) {
  double un = 0.0;
#pragma unroll
  for (int q = 0; q < ND; ++q) un += fsu[q] * Sf[q] * (double)s;
  return un < 0.0;
}

// Ghost reconstructed state beyond side (d, s) of interior cell c.
template <class G, int ND>
__device__ __forceinline__ void recon_ghost(const DevGrid& g, int c, int i, int j, int k, int d,
                                            int s, double* v) {
  using A = Aux<G, ND>;
  const int b = g.bc[2 * d + (s > 0)];
  if (b == BC_FARFIELD) {
    const double* Sf = face_vec(g, d, i, j, k, s);
    if (farfield_inflow<ND>(g, g.fsW + A::U, Sf, s)) {
      recon_load<G, ND>(g.fsW, 1, 0, v);
      return;
    }
  }
  recon_load<G, ND>(g.W, g.N, c, v);
  if (b == BC_WALL) {
#pragma unroll
    for (int q = 0; q < ND; ++q) v[G::NS + q] = -v[G::NS + q];
  }
}

__device__ __forceinline__ double limiter(int type, double a, double b) {
  if (a * b <= 0.0) return 0.0;
  if (type == 1) return fabs(a) < fabs(b) ? a : b;
  return (a * b * (a + b)) / (a * a + b * b);
}

// Roe flux (Sec. 3.2 names Roe's scheme) from two reconstructed states, Roe average with
// sqrt(rho) weights; F = flux * |S|.  Harten's entropy fix
// width is max(efix (|u_n| + c), 2 etaH), etaH being the face's H-correction (0 for none).
template <class G, int ND>
__device__ void roe(const double* L, const double* R, const double* S, double efix, double etaH,
                    double* F) {
  constexpr int NS = G::NS, NQ = Aux<G, ND>::NQ;
  constexpr bool TWO = G::NTEMP == 2;
  double rl = 0.0, rr = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) { rl += L[s]; rr += R[s]; }
  const double irl = 1.0 / rl, irr = 1.0 / rr;
  double a2 = 0.0, UL = 0.0, UR = 0.0, kl = 0.0, kr = 0.0;
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    a2 += S[d] * S[d];
    UL += L[NS + d] * S[d];
    UR += R[NS + d] * S[d];
    kl += 0.5 * L[NS + d] * L[NS + d];
    kr += 0.5 * R[NS + d] * R[NS + d];
  }
  const double pl = L[NS + ND], pr = R[NS + ND];
  const double EL = L[NS + ND + 1] * pl + rl * kl, ER = R[NS + ND + 1] * pr + rr * kr;
  const double evl = TWO ? L[NS + ND + 3] : 0.0, evr = TWO ? R[NS + ND + 3] : 0.0;
  const double area = sqrt(a2), ia = 1.0 / area;
  const double sl = sqrt(rl), sr = sqrt(rr), wl = sl / (sl + sr), wr = 1.0 - wl;
  const double rt = sl * sr;
  double ut[ND], un = 0.0, du2 = 0.0, dun = 0.0;
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    ut[d] = wl * L[NS + d] + wr * R[NS + d];
    const double nh = S[d] * ia;
    un += ut[d] * nh;
    const double du = R[NS + d] - L[NS + d];
    du2 += du * du;
    dun += du * nh;
  }
  const double HL = (EL + pl) * irl, HR = (ER + pr) * irr;
  const double Ht = wl * HL + wr * HR;
  const double bt = wl * L[NS + ND + 2] + wr * R[NS + ND + 2];
  const double prt = wl * pl * irl + wr * pr * irr;
  const double evt = wl * evl + wr * evr;
  const double c2 = (1.0 + bt) * prt + 0.5 * bt * wl * wr * du2;
  const double ct = sqrt(c2);
  const double delta = fmax(efix * (fabs(un) + ct), 2.0 * etaH);
  auto hfix = [delta](double l) {
    const double a = fabs(l);
    return a < delta ? (l * l + delta * delta) / (2.0 * delta) : a;
  };
  const double l1 = hfix(un - ct), l2 = hfix(un), l3 = hfix(un + ct);
  const double dp = pr - pl;
  const double i2c2 = 0.5 / c2;
  const double ap = (dp + rt * ct * dun) * i2c2, am = (dp - rt * ct * dun) * i2c2;
  const double cp = (l3 - l2) * ap, cm = (l1 - l2) * am;
  const double ha = 0.5 * area;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const double Yt = wl * L[s] * irl + wr * R[s] * irr;
    const double D = l2 * (R[s] - L[s]) + (cp + cm) * Yt;
    F[s] = 0.5 * (L[s] * UL + R[s] * UR) - ha * D;
  }
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const double nh = S[d] * ia;
    const double D = l2 * (rr * R[NS + d] - rl * L[NS + d]) + cp * (ut[d] + ct * nh) + cm * (ut[d] - ct * nh);
    F[NS + d] = 0.5 * (rl * L[NS + d] * UL + pl * S[d] + rr * R[NS + d] * UR + pr * S[d]) - ha * D;
  }
  {
    const double D = l2 * (ER - EL) + cp * (Ht + un * ct) + cm * (Ht - un * ct);
    F[NS + ND] = 0.5 * ((EL + pl) * UL + (ER + pr) * UR) - ha * D;
  }
  if (TWO) {
    const double D = l2 * (rr * evr - rl * evl) + (cp + cm) * evt;
    F[NQ - 1] = 0.5 * (rl * evl * UL + rr * evr * UR) - ha * D;
  }
}

template <class G, int ND>
__device__ __forceinline__ bool recon_ok(const double* v) {
  constexpr int NS = G::NS;
  double rho = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if (v[s] < 0.0) return false;
    rho += v[s];
  }
  if (!(v[NS + ND] > 0.0) || !(v[NS + ND + 1] > 0.0) || !(v[NS + ND + 2] > 0.0)) return false;
  if (G::NTEMP == 2 && v[NS + ND + 3] < 0.0) return false;
  return rho > 0.0;
}

// gradient variables of a cell: u, T, [Tv], Y
template <class G, int ND>
__device__ __forceinline__ void grad_vars(const double* W, size_t N, int c, double* v) {
  using A = Aux<G, ND>;
  int k = 0;
#pragma unroll
  for (int d = 0; d < ND; ++d) v[k++] = W[(A::U + d) * N + c];
  v[k++] = W[A::T * N + c];
  if (G::NTEMP == 2) v[k++] = W[A::TV * N + c];
#pragma unroll
  for (int s = 0; s < G::NS; ++s) v[k++] = W[(A::Y + s) * N + c];
}

// face value of the gradient variables on boundary side (d, s) of cell c
template <class G, int ND>
__device__ __forceinline__ void grad_boundary(const DevGrid& g, int c, int i, int j, int k, int d,
                                              int s, double* v) {
  using A = Aux<G, ND>;
  constexpr int NG = A::NG;
  const int b = g.bc[2 * d + (s > 0)];
  grad_vars<G, ND>(g.W, g.N, c, v);
  if (b == BC_WALL) {
#pragma unroll
    for (int q = 0; q < ND; ++q) v[q] = 0.0;
    v[ND] = g.Tw;
    if (G::NTEMP == 2) v[ND + 1] = g.Tw;
  } else if (b == BC_FARFIELD) {
    const double* Sf = face_vec(g, d, i, j, k, s);
    if (farfield_inflow<ND>(g, g.fsW + A::U, Sf, s)) {
      double vg[NG];
      grad_vars<G, ND>(g.fsW, 1, 0, vg);
#pragma unroll
      for (int q = 0; q < NG; ++q) v[q] = 0.5 * (v[q] + vg[q]);
    }
  }
}

// ---------------------------------------------------------------------------------------
// K2: Green-Gauss cell gradients (per cell)
// ---------------------------------------------------------------------------------------
template <class G, int ND>
__global__ void __launch_bounds__(128) k_gradient(DevGrid g) {
  using A = Aux<G, ND>;
  constexpr int NG = A::NG;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  int i, j, k;
  cell_ijk(g, c, i, j, k);
  const size_t N = g.N;
  double vc[NG], gr[NG][ND];
  grad_vars<G, ND>(g.W, N, c, vc);
#pragma unroll
  for (int v = 0; v < NG; ++v)
#pragma unroll
    for (int q = 0; q < ND; ++q) gr[v][q] = 0.0;
#pragma unroll
  for (int d = 0; d < ND; ++d)
#pragma unroll
    for (int s = -1; s <= 1; s += 2) {
      const double* Sf = face_vec(g, d, i, j, k, s);
      double vf[NG];
      bool lower;
      const int nb = neighbour(g, i, j, k, d, s, lower);
      if (nb >= 0) {
        grad_vars<G, ND>(g.W, N, nb, vf);
#pragma unroll
        for (int v = 0; v < NG; ++v) vf[v] = 0.5 * (vc[v] + vf[v]);
      } else {
        grad_boundary<G, ND>(g, c, i, j, k, d, s, vf);
      }
#pragma unroll
      for (int v = 0; v < NG; ++v)
#pragma unroll
        for (int q = 0; q < ND; ++q) gr[v][q] += (double)s * vf[v] * Sf[q];
    }
  const double iV = 1.0 / g.V[c];
#pragma unroll
  for (int v = 0; v < NG; ++v)
#pragma unroll
    for (int q = 0; q < ND; ++q) g.grad[(v * 3 + q) * N + c] = gr[v][q] * iV;
}

// Viscous / diffusive flux through S from face gradients (Sec. 2.1 tau, q, q_v and Fick
// diffusion; the energy flux includes -k_v grad Tv).
// rDs (nullable): per-species rho D_s of the species transport model, with Yf the face mass
// fractions: the electrons' flux then follows from no net charge flux, J_e = M_e sum_ions J_i /
// M_i, and a correction velocity makes the fluxes sum to zero, J_s -= Y_s sum_r J_r.  Without
// rDs one coefficient rhoD serves every species (the fluxes then sum to zero by themselves).
template <class G, int ND>
__device__ void viscous(const double (*gf)[ND], const double* uf, double mu, double kt, double kv,
                        double rhoD, const double* rDs, const double* Yf, const double* hs,
                        const double* eve, const double* S, bool wall, double* F) {
  constexpr int NS = G::NS, NQ = Aux<G, ND>::NQ;
  constexpr bool TWO = G::NTEMP == 2;
  constexpr int iT = ND, iTv = ND + 1, iY = ND + 1 + (TWO ? 1 : 0);
  double div = 0.0;
#pragma unroll
  for (int a = 0; a < ND; ++a) div += gf[a][a];
  double Js[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double J = 0.0;
    if (!wall) {
      const double r = rDs ? rDs[s] : rhoD;
#pragma unroll
      for (int q = 0; q < ND; ++q) J -= r * gf[iY + s][q] * S[q];
    }
    Js[s] = J;
  }
  if (rDs && !wall) {
    double je = 0.0, sum = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (s >= 5 && s < 10) je += Js[s] * c_gas.invM[s];   // the ions NO+ .. O+ of the air table
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if (G::sp(s).kind == ELECTRON) Js[s] = je * G::sp(s).M;
      sum += Js[s];
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) Js[s] -= Yf[s] * sum;
  }
  double qd = 0.0, qvd = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    F[s] = Js[s];
    qd += Js[s] * hs[s];
    if (TWO) qvd += Js[s] * eve[s];
  }
  double work = 0.0;
#pragma unroll
  for (int a = 0; a < ND; ++a) {
    double ts = 0.0;
#pragma unroll
    for (int l = 0; l < ND; ++l) {
      const double tau = mu * (gf[a][l] + gf[l][a]) - (a == l ? (2.0 / 3.0) * mu * div : 0.0);
      ts += tau * S[l];
    }
    F[NS + a] = -ts;
    work += uf[a] * ts;
  }
  double gT = 0.0, gTv = 0.0;
#pragma unroll
  for (int q = 0; q < ND; ++q) {
    gT += gf[iT][q] * S[q];
    if (TWO) gTv += gf[iTv][q] * S[q];
  }
  F[NS + ND] = -work - kt * gT - kv * gTv + qd;
  if (TWO) F[NQ - 1] = -kv * gTv + qvd;
}

// ---------------------------------------------------------------------------------------
// Multidimensional H-correction of the entropy fix (Sanders, Morano and Druguet, J. Comput.
// Phys. 145, 1998).  eta of a face = half the largest jump of u.n - c, u.n, u.n + c between the
// cell-centre states on its two sides = (|jump of u.n| + |jump of c|) / 2; the H width of a
// face is the largest eta over the face itself and the faces of the other directions that
// bound its two cells.  Faces on a non-periodic boundary have eta = 0.
// ---------------------------------------------------------------------------------------
template <class G, int ND>
__device__ __forceinline__ double eta_cells(const DevGrid& g, int a, int b, const double* S) {
  using A = Aux<G, ND>;
  const size_t N = g.N;
  double a2 = 0.0, dun = 0.0;
#pragma unroll
  for (int d = 0; d < ND; ++d) a2 += S[d] * S[d];
  const double area = sqrt(a2);
#pragma unroll
  for (int d = 0; d < ND; ++d) dun += (g.W[(A::U + d) * N + b] - g.W[(A::U + d) * N + a]) * (S[d] / area);
  return 0.5 * (fabs(dun) + fabs(g.W[A::C * N + b] - g.W[A::C * N + a]));
}

// eta of every direction-D face, once per residual (k_eta): the face's two cells (interior, or
// across a periodic seam), 0 on a non-periodic boundary.  eta_cells is symmetric in its two
// cells (the jumps enter through their magnitudes), so a face's eta is the same whichever of
// its cells asks for it.
template <class G, int ND, int D>
__global__ void __launch_bounds__(256) k_eta(DevGrid g) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= g.nf[D]) return;
  const int fi = g.ni + (D == 0), fj = g.nj + (D == 1);
  const int i = f % fi, j = (f / fi) % fj, k = f / (fi * fj);
  const int n = extent(g, D), pos = coord(D, i, j, k);
  int p[3] = {i, j, k};
  int a = -1, b = -1;
  if (pos > 0 && pos < n) {
    p[D] = pos - 1; a = cell_of(g, p[0], p[1], p[2]);
    p[D] = pos;     b = cell_of(g, p[0], p[1], p[2]);
  } else if (g.bc[2 * D] == BC_PERIODIC) {
    p[D] = n - 1; a = cell_of(g, p[0], p[1], p[2]);
    p[D] = 0;     b = cell_of(g, p[0], p[1], p[2]);
  }
  g.eta[D][f] = a >= 0 ? eta_cells<G, ND>(g, a, b, g.S[D] + 3 * (size_t)f) : 0.0;
}

// H width of the direction-D face f with cells a (minus side) and b (plus side), either of
// which is -1 on a non-periodic boundary: the largest eta over the face itself and the faces
// of the other directions that bound its cells (from k_eta)
template <class G, int ND, int D>
__device__ __forceinline__ double eta_h(const DevGrid& g, int a, int b, int f) {
  double eta = g.eta[D][f];
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const int c = m ? b : a;
    if (c < 0) continue;
    int ci, cj, ck;
    cell_ijk(g, c, ci, cj, ck);
#pragma unroll
    for (int e = 0; e < ND; ++e) {
      if (e == D) continue;
      int q[3] = {ci, cj, ck};
      eta = fmax(eta, g.eta[e][face_of(g, e, q[0], q[1], q[2])]);
      q[e]++;
      eta = fmax(eta, g.eta[e][face_of(g, e, q[0], q[1], q[2])]);
    }
  }
  return eta;
}

// ---------------------------------------------------------------------------------------
// K3: face fluxes along direction D (per face): MUSCL + Roe + central viscous.
// ---------------------------------------------------------------------------------------
template <class G, int ND, int D>
__global__ void __launch_bounds__(128) k_flux(DevGrid g) {
  using A = Aux<G, ND>;
  constexpr int NS = G::NS, NQ = A::NQ, NR = A::NRC, NG = A::NG;
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= g.nf[D]) return;
  const int fi = g.ni + (D == 0), fj = g.nj + (D == 1);
  const int i = f % fi, j = (f / fi) % fj, k = f / (fi * fj);
  const int n = extent(g, D);
  const int pos = coord(D, i, j, k);
  const double* S = g.S[D] + 3 * (size_t)f;
  const size_t N = g.N;
  double Fi[NQ], Fv[NQ];
  const bool per = g.bc[2 * D] == BC_PERIODIC;
  int a = -1, b = -1;     // minus / plus side cells
  int p[3] = {i, j, k};
  if (pos > 0 && pos < n) {
    p[D] = pos - 1; a = cell_of(g, p[0], p[1], p[2]);
    p[D] = pos;     b = cell_of(g, p[0], p[1], p[2]);
  } else if (per) {
    p[D] = n - 1; a = cell_of(g, p[0], p[1], p[2]);
    p[D] = 0;     b = cell_of(g, p[0], p[1], p[2]);
  }
  if (a >= 0) {
    // ---- interior face: MUSCL on (rho_s, u, p, Gam, beta, [e_v]) ----
    int ai, aj, ak, bi, bj, bk;
    cell_ijk(g, a, ai, aj, ak);
    cell_ijk(g, b, bi, bj, bk);
    double wa[NR], wb[NR], wam[NR], wbp[NR];
    recon_load<G, ND>(g.W, N, a, wa);
    recon_load<G, ND>(g.W, N, b, wb);
    bool lw;
    const int am = neighbour(g, ai, aj, ak, D, -1, lw);
    if (am >= 0) recon_load<G, ND>(g.W, N, am, wam);
    else recon_ghost<G, ND>(g, a, ai, aj, ak, D, -1, wam);
    const int bp = neighbour(g, bi, bj, bk, D, +1, lw);
    if (bp >= 0) recon_load<G, ND>(g.W, N, bp, wbp);
    else recon_ghost<G, ND>(g, b, bi, bj, bk, D, +1, wbp);
    double vl[NR], vr[NR];
#pragma unroll
    for (int v = 0; v < NR; ++v) {
      vl[v] = wa[v];
      vr[v] = wb[v];
      if (g.limiter) {
        const double dm = wa[v] - wam[v], dc = wb[v] - wa[v], dp = wbp[v] - wb[v];
        vl[v] += 0.5 * limiter(g.limiter, dm, dc);
        vr[v] -= 0.5 * limiter(g.limiter, dc, dp);
      }
    }
    const double etaH = g.hcorr ? eta_h<G, ND, D>(g, a, b, f) : 0.0;
    if (!recon_ok<G, ND>(vl) || !recon_ok<G, ND>(vr)) {
      roe<G, ND>(wa, wb, S, g.efix, etaH, Fi);
    } else {
      roe<G, ND>(vl, vr, S, g.efix, etaH, Fi);
    }
    // ---- viscous: mean of the cell gradients, centroid-line component replaced ----
    double t[3], tl = 0.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      t[q] = g.xc[q * N + b] - g.xc[q * N + a];
      tl += t[q] * t[q];
    }
    tl = sqrt(tl);
    const double itl = 1.0 / tl;
#pragma unroll
    for (int q = 0; q < 3; ++q) t[q] *= itl;
    double va[NG], vb[NG], gf[NG][ND];
    grad_vars<G, ND>(g.W, N, a, va);
    grad_vars<G, ND>(g.W, N, b, vb);
#pragma unroll
    for (int v = 0; v < NG; ++v) {
      double gt = 0.0;
#pragma unroll
      for (int q = 0; q < ND; ++q) {
        gf[v][q] = 0.5 * (g.grad[(v * 3 + q) * N + a] + g.grad[(v * 3 + q) * N + b]);
        gt += gf[v][q] * t[q];
      }
      const double corr = (vb[v] - va[v]) * itl - gt;
#pragma unroll
      for (int q = 0; q < ND; ++q) gf[v][q] += corr * t[q];
    }
    double uf[ND], hs[NS], eve[NS];
#pragma unroll
    for (int q = 0; q < ND; ++q) uf[q] = 0.5 * (g.W[(A::U + q) * N + a] + g.W[(A::U + q) * N + b]);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      hs[s] = 0.5 * (g.W[(A::HS + s) * N + a] + g.W[(A::HS + s) * N + b]);
      eve[s] = 0.5 * (g.W[(A::EVE + s) * N + a] + g.W[(A::EVE + s) * N + b]);
    }
    const double mu = 0.5 * (g.W[A::MU * N + a] + g.W[A::MU * N + b]);
    const double kt = 0.5 * (g.W[A::KT * N + a] + g.W[A::KT * N + b]);
    const double kv = 0.5 * (g.W[A::KV * N + a] + g.W[A::KV * N + b]);
    const double rd = 0.5 * (g.W[A::RHOD * N + a] + g.W[A::RHOD * N + b]);
    if (g.transport) {
      double rDs[NS], Yf[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        rDs[s] = 0.5 * (g.W[(A::RHODS + s) * N + a] + g.W[(A::RHODS + s) * N + b]);
        Yf[s] = 0.5 * (g.W[(A::Y + s) * N + a] + g.W[(A::Y + s) * N + b]);
      }
      viscous<G, ND>(gf, uf, mu, kt, kv, rd, rDs, Yf, hs, eve, S, false, Fv);
    } else {
      viscous<G, ND>(gf, uf, mu, kt, kv, rd, nullptr, nullptr, hs, eve, S, false, Fv);
    }
  } else {
    // ---- boundary face ----
    const int s = (pos == 0) ? -1 : +1;
    p[D] = (pos == 0) ? 0 : n - 1;
    const int c = cell_of(g, p[0], p[1], p[2]);
    const int bcode = g.bc[2 * D + (s > 0)];
#pragma unroll
    for (int v = 0; v < NQ; ++v) { Fi[v] = 0.0; Fv[v] = 0.0; }
    if (bcode == BC_WALL) {
      const double pc = g.W[A::P * N + c];
#pragma unroll
      for (int q = 0; q < ND; ++q) Fi[NS + q] = pc * S[q];
      // wall viscous flux: no slip, T = Tw at the face, no species flux
      const double* xf = g.fc[D] + 3 * (size_t)f;
      double t[3], tl = 0.0;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        t[q] = (s < 0) ? g.xc[q * N + c] - xf[q] : xf[q] - g.xc[q * N + c];
        tl += t[q] * t[q];
      }
      tl = sqrt(tl);
      const double itl = 1.0 / tl;
#pragma unroll
      for (int q = 0; q < 3; ++q) t[q] *= itl;
      double vc[NG], vw[NG], gf[NG][ND];
      grad_vars<G, ND>(g.W, N, c, vc);
      grad_boundary<G, ND>(g, c, p[0], p[1], p[2], D, s, vw);
#pragma unroll
      for (int v = 0; v < NG; ++v) {
        double gt = 0.0;
#pragma unroll
        for (int q = 0; q < ND; ++q) {
          gf[v][q] = g.grad[(v * 3 + q) * N + c];
          gt += gf[v][q] * t[q];
        }
        const double corr = ((s < 0) ? (vc[v] - vw[v]) : (vw[v] - vc[v])) * itl - gt;
#pragma unroll
        for (int q = 0; q < ND; ++q) gf[v][q] += corr * t[q];
      }
      double uf[ND], hs[NS], eve[NS];
#pragma unroll
      for (int q = 0; q < ND; ++q) uf[q] = 0.0;
#pragma unroll
      for (int sp = 0; sp < NS; ++sp) {
        hs[sp] = g.W[(A::HS + sp) * N + c];
        eve[sp] = g.W[(A::EVE + sp) * N + c];
      }
      viscous<G, ND>(gf, uf, g.W[A::MU * N + c], g.W[A::KT * N + c], g.W[A::KV * N + c],
                     g.W[A::RHOD * N + c], nullptr, nullptr, hs, eve, S, true, Fv);
    } else if (bcode == BC_FARFIELD || bcode == BC_OUTFLOW) {
      double wi[NR], wg[NR];
      recon_load<G, ND>(g.W, N, c, wi);
      recon_ghost<G, ND>(g, c, p[0], p[1], p[2], D, s, wg);
      const double etaH = g.hcorr ? eta_h<G, ND, D>(g, s > 0 ? c : -1, s > 0 ? -1 : c, f) : 0.0;
      if (s > 0) roe<G, ND>(wi, wg, S, g.efix, etaH, Fi);
      else roe<G, ND>(wg, wi, S, g.efix, etaH, Fi);
    }
  }
#pragma unroll
  for (int v = 0; v < NQ; ++v) g.F[D][(size_t)v * g.nf[D] + f] = Fi[v] + Fv[v];
}

// ---------------------------------------------------------------------------------------
// K4: residual assembly R = sum_d (F_+ - F_-) - V S, plus per-block norm partial sums.
// ---------------------------------------------------------------------------------------
template <class G, int ND>
__global__ void __launch_bounds__(256) k_assemble(DevGrid g) {
  using A = Aux<G, ND>;
  constexpr int NS = G::NS, NQ = A::NQ;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double rs = 0.0, re = 0.0;
  if (c < g.N) {
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    const size_t N = g.N;
    double r[NQ];
#pragma unroll
    for (int v = 0; v < NQ; ++v) r[v] = 0.0;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      const int fm = face_of(g, d, i, j, k);
      int p[3] = {i, j, k};
      p[d]++;
      const int fp = face_of(g, d, p[0], p[1], p[2]);
      const size_t nf = g.nf[d];
#pragma unroll
      for (int v = 0; v < NQ; ++v) r[v] += g.F[d][v * nf + fp] - g.F[d][v * nf + fm];
    }
    const double V = g.V[c];
#pragma unroll
    for (int s = 0; s < NS; ++s) r[s] -= V * g.W[(A::OM + s) * N + c];
    if (G::NTEMP == 2) r[NQ - 1] -= V * g.W[A::OMV * N + c];
    // dual time stepping (Sec. 2.3): + V [(1+theta)(Q - Q^n) - theta (Q^n - Q^{n-1})] / dt
    const double da = g.params[1];
    if (da > 0.0) {
      const double db = g.params[2];
#pragma unroll
      for (int v = 0; v < NQ; ++v) {
        const double qn = g.Qn[v * N + c];
        r[v] += V * (da * (g.Q[v * N + c] - qn) - db * (qn - g.Qnm1[v * N + c]));
      }
    }
#pragma unroll
    for (int v = 0; v < NQ; ++v) g.R[v * N + c] = r[v];
    const double iV = 1.0 / V;
#pragma unroll
    for (int s = 0; s < NS; ++s) rs += (r[s] * iV) * (r[s] * iV);
    re = (r[NS + ND] * iV) * (r[NS + ND] * iV);
  }
  // deterministic block reduction
  __shared__ double sh[2][256];
  sh[0][threadIdx.x] = rs;
  sh[1][threadIdx.x] = re;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    g.red[2 * blockIdx.x] = sh[0][0];
    g.red[2 * blockIdx.x + 1] = sh[1][0];
  }
}

// final reduction of the norm partials (one block); out[0..1] = sqrt of sums; also computes
// the stagnation heat flux of cell `stag` (q_w = k (T_1 - Tw)/d_1 [+ k_v (Tv_1 - Tw)/d_1]).
template <class G, int ND>
__global__ void __launch_bounds__(256) k_norms(DevGrid g, int nblocks, int stag, double* out) {
  using A = Aux<G, ND>;
  __shared__ double sh[2][256];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += blockDim.x) {
    a += g.red[2 * k];
    b += g.red[2 * k + 1];
  }
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sqrt(sh[0][0]);
    out[1] = sqrt(sh[1][0]);
    out[2] = 0.0;
    if (stag >= 0 && g.bc[2] == BC_WALL) {
      const size_t N = g.N;
      int i, j, k;
      cell_ijk(g, stag, i, j, k);
      const int f = face_of(g, 1, i, j, k);
      const double* Sf = g.S[1] + 3 * (size_t)f;
      const double* xf = g.fc[1] + 3 * (size_t)f;
      double area = 0.0, dist = 0.0;
      for (int q = 0; q < 3; ++q) area += Sf[q] * Sf[q];
      area = sqrt(area);
      for (int q = 0; q < 3; ++q) dist += (g.xc[q * N + stag] - xf[q]) * Sf[q] / area;
      dist = fabs(dist);
      double qw = g.W[A::KT * N + stag] * (g.W[A::T * N + stag] - g.Tw) / dist;
      if (G::NTEMP == 2) qw += g.W[A::KV * N + stag] * (g.W[A::TV * N + stag] - g.Tw) / dist;
      out[2] = qw;
    }
  }
}

// ---------------------------------------------------------------------------------------
// K5: spectral radii, local time step, split diagonals (per cell).  Readings 7, 8, 9.
// ---------------------------------------------------------------------------------------
template <class G, int ND>
__global__ void __launch_bounds__(128) k_spectral(DevGrid g) {
  using A = Aux<G, ND>;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  int i, j, k;
  cell_ijk(g, c, i, j, k);
  const size_t N = g.N;
  const double* W = g.W;
  const double rho = W[A::RHO * N + c], mu = W[A::MU * N + c], kt = W[A::KT * N + c];
  double nuF;
  if (G::NTEMP == 2) {
    nuF = fmax(4.0 * mu / 3.0, kt / W[A::CVTR * N + c]);
    const double cvve = W[A::CVVE * N + c];
    if (cvve > 0.0) nuF = fmax(nuF, W[A::KV * N + c] / cvve);
  } else {
    nuF = fmax(4.0 * mu / 3.0, kt / W[A::CV * N + c]);
  }
  const double irho = 1.0 / rho;
  nuF *= irho;
  const double nuC = W[A::RHOD * N + c] * irho;
  const double nuCI = fmax(nuF, nuC);
  const double V = g.V[c], iV = 1.0 / V, cs = W[A::C * N + c];
  double sumdt = 0.0, sF = 0.0, sC = 0.0, sCI = 0.0;
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const double* Sm = face_vec(g, d, i, j, k, -1);
    const double* Sp = face_vec(g, d, i, j, k, +1);
    double a2 = 0.0, U = 0.0;
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      const double sb = 0.5 * (Sm[q] + Sp[q]);
      a2 += sb * sb;
      U += W[(A::U + q) * N + c] * sb;
    }
    const double a = sqrt(a2);
    const double liF = fabs(U) + cs * a, liC = fabs(U);
    const double lvF = nuF * a2 * iV, lvC = nuC * a2 * iV, lvCI = nuCI * a2 * iV;
    const double lF = liF + 2.0 * lvF, lC = liC + 2.0 * lvC, lCI = liF + 2.0 * lvCI;
    g.lamF[d * N + c] = lF;
    g.lamC[d * N + c] = lC;
    g.lamCI[d * N + c] = g.cisplit ? 2.0 * lvCI : lCI;   // eigenvalue splitting: viscous part only
    sumdt += liF + lvF;
    sF += lF;
    sC += lC;
    sCI += g.cisplit ? 2.0 * lvCI : lCI;
  }
  // Sec. 2.2 (Delta tau) with its source term: lambda_S, read as the largest magnitude on the
  // diagonal of the source Jacobian (species d omega_s / d rho_s, and the vibrational
  // relaxation rate), joins the radii of the local time step
  if (g.dtau_src && g.react) {
    double lS = G::NTEMP == 2 ? W[A::RELAX * N + c] : 0.0;
#pragma unroll
    for (int s = 0; s < G::NS; ++s) lS = fmax(lS, fabs(W[(A::DOM + s) * N + c]));
    sumdt += V * lS;
  }
  // V / dtau, plus (1+theta) V / dt under dual time stepping (every diagonal carries it)
  const double Vdt = sumdt / g.params[0] + g.params[1] * V;
  g.Vdt[c] = Vdt;
  const double DF = Vdt + sF, DFev = Vdt + sF + V * W[A::RELAX * N + c];
  g.DF[c] = DF;
  g.DFev[c] = DFev;
  g.invD[c] = 1.0 / DF;
  g.invD[N + c] = 1.0 / DFev;
  double py = 0.0, rr = 0.0;
#pragma unroll
  for (int s = 0; s < G::NS; ++s) {
    const double Ds = Vdt + sC + V * fmax(0.0, -W[(A::DOM + s) * N + c]);
    g.Ds[s * N + c] = Ds;
    g.invD[(2 + s) * N + c] = 1.0 / Ds;
    py += W[(A::Y + s) * N + c] * W[(A::PRS + s) * N + c];
    rr += g.R[s * N + c];
  }
  // per-cell inputs of the sweeps: p_Y = sum_s Y_s dp/drho_s (frozen-composition pressure
  // derivative of the flow block) and the flow right-hand side
  g.W[A::PY * N + c] = py;
  g.rhsF[c] = -rr;
#pragma unroll
  for (int q = 1; q < A::NF; ++q) g.rhsF[q * N + c] = -g.R[(G::NS + q - 1) * N + c];
  if (g.DLU) g.DLU[(size_t)c * A::NCI * A::NCI] = sCI;   // sum of coupled radii, read by k_ci_block
}

// ---------------------------------------------------------------------------------------
// Flux Jacobian times a vector at a cell state (Sec. 2.3 Eq. (convectiveJacobian)),
// matrix-free.  Flow block with frozen mass fractions (Sec. 2.3.1) and coupled variables.
// ---------------------------------------------------------------------------------------
template <class G, int ND, class T = double>
struct CellState {       // what the flow Jacobian needs from the neighbour cell
  T u[ND], H, ev, beta, prev, pY;   // pY = sum_s Y_s dp/drho_s
};

template <class G, int ND, class T>
__device__ __forceinline__ void load_state(const DevGrid& g, int c, CellState<G, ND, T>& s) {
  using A = Aux<G, ND>;
  const size_t N = g.N;
  const double* W = g.W;
#pragma unroll
  for (int d = 0; d < ND; ++d) s.u[d] = (T)W[(A::U + d) * N + c];
  s.H = (T)W[A::H * N + c];
  s.ev = (G::NTEMP == 2) ? (T)W[A::EV * N + c] : T(0);
  s.beta = (T)W[A::BETA * N + c];
  s.prev = (T)W[A::PREV * N + c];
  s.pY = (T)W[A::PY * N + c];
}

// flow block: x = (drho, dm, drhoE, [drho e_v]) -> A(S) x.  With a = rho dU = S.dm - U drho
// the product needs no division: dF_m = dm U + u a + dp S, dF_E = (drhoE + dp) U + H a,
// dF_ev = d(rho e_v) U + e_v a.  T is the compute type of the operator (FP64, or FP32 in the
// mixed-precision form).
template <class G, int ND, class T>
__device__ __forceinline__ void jvp_flow(const CellState<G, ND, T>& w, const T* S, const T* x, T* y) {
  constexpr int NF = Aux<G, ND>::NF;
  T U = 0, Sdm = 0, dp = w.pY * x[0] + w.beta * x[ND + 1];
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    U += w.u[d] * S[d];
    Sdm += S[d] * x[1 + d];
    dp -= w.beta * w.u[d] * x[1 + d];
  }
  if (G::NTEMP == 2) dp += w.prev * x[NF - 1];
  const T a = Sdm - U * x[0];
  y[0] = Sdm;
#pragma unroll
  for (int d = 0; d < ND; ++d) y[1 + d] = x[1 + d] * U + w.u[d] * a + dp * S[d];
  y[ND + 1] = (x[ND + 1] + dp) * U + w.H * a;
  if (G::NTEMP == 2) y[NF - 1] = x[NF - 1] * U + w.ev * a;
}

// ---------------------------------------------------------------------------------------
// K6: split LU-SGS sweeps on hyperplanes h = i+j(+k) (Sec. 2.2 + 2.3.1-2.3.2).
// One launch per hyperplane; each thread owns one cell of the hyperplane.
// FWD: x = dQ* = D^-1(-R - sum_L coef x_nb); BWD: y = x + D^-1 sum_U (-coef) y_nb.
// ---------------------------------------------------------------------------------------
template <class G, int ND>
__device__ __forceinline__ bool hyperplane_cell(const DevGrid& g, int h, int t, int& i, int& j, int& k) {
  if (ND == 2) {
    j = t;
    k = 0;
    if (j >= g.nj) return false;
    i = h - j;
  } else {
    j = t % g.nj;
    k = t / g.nj;
    if (k >= g.nk) return false;
    i = h - j - k;
  }
  return i >= 0 && i < g.ni;
}

template <class G, int ND, bool FWD, class T>
__global__ void __launch_bounds__(64) k_sweep_split(DevGrid g, int h, int off, int cnt) {
  using A = Aux<G, ND>;
  constexpr int NS = G::NS, NF = A::NF;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (t >= cnt || !hyperplane_cell<G, ND>(g, h, t + off, i, j, k)) return;
  const int c = cell_of(g, i, j, k);
  const size_t N = g.N;
  T acc[NF], accs[NS];
  if (FWD) {
#pragma unroll
    for (int s = 0; s < NS; ++s) accs[s] = (T)(-g.R[s * N + c]);
#pragma unroll
    for (int q = 0; q < NF; ++q) acc[q] = (T)g.rhsF[q * N + c];
  } else {
#pragma unroll
    for (int q = 0; q < NF; ++q) acc[q] = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s) accs[s] = 0;
  }
  const double* X = FWD ? g.dQs : g.dQ;     // solution being built by this sweep
#pragma unroll
  for (int d = 0; d < ND; ++d)
#pragma unroll
    for (int s = -1; s <= 1; s += 2) {
      bool lower;
      const int nb = neighbour(g, i, j, k, d, s, lower);
      if (nb < 0 || lower != FWD) continue;
      const double* Sd = face_vec(g, d, i, j, k, s);
      T Sf[ND];
#pragma unroll
      for (int q = 0; q < ND; ++q) Sf[q] = (T)Sd[q];
      CellState<G, ND, T> w;
      load_state<G, ND, T>(g, nb, w);
      T xn[NF], ax[NF];
#pragma unroll
      for (int q = 0; q < NF; ++q) xn[q] = (T)X[q * N + nb];
      jvp_flow<G, ND, T>(w, Sf, xn, ax);
      const T l = (T)g.lamF[d * N + nb];
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        if (s < 0) acc[q] += T(0.5) * (ax[q] + l * xn[q]);
        else acc[q] -= T(0.5) * (ax[q] - l * xn[q]);
      }
      T U = 0;
#pragma unroll
      for (int q = 0; q < ND; ++q) U += w.u[q] * Sf[q];
      const T lc = (T)g.lamC[d * N + nb];
#pragma unroll
      for (int sp = 0; sp < NS; ++sp) {
        const T xs = (T)X[(NF + sp) * N + nb];
        if (s < 0) accs[sp] += T(0.5) * (U * xs + lc * xs);
        else accs[sp] -= T(0.5) * (U * xs - lc * xs);
      }
    }
  double* Y = FWD ? g.dQs : g.dQ;
#pragma unroll
  for (int q = 0; q < NF; ++q) {
    const T iD = (T)((G::NTEMP == 2 && q == NF - 1) ? g.invD[N + c] : g.invD[c]);
    const T v = acc[q] * iD;
    Y[q * N + c] = FWD ? (double)v : (double)((T)g.dQs[q * N + c] + v);
  }
#pragma unroll
  for (int sp = 0; sp < NS; ++sp) {
    const T v = accs[sp] * (T)g.invD[(2 + sp) * N + c];
    Y[(NF + sp) * N + c] = FWD ? (double)v : (double)((T)g.dQs[(NF + sp) * N + c] + v);
  }
}

// ---------------------------------------------------------------------------------------
// K6b: split LU-SGS sweeps in thread-block clusters (2D).  The flow block and every species
// equation are independent operators (Sec. 2.3: "solved without specific order"), so each
// gets its own cluster: cluster 0 sweeps the flow block, cluster 1+s species s.  In a cluster
// of C CTAs, CTA r owns rows j in [r R, (r+1) R), one thread per row; at hyperplane h the
// thread of row j updates cell (h - j, j).  The recurrence stays on chip: the previous cell of
// the row (and the first cell, for the periodic wrap in i) is in registers, the row below /
// above comes from shared memory, across a CTA boundary through distributed shared memory,
// and one hardware cluster barrier separates consecutive hyperplanes.  Forward and backward
// sweeps run in the same launch.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_nctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;\n" : "=r"(r));
  return r;
}
// generic address of the same shared variable in CTA `rank` of the cluster
template <class T>
__device__ __forceinline__ T* dsmem(T* p, unsigned rank) {
  unsigned long long in = reinterpret_cast<unsigned long long>(p), out;
  asm volatile("mapa.u64 %0, %1, %2;\n" : "=l"(out) : "l"(in), "r"(rank));
  return reinterpret_cast<T*>(out);
}

constexpr int kClusterRows = 32;   // max rows per CTA
// Warps per CTA of the direct-load cluster kernel: 1 or 2, both covering the CTA's R rows (one
// lane per row).  With 2, the flow cluster splits each step's FP64 work: warp 0 takes the
// coupling of the neighbouring row and the update, warp 1 the row's own earlier cells (GB300
// issues FP64 at ~1/64 of its FP32 rate; the two warps run on two SM sub-partitions), 5 % faster
// for one grid; with 1 a CTA needs half the registers, so twice as many CTAs stay resident, which
// is what a batch of many grids needs.  Splitting rows over more warps instead was measured
// slower (more FP64 instructions at the same cost each).  In a species cluster the second warp
// only takes part in the barriers.
// Row handled by this lane (the first lane of each of the R lane groups), or -1 for a lane
// that only takes part in the barriers.
__device__ __forceinline__ int cluster_row(int R) {
  const int lane = threadIdx.x & 31;
  const int stride = 32 / R;
  if (lane % stride != 0) return -1;
  const int t = lane / stride;
  return t < R ? t : -1;
}

template <class G, int NV, class T>
struct Xchg {
  T v[2][kClusterRows][NV];
};

// one neighbour contribution of the flow block: nb on side s of direction d
template <class G, class T>
__device__ __forceinline__ void flow_contrib(const CellState<G, 2, T>& w, T lam, const T* Sf,
                                             const T* xn, int side, T* acc) {
  constexpr int NF = Aux<G, 2>::NF;
  T ax[NF];
  jvp_flow<G, 2, T>(w, Sf, xn, ax);
#pragma unroll
  for (int q = 0; q < NF; ++q) {
    if (side < 0) acc[q] += T(0.5) * (ax[q] + lam * xn[q]);
    else acc[q] -= T(0.5) * (ax[q] - lam * xn[q]);
  }
}

// Static inputs of one cell for the flow sweep (loaded one step ahead).
template <class G, class T>
struct FlowStep {
  static constexpr int NF = Aux<G, 2>::NF;
  CellState<G, 2, T> me, jn;
  T lam0, jlam, iD, iDev, base[NF], Si[2], Sj[2], Sw[2];
  int c;
  bool act, hasj;
};

template <class G, class T>
__device__ __forceinline__ void flow_step_load(const DevGrid& g, int q, int j, bool row, bool fwd,
                                               FlowStep<G, T>& f) {
  constexpr int NF = Aux<G, 2>::NF;
  const size_t N = g.N;
  const int ni = g.ni, nj = g.nj, H = ni + nj - 2;
  const int h = fwd ? q : H - q;
  const int i = h - j;
  f.act = row && q <= H && i >= 0 && i < ni;
  const int jj = fwd ? j - 1 : j + 1;
  f.hasj = f.act && jj >= 0 && jj < nj;
  if (!f.act) return;
  const int c = i + ni * j;
  f.c = c;
  load_state<G, 2, T>(g, c, f.me);
  f.lam0 = (T)g.lamF[c];
  f.iD = (T)g.invD[c];
  f.iDev = (T)g.invD[N + c];
#pragma unroll
  for (int v = 0; v < NF; ++v) f.base[v] = (T)(fwd ? g.rhsF[v * N + c] : g.dQs[v * N + c]);
  const double* Si = g.S[0] + 3 * (size_t)face_of(g, 0, fwd ? i : i + 1, j, 0);
  const double* Sj = g.S[1] + 3 * (size_t)face_of(g, 1, i, fwd ? j : j + 1, 0);
  const double* Sw = g.S[0] + 3 * (size_t)face_of(g, 0, fwd ? ni : 0, j, 0);
  f.Si[0] = (T)Si[0]; f.Si[1] = (T)Si[1];
  f.Sj[0] = (T)Sj[0]; f.Sj[1] = (T)Sj[1];
  f.Sw[0] = (T)Sw[0]; f.Sw[1] = (T)Sw[1];
  if (f.hasj) {
    const int cn = i + ni * jj;
    load_state<G, 2, T>(g, cn, f.jn);
    f.jlam = (T)g.lamF[N + cn];
  }
}

// One warp per CTA: the row's own earlier cells are coupled while the cluster barrier is
// pending, the neighbouring row after it (the variant with fewer registers per CTA, for batches).
template <class G, class T>
__device__ void sweep_flow_cluster1(const DevGrid& g, int R, Xchg<G, Aux<G, 2>::NF, T>& xc) {
  using A = Aux<G, 2>;
  constexpr int NF = A::NF;
  const size_t N = g.N;
  const unsigned rank = cluster_ctarank();
  const int t = cluster_row(R);
  const int j = rank * R + t;
  const bool row = t >= 0 && j < g.nj;
  const bool per = g.bc[0] == BC_PERIODIC;
  const int ni = g.ni, H = ni + g.nj - 2;
  for (int pass = 0; pass < 2; ++pass) {
    const bool fwd = pass == 0;
    T prevx[NF], firstx[NF];
    CellState<G, 2, T> prevS, firstS;
    T prevL = 0, firstL = 0;
    FlowStep<G, T> cur, nxt;
    flow_step_load<G, T>(g, 0, j, row, fwd, cur);
    for (int q = 0; q <= H; ++q) {
      const int i = (fwd ? q : H - q) - j;
      flow_step_load<G, T>(g, q + 1, j, row, fwd, nxt);     // prefetch the next step
      // contributions of this row's own earlier results (the i-neighbour, the periodic
      // neighbour) need no other CTA: computed while the cluster barrier is pending
      T acc[NF];
      if (cur.act) {
#pragma unroll
        for (int v = 0; v < NF; ++v) acc[v] = fwd ? cur.base[v] : T(0);
        if (fwd) {
          if (i > 0) flow_contrib<G, T>(prevS, prevL, cur.Si, prevx, -1, acc);
          if (per && i == ni - 1) flow_contrib<G, T>(firstS, firstL, cur.Sw, firstx, +1, acc);
        } else {
          if (per && i == 0) flow_contrib<G, T>(firstS, firstL, cur.Sw, firstx, -1, acc);
          if (i < ni - 1) flow_contrib<G, T>(prevS, prevL, cur.Si, prevx, +1, acc);
        }
      }
      if (q > 0) cluster_wait();
      if (cur.act) {
        if (cur.hasj) {
          const T* src;
          const int par = (q - 1) & 1;
          if (fwd) src = (t > 0) ? xc.v[par][t - 1] : dsmem(&xc.v[par][R - 1][0], rank - 1);
          else src = (t < R - 1) ? xc.v[par][t + 1] : dsmem(&xc.v[par][0][0], rank + 1);
          T xn[NF];
#pragma unroll
          for (int v = 0; v < NF; ++v) xn[v] = src[v];
          flow_contrib<G, T>(cur.jn, cur.jlam, cur.Sj, xn, fwd ? -1 : +1, acc);
        }
        double* out = fwd ? g.dQs : g.dQ;
#pragma unroll
        for (int v = 0; v < NF; ++v) {
          const T d = (G::NTEMP == 2 && v == NF - 1) ? cur.iDev : cur.iD;
          const T x = fwd ? acc[v] * d : cur.base[v] + acc[v] * d;
          out[v * N + cur.c] = (double)x;
          xc.v[q & 1][t][v] = x;
          prevx[v] = x;
        }
        prevS = cur.me;
        prevL = cur.lam0;
        if (i == (fwd ? 0 : ni - 1)) {
#pragma unroll
          for (int v = 0; v < NF; ++v) firstx[v] = prevx[v];
          firstS = cur.me;
          firstL = cur.lam0;
        }
      }
      cluster_arrive();
      cur = nxt;
    }
    cluster_wait();
  }
}

// Two warps per CTA: warp 0 couples the neighbouring row and updates, warp 1 couples the row's
// own earlier cells.
template <class G, class T>
__device__ void sweep_flow_cluster2(const DevGrid& g, int R, Xchg<G, Aux<G, 2>::NF, T>& xc,
                                    T (&accI)[kClusterRows][Aux<G, 2>::NF]) {
  using A = Aux<G, 2>;
  constexpr int NF = A::NF;
  const size_t N = g.N;
  const unsigned rank = cluster_ctarank();
  const bool lead = threadIdx.x < 32;          // warp 0: neighbour row + update; warp 1: own row
  const int t = cluster_row(R);
  const int j = rank * R + t;
  const bool row = t >= 0 && j < g.nj;
  const bool per = g.bc[0] == BC_PERIODIC;
  const int ni = g.ni, H = ni + g.nj - 2;
  for (int pass = 0; pass < 2; ++pass) {
    const bool fwd = pass == 0;
    T prevx[NF], firstx[NF];
    CellState<G, 2, T> prevS, firstS;
    T prevL = 0, firstL = 0;
    FlowStep<G, T> cur, nxt;
    flow_step_load<G, T>(g, 0, j, row, fwd, cur);
    for (int q = 0; q <= H; ++q) {
      const int i = (fwd ? q : H - q) - j;
      flow_step_load<G, T>(g, q + 1, j, row, fwd, nxt);     // prefetch the next step
      T acc[NF];
#pragma unroll
      for (int v = 0; v < NF; ++v) acc[v] = T(0);
      if (lead) {
        // coupling of the neighbouring row: its result of step q-1 comes from this CTA's shared
        // memory or, across a CTA boundary, the neighbour CTA's, after the cluster barrier
        if (q > 0) cluster_wait();
        if (cur.act && cur.hasj) {
          const T* src;
          const int par = (q - 1) & 1;
          if (fwd) src = (t > 0) ? xc.v[par][t - 1] : dsmem(&xc.v[par][R - 1][0], rank - 1);
          else src = (t < R - 1) ? xc.v[par][t + 1] : dsmem(&xc.v[par][0][0], rank + 1);
          T xn[NF];
#pragma unroll
          for (int v = 0; v < NF; ++v) xn[v] = src[v];
          flow_contrib<G, T>(cur.jn, cur.jlam, cur.Sj, xn, fwd ? -1 : +1, acc);
        }
      } else if (cur.act) {
        // the row's own earlier results (the i-neighbour, the periodic neighbour): no other
        // CTA is involved, so this runs while warp 0 waits for the cluster barrier
        if (fwd) {
          if (i > 0) flow_contrib<G, T>(prevS, prevL, cur.Si, prevx, -1, acc);
          if (per && i == ni - 1) flow_contrib<G, T>(firstS, firstL, cur.Sw, firstx, +1, acc);
        } else {
          if (per && i == 0) flow_contrib<G, T>(firstS, firstL, cur.Sw, firstx, -1, acc);
          if (i < ni - 1) flow_contrib<G, T>(prevS, prevL, cur.Si, prevx, +1, acc);
        }
#pragma unroll
        for (int v = 0; v < NF; ++v) accI[t][v] = acc[v];
      }
      __syncthreads();                 // warp 1's contributions are in accI
      if (lead && cur.act) {
        double* out = fwd ? g.dQs : g.dQ;
#pragma unroll
        for (int v = 0; v < NF; ++v) {
          const T d = (G::NTEMP == 2 && v == NF - 1) ? cur.iDev : cur.iD;
          const T a = acc[v] + accI[t][v];
          const T x = fwd ? (cur.base[v] + a) * d : cur.base[v] + a * d;
          out[v * N + cur.c] = (double)x;
          xc.v[q & 1][t][v] = x;
        }
      }
      __syncthreads();                 // this step's results are in xc.v[q & 1]
      if (!lead) {
        if (cur.act) {
#pragma unroll
          for (int v = 0; v < NF; ++v) prevx[v] = xc.v[q & 1][t][v];
          prevS = cur.me;
          prevL = cur.lam0;
          if (i == (fwd ? 0 : ni - 1)) {
#pragma unroll
            for (int v = 0; v < NF; ++v) firstx[v] = prevx[v];
            firstS = cur.me;
            firstL = cur.lam0;
          }
        }
        if (q > 0) cluster_wait();     // complete the previous phase before arriving again
      }
      cluster_arrive();
      cur = nxt;
    }
    cluster_wait();
  }
}

// Species per component (they share u, lambda and S).  The record kernels (k_pack_wave,
// k_split_wave, k_split_block) move a group's values with 16-byte cp.async copies, so their
// group times the element size must be a multiple of 16 bytes; the direct-load cluster kernel
// takes two species per cluster, which keeps the FP64 work of a species step below the flow
// block's.
constexpr int kSpeciesGroup = 4;
constexpr int kClusterSpeciesGroup = 4;
static_assert(kSpeciesGroup * sizeof(float) % 16 == 0, "record groups must be whole 16-byte pieces");

template <class G, class T>
__device__ void sweep_species_cluster(const DevGrid& g, int R, int s0, Xchg<G, kClusterSpeciesGroup, T>& xc) {
  using A = Aux<G, 2>;
  constexpr int NF = A::NF, SG = kClusterSpeciesGroup;
  const size_t N = g.N;
  if (threadIdx.x >= 32) {
    // the second warp of a species CTA: the same sequence of cluster barriers as warp 0
    const int H = g.ni + g.nj - 2;
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = 0; q <= H; ++q) {
        if (q > 0) cluster_wait();
        cluster_arrive();
      }
      cluster_wait();
    }
    return;
  }
  const unsigned rank = cluster_ctarank();
  const int t = cluster_row(R);
  const int j = rank * R + t;
  const bool row = t >= 0 && j < g.nj;
  const bool per = g.bc[0] == BC_PERIODIC;
  const int ni = g.ni, nj = g.nj, H = ni + nj - 2;
  const int ns = (G::NS - s0 < SG) ? G::NS - s0 : SG;
  for (int pass = 0; pass < 2; ++pass) {
    const bool fwd = pass == 0;
    T prevx[SG], firstx[SG], prevU[2] = {0, 0}, firstU[2] = {0, 0}, prevL = 0, firstL = 0;
#pragma unroll
    for (int k = 0; k < SG; ++k) { prevx[k] = 0; firstx[k] = 0; }
    for (int q = 0; q <= H; ++q) {
      const int h = fwd ? q : H - q;
      const int i = h - j;
      const bool act = row && i >= 0 && i < ni;
      const int jj = fwd ? j - 1 : j + 1;
      const bool hasj = act && jj >= 0 && jj < nj;
      T u0 = 0, u1 = 0, lam0 = 0, iD[SG], base[SG], ju0 = 0, ju1 = 0, jlam = 0;
      T Si0 = 0, Si1 = 0, Sj0 = 0, Sj1 = 0, Sw0 = 0, Sw1 = 0;
      int c = 0;
      if (act) {
        c = i + ni * j;
        u0 = (T)g.W[A::U * N + c];
        u1 = (T)g.W[(A::U + 1) * N + c];
        lam0 = (T)g.lamC[c];
#pragma unroll
        for (int k = 0; k < SG; ++k) {
          if (k >= ns) continue;
          iD[k] = (T)g.invD[(2 + s0 + k) * N + c];
          base[k] = (T)(fwd ? -g.R[(size_t)(s0 + k) * N + c] : g.dQs[(size_t)(NF + s0 + k) * N + c]);
        }
        const double* Si = g.S[0] + 3 * (size_t)face_of(g, 0, fwd ? i : i + 1, j, 0);
        const double* Sj = g.S[1] + 3 * (size_t)face_of(g, 1, i, fwd ? j : j + 1, 0);
        const double* Sw = g.S[0] + 3 * (size_t)face_of(g, 0, fwd ? ni : 0, j, 0);
        Si0 = (T)Si[0]; Si1 = (T)Si[1]; Sj0 = (T)Sj[0]; Sj1 = (T)Sj[1]; Sw0 = (T)Sw[0]; Sw1 = (T)Sw[1];
        if (hasj) {
          const int cn = i + ni * jj;
          ju0 = (T)g.W[A::U * N + cn];
          ju1 = (T)g.W[(A::U + 1) * N + cn];
          jlam = (T)g.lamC[N + cn];
        }
      }
      if (q > 0) cluster_wait();
      if (act) {
        T acc[SG];
#pragma unroll
        for (int k = 0; k < SG; ++k) acc[k] = fwd ? base[k] : T(0);
        // coefficient of a neighbour: minus side (U + lam)/2, plus side -(U - lam)/2
        auto coef = [](T ua, T ub, T lam, T s0_, T s1_, int side) {
          const T U = ua * s0_ + ub * s1_;
          return side < 0 ? T(0.5) * (U + lam) : T(-0.5) * (U - lam);
        };
        if (fwd) {
          if (i > 0) {
            const T k0 = coef(prevU[0], prevU[1], prevL, Si0, Si1, -1);
#pragma unroll
            for (int k = 0; k < SG; ++k) acc[k] += k0 * prevx[k];
          }
          if (per && i == ni - 1) {
            const T k0 = coef(firstU[0], firstU[1], firstL, Sw0, Sw1, +1);
#pragma unroll
            for (int k = 0; k < SG; ++k) acc[k] += k0 * firstx[k];
          }
        } else {
          if (per && i == 0) {
            const T k0 = coef(firstU[0], firstU[1], firstL, Sw0, Sw1, -1);
#pragma unroll
            for (int k = 0; k < SG; ++k) acc[k] += k0 * firstx[k];
          }
          if (i < ni - 1) {
            const T k0 = coef(prevU[0], prevU[1], prevL, Si0, Si1, +1);
#pragma unroll
            for (int k = 0; k < SG; ++k) acc[k] += k0 * prevx[k];
          }
        }
        if (hasj) {
          const int par = (q - 1) & 1;
          const T* src;
          if (fwd) src = (t > 0) ? xc.v[par][t - 1] : dsmem(&xc.v[par][R - 1][0], rank - 1);
          else src = (t < R - 1) ? xc.v[par][t + 1] : dsmem(&xc.v[par][0][0], rank + 1);
          const T k0 = coef(ju0, ju1, jlam, Sj0, Sj1, fwd ? -1 : +1);
#pragma unroll
          for (int k = 0; k < SG; ++k) acc[k] += k0 * src[k];
        }
#pragma unroll
        for (int k = 0; k < SG; ++k) {
          if (k >= ns) { xc.v[q & 1][t][k] = 0; prevx[k] = 0; continue; }
          const T x = fwd ? acc[k] * iD[k] : base[k] + acc[k] * iD[k];
          (fwd ? g.dQs : g.dQ)[(size_t)(NF + s0 + k) * N + c] = (double)x;
          xc.v[q & 1][t][k] = x;
          prevx[k] = x;
        }
        prevU[0] = u0;
        prevU[1] = u1;
        prevL = lam0;
        if (i == (fwd ? 0 : ni - 1)) {
#pragma unroll
          for (int k = 0; k < SG; ++k) firstx[k] = prevx[k];
          firstU[0] = u0;
          firstU[1] = u1;
          firstL = lam0;
        }
      }
      cluster_arrive();
    }
    cluster_wait();
  }
}


// ---------------------------------------------------------------------------------------
// K6c: 2D split sweeps, wavefront-record cluster kernel.  Same arithmetic as K6/K6b; the
// layout is built for GB300, where a dependent FP64 operation costs ~70 cycles and a scattered
// global load ~1 us: (1) k_pack_wave writes each cell's sweep inputs into a record, records
// stored hyperplane by hyperplane, so that the rows one CTA needs at a step are contiguous;
// (2) every CTA streams its chunk of records into a shared-memory ring with cp.async, kWaveD
// steps ahead; (3) between the cluster barrier's wait and arrive a row does only the coupling
// of the neighbouring row (an explicit NF x NF matrix built beforehand) and the diagonal
// scaling; the contribution of the row's previous cell and the next step's matrices are
// computed after the arrive, overlapping the barrier latency; (4) the value of a CTA's
// boundary row is pushed into the neighbouring CTA's shared memory before the arrive.
// ---------------------------------------------------------------------------------------
constexpr int kRecF = 24;            // flow record (compute-type values)
constexpr int kRecS = 20;            // species-group record
constexpr int kWaveD = 3;            // prefetch distance (steps)
constexpr int kWaveSlots = kWaveD + 1;
constexpr int kWaveRows = 32;        // max rows per CTA

// flow record fields
enum { RF_U = 0, RF_H = 2, RF_EV = 3, RF_BETA = 4, RF_PREV = 5, RF_PY = 6, RF_L0 = 7, RF_L1 = 8,
       RF_ID = 9, RF_IDEV = 10, RF_RHS = 11, RF_SIM = 16, RF_SIP = 18, RF_SJM = 20, RF_SJP = 22 };
// species-group record fields
enum { RS_U = 0, RS_L0 = 2, RS_L1 = 3, RS_SIM = 4, RS_SIP = 6, RS_SJM = 8, RS_SJP = 10,
       RS_RHS = 12, RS_ID = 16 };

__device__ __forceinline__ int wave_jlo(int h, int ni) { return h - ni + 1 > 0 ? h - ni + 1 : 0; }
__device__ __forceinline__ int wave_jhi(int h, int nj) { return h < nj - 1 ? h : nj - 1; }

template <class G, class T>
__global__ void __launch_bounds__(128) k_pack_wave(DevGrid g) {
  using A = Aux<G, 2>;
  constexpr int NF = A::NF, NS = G::NS, SG = kSpeciesGroup;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  const size_t N = g.N;
  const int ni = g.ni, i = c % ni, j = c / ni, h = i + j;
  const size_t w = (size_t)__ldg(&g.woff[h]) + (j - wave_jlo(h, ni));
  const double* W = g.W;
  const double* Si0 = g.S[0] + 3 * (size_t)face_of(g, 0, i, j, 0);
  const double* Si1 = g.S[0] + 3 * (size_t)face_of(g, 0, i + 1, j, 0);
  const double* Sj0 = g.S[1] + 3 * (size_t)face_of(g, 1, i, j, 0);
  const double* Sj1 = g.S[1] + 3 * (size_t)face_of(g, 1, i, j + 1, 0);
  T* r = static_cast<T*>(g.wrec) + w * kRecF;
  r[RF_U] = (T)W[A::U * N + c];
  r[RF_U + 1] = (T)W[(A::U + 1) * N + c];
  r[RF_H] = (T)W[A::H * N + c];
  r[RF_EV] = (G::NTEMP == 2) ? (T)W[A::EV * N + c] : T(0);
  r[RF_BETA] = (T)W[A::BETA * N + c];
  r[RF_PREV] = (T)W[A::PREV * N + c];
  r[RF_PY] = (T)W[A::PY * N + c];
  r[RF_L0] = (T)g.lamF[c];
  r[RF_L1] = (T)g.lamF[N + c];
  r[RF_ID] = (T)g.invD[c];
  r[RF_IDEV] = (T)g.invD[N + c];
#pragma unroll
  for (int v = 0; v < 5; ++v) r[RF_RHS + v] = v < NF ? (T)g.rhsF[v * N + c] : T(0);
  r[RF_SIM] = (T)Si0[0]; r[RF_SIM + 1] = (T)Si0[1];
  r[RF_SIP] = (T)Si1[0]; r[RF_SIP + 1] = (T)Si1[1];
  r[RF_SJM] = (T)Sj0[0]; r[RF_SJM + 1] = (T)Sj0[1];
  r[RF_SJP] = (T)Sj1[0]; r[RF_SJP + 1] = (T)Sj1[1];
  constexpr int NGRP = (NS + SG - 1) / SG;
#pragma unroll
  for (int gi = 0; gi < NGRP; ++gi) {
    T* q = static_cast<T*>(g.wrecs) + ((size_t)gi * N + w) * kRecS;
    q[RS_U] = r[RF_U];
    q[RS_U + 1] = r[RF_U + 1];
    q[RS_L0] = (T)g.lamC[c];
    q[RS_L1] = (T)g.lamC[N + c];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[RS_SIM + k] = r[RF_SIM + k];
#pragma unroll
    for (int k = 0; k < SG; ++k) {
      const int s = gi * SG + k;
      q[RS_RHS + k] = s < NS ? (T)(-g.R[(size_t)s * N + c]) : T(0);
      q[RS_ID + k] = s < NS ? (T)g.invD[(2 + s) * N + c] : T(0);
    }
  }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Copy the records of rows [j0-1, j0+R] of hyperplane h (those that exist) into a ring slot of
// (R+2) records; slot row index = j - (j0 - 1).  Whole CTA; the caller commits the group.
template <class T>
__device__ __forceinline__ void wave_fetch(const T* src, int rec, const int* woff, int h, int H,
                                           int ni, int nj, int j0, int R, T* slot) {
  if (h >= 0 && h <= H) {
    const int jlo = wave_jlo(h, ni), jhi = wave_jhi(h, nj);
    const int lo = max(j0 - 1, jlo), hi = min(j0 + R, jhi);
    if (lo <= hi) {
      const T* from = src + ((size_t)woff[h] + (lo - jlo)) * rec;
      T* to = slot + (size_t)(lo - (j0 - 1)) * rec;
      const int pieces = (hi - lo + 1) * rec * (int)sizeof(T) / 16;
      for (int k = threadIdx.x; k < pieces; k += blockDim.x)
        cp_async16(reinterpret_cast<char*>(to) + 16 * k, reinterpret_cast<const char*>(from) + 16 * k);
    }
  }
}

template <class G, class T>
__device__ __forceinline__ void rec_state(const T* r, CellState<G, 2, T>& w) {
  w.u[0] = r[RF_U];
  w.u[1] = r[RF_U + 1];
  w.H = r[RF_H];
  w.ev = r[RF_EV];
  w.beta = r[RF_BETA];
  w.prev = r[RF_PREV];
  w.pY = r[RF_PY];
}

// coupling matrix M of a neighbour (state w, radius lam, face S): minus side M = (A + lam)/2,
// plus side M = -(A - lam)/2, with A(S) the frozen-composition flow Jacobian of Sec. 2.3.1
// written out entry by entry (the matrix jvp_flow applies: columns rho, m_1, m_2, rhoE,
// [rho e_v])
template <class G, class T>
__device__ __forceinline__ void wave_matrix(const CellState<G, 2, T>& w, T lam, const T* S, int side,
                                            T (*M)[Aux<G, 2>::NF]) {
  constexpr int NF = Aux<G, 2>::NF;
  constexpr bool TWO = G::NTEMP == 2;
  const T U = w.u[0] * S[0] + w.u[1] * S[1];
  T A[NF][NF];
  A[0][0] = 0;
  A[1][0] = w.pY * S[0] - w.u[0] * U;
  A[2][0] = w.pY * S[1] - w.u[1] * U;
  A[3][0] = (w.pY - w.H) * U;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const T bu = w.beta * w.u[k];
    A[0][1 + k] = S[k];
    A[1][1 + k] = w.u[0] * S[k] - bu * S[0] + (k == 0 ? U : T(0));
    A[2][1 + k] = w.u[1] * S[k] - bu * S[1] + (k == 1 ? U : T(0));
    A[3][1 + k] = w.H * S[k] - bu * U;
  }
  A[0][3] = 0;
  A[1][3] = w.beta * S[0];
  A[2][3] = w.beta * S[1];
  A[3][3] = (T(1) + w.beta) * U;
  if (TWO) {
    A[NF - 1][0] = -w.ev * U;
    A[NF - 1][1] = w.ev * S[0];
    A[NF - 1][2] = w.ev * S[1];
    A[NF - 1][3] = 0;
    A[0][NF - 1] = 0;
    A[1][NF - 1] = w.prev * S[0];
    A[2][NF - 1] = w.prev * S[1];
    A[3][NF - 1] = w.prev * U;
    A[NF - 1][NF - 1] = U;
  }
  const T h = side < 0 ? T(0.5) : T(-0.5), l = side < 0 ? lam : -lam;
#pragma unroll
  for (int r = 0; r < NF; ++r)
#pragma unroll
    for (int c = 0; c < NF; ++c) M[r][c] = h * (A[r][c] + (r == c ? l : T(0)));
}

// contribution of x (at a cell with state w, radius lam) to the neighbour across face S on its
// side `side`: minus side (A x + lam x)/2, plus side -(A x - lam x)/2
template <class G, class T>
__device__ __forceinline__ void wave_contrib(const CellState<G, 2, T>& w, T lam, const T* S, int side,
                                             const T* x, T* out) {
  constexpr int NF = Aux<G, 2>::NF;
  T ax[NF];
  jvp_flow<G, 2, T>(w, S, x, ax);
#pragma unroll
  for (int v = 0; v < NF; ++v)
    out[v] = side < 0 ? T(0.5) * (ax[v] + lam * x[v]) : T(-0.5) * (ax[v] - lam * x[v]);
}

template <class G, class T, int ROWS = kWaveRows>
struct WaveSmemF {
  T ring[kWaveSlots][ROWS + 2][kRecF];
  T base[kWaveSlots][ROWS + 2][8];
  T x[2][ROWS][Aux<G, 2>::NF];
  T mbox[2][Aux<G, 2>::NF];
};

// BLK: one CTA holds every row (R = nj threads) and __syncthreads replaces the cluster barrier
template <class G, class T, int ROWS = kWaveRows, bool BLK = false>
__device__ void wave_flow(const DevGrid& g, int R, WaveSmemF<G, T, ROWS>& sm) {
  using A = Aux<G, 2>;
  constexpr int NF = A::NF;
  const size_t N = g.N;
  constexpr int D = BLK ? 2 : kWaveD;   // prefetch distance (see k_split_block)
  const unsigned rank = BLK ? 0u : cluster_ctarank(), C = BLK ? 1u : cluster_nctarank();
  const int t = threadIdx.x;
  const int ni = g.ni, nj = g.nj, H = ni + nj - 2;
  const int j0 = rank * R, j = j0 + t;
  const bool row = t < R && j < nj;
  const bool per = g.bc[0] == BC_PERIODIC;
  const T* rec = static_cast<const T*>(g.wrec);
  T* base = static_cast<T*>(g.wbase);
  for (int pass = 0; pass < 2; ++pass) {
    const bool fwd = pass == 0;
    const int hs = fwd ? 1 : -1;      // hyperplane step
    auto hof = [&](int q) { return fwd ? q : H - q; };
    if (!fwd) __threadfence();   // forward results in `base` are read back through cp.async
    for (int q = 0; q < D; ++q) {
      wave_fetch<T>(rec, kRecF, g.woff, hof(q), H, ni, nj, j0, R, &sm.ring[q % kWaveSlots][0][0]);
      if (!fwd) wave_fetch<T>(base, 8, g.woff, hof(q), H, ni, nj, j0, R, &sm.base[q % kWaveSlots][0][0]);
      cp_async_commit();
    }
    // FP32: the j-neighbour's coupling is built as a matrix before the barrier (cheap in
    // FP32, shortens the dependent chain after it); FP64: the neighbour's state is kept and its
    // Jacobian-vector product applied after the barrier (fewer FP64 operations per step, the
    // FP64 pipe being the narrow resource)
    constexpr bool kJvpJ = sizeof(T) == 8;
    T acc[NF], Mj[kJvpJ ? 1 : NF][NF], carry[NF], wrapc[NF], x[NF];
    T iD = 0, iDev = 0, lam0 = 0, Sn[2] = {0, 0}, Sw[2] = {0, 0};
    T jlam = 0, Sjv[2] = {0, 0};
    CellState<G, 2, T> ws, wjn;
    bool act = false, hasj = false;
    int cidx = 0, wcur = 0;
#pragma unroll
    for (int v = 0; v < NF; ++v) { carry[v] = 0; wrapc[v] = 0; x[v] = 0; }
    // per-step set-up from the records (step q); also used for the first step
    auto setup = [&](int q) {
      cp_async_wait<D - 1>();
      if (BLK) __syncthreads(); else __syncwarp();
      const int h = hof(q), i = h - j;
      act = row && q <= H && i >= 0 && i < ni;
      const int jj = j - hs;
      hasj = act && jj >= 0 && jj < nj;
      if (!act) return;
      const T* me = sm.ring[q % kWaveSlots][t + 1];
      rec_state<G, T>(me, ws);
      lam0 = me[RF_L0];
      Sn[0] = me[fwd ? RF_SIP : RF_SIM];          // face towards the next cell of the row
      Sn[1] = me[(fwd ? RF_SIP : RF_SIM) + 1];
      Sw[0] = me[fwd ? RF_SIM : RF_SIP];          // face across the periodic cut
      Sw[1] = me[(fwd ? RF_SIM : RF_SIP) + 1];
      iD = me[RF_ID];
      iDev = me[RF_IDEV];
      cidx = i + ni * j;
      wcur = __ldg(&g.woff[h]) + (j - wave_jlo(h, ni));
      const bool prev_exists = fwd ? i > 0 : i < ni - 1;
      const bool wrap = per && (fwd ? i == ni - 1 : i == 0);
#pragma unroll
      for (int v = 0; v < NF; ++v) {
        acc[v] = fwd ? me[RF_RHS + v] : T(0);
        if (prev_exists) acc[v] += carry[v];
        if (wrap) acc[v] += wrapc[v];
      }
      if (hasj) {
        const T* nb = sm.ring[(q + kWaveSlots - 1) % kWaveSlots][fwd ? t : t + 2];
        if constexpr (kJvpJ) {
          rec_state<G, T>(nb, wjn);
          jlam = nb[RF_L1];
          Sjv[0] = me[fwd ? RF_SJM : RF_SJP];
          Sjv[1] = me[(fwd ? RF_SJM : RF_SJP) + 1];
        } else {
          CellState<G, 2, T> wn;
          rec_state<G, T>(nb, wn);
          wave_matrix<G, T>(wn, nb[RF_L1], me + (fwd ? RF_SJM : RF_SJP), fwd ? -1 : +1, Mj);
        }
      }
    };
    setup(0);
    for (int q = 0; q <= H; ++q) {
      const int h = hof(q), i = h - j;
      if (!BLK && q > 0) cluster_wait();
      if (act) {
        if (hasj) {
          const bool remote = fwd ? t == 0 : t == R - 1;
          const T* src = remote ? sm.mbox[(q - 1) & 1] : sm.x[(q - 1) & 1][fwd ? t - 1 : t + 1];
          T xn[NF];
#pragma unroll
          for (int v = 0; v < NF; ++v) xn[v] = src[v];
          if constexpr (kJvpJ) {
            flow_contrib<G, T>(wjn, jlam, Sjv, xn, fwd ? -1 : +1, acc);
          } else {
#pragma unroll
            for (int r = 0; r < NF; ++r)
#pragma unroll
              for (int c = 0; c < NF; ++c) acc[r] += Mj[r][c] * xn[c];
          }
        }
        const T* bse = sm.base[q % kWaveSlots][t + 1];
#pragma unroll
        for (int v = 0; v < NF; ++v) {
          const T d = (G::NTEMP == 2 && v == NF - 1) ? iDev : iD;
          x[v] = fwd ? acc[v] * d : bse[v] + acc[v] * d;
          sm.x[q & 1][t][v] = x[v];
        }
        // push the CTA-boundary row to the neighbouring CTA
        if (fwd ? (t == R - 1 && rank + 1 < C) : (t == 0 && rank > 0)) {
          T* dst = dsmem(&sm.mbox[q & 1][0], fwd ? rank + 1 : rank - 1);
#pragma unroll
          for (int v = 0; v < NF; ++v) dst[v] = x[v];
        }
      }
      if (!BLK) cluster_arrive();
      if (act) {
        double* out = fwd ? g.dQs : g.dQ;
#pragma unroll
        for (int v = 0; v < NF; ++v) out[v * N + cidx] = (double)x[v];
        if (fwd) {
          T* b = base + (size_t)wcur * 8;
#pragma unroll
          for (int v = 0; v < NF; ++v) b[v] = x[v];
        }
        // contribution of this cell to the next cell of the row (minus side of that cell in
        // the forward sweep, plus side in the backward sweep) and across the periodic cut
        const bool next_exists = fwd ? i < ni - 1 : i > 0;
        if (next_exists) wave_contrib<G, T>(ws, lam0, Sn, fwd ? -1 : +1, x, carry);
        if (per && i == (fwd ? 0 : ni - 1)) wave_contrib<G, T>(ws, lam0, Sw, fwd ? +1 : -1, x, wrapc);
      }
      // prefetch step q + D, then prepare step q + 1
      if (q + D <= H) {
        wave_fetch<T>(rec, kRecF, g.woff, hof(q + D), H, ni, nj, j0, R,
                      &sm.ring[(q + D) % kWaveSlots][0][0]);
        if (!fwd)
          wave_fetch<T>(base, 8, g.woff, hof(q + D), H, ni, nj, j0, R,
                        &sm.base[(q + D) % kWaveSlots][0][0]);
      }
      cp_async_commit();        // one group per step, possibly empty
      setup(q + 1);
    }
    if (!BLK) cluster_wait();
    cp_async_wait<0>();
    if (BLK) __syncthreads(); else __syncwarp();
  }
}


template <class G, class T, int ROWS = kWaveRows>
struct WaveSmemS {
  T ring[kWaveSlots][ROWS + 2][kRecS];
  T base[kWaveSlots][ROWS + 2][kSpeciesGroup];
  T x[2][ROWS][kSpeciesGroup];
  T mbox[2][kSpeciesGroup];
};

// scalar coupling of a neighbour in the component operator: minus side (U + lam)/2, plus
// side -(U - lam)/2, U = u_nb . S_f (Sec. 2.3.2)
template <class T>
__device__ __forceinline__ T wave_coef(const T* u, T lam, const T* S, int side) {
  const T U = u[0] * S[0] + u[1] * S[1];
  return side < 0 ? T(0.5) * (U + lam) : T(-0.5) * (U - lam);
}

template <class G, class T, int ROWS = kWaveRows, bool BLK = false>
__device__ void wave_species(const DevGrid& g, int R, int grp, WaveSmemS<G, T, ROWS>& sm) {
  using A = Aux<G, 2>;
  constexpr int NF = A::NF, SG = kSpeciesGroup, NS = G::NS;
  const size_t N = g.N;
  constexpr int D = BLK ? 2 : kWaveD;   // prefetch distance (see k_split_block)
  const unsigned rank = BLK ? 0u : cluster_ctarank(), C = BLK ? 1u : cluster_nctarank();
  const int t = threadIdx.x;
  const int ni = g.ni, nj = g.nj, H = ni + nj - 2;
  const int j0 = rank * R, j = j0 + t;
  const bool row = t < R && j < nj;
  const bool per = g.bc[0] == BC_PERIODIC;
  const int s0 = grp * SG;
  const int ns = (NS - s0 < SG) ? NS - s0 : SG;
  const T* rec = static_cast<const T*>(g.wrecs) + (size_t)grp * N * kRecS;
  T* base = static_cast<T*>(g.wbase) + (size_t)N * 8 + (size_t)grp * N * SG;
  for (int pass = 0; pass < 2; ++pass) {
    const bool fwd = pass == 0;
    const int hs = fwd ? 1 : -1;
    auto hof = [&](int q) { return fwd ? q : H - q; };
    if (!fwd) __threadfence();
    for (int q = 0; q < D; ++q) {
      wave_fetch<T>(rec, kRecS, g.woff, hof(q), H, ni, nj, j0, R, &sm.ring[q % kWaveSlots][0][0]);
      if (!fwd) wave_fetch<T>(base, SG, g.woff, hof(q), H, ni, nj, j0, R, &sm.base[q % kWaveSlots][0][0]);
      cp_async_commit();
    }
    T acc[SG], iD[SG], carry[SG], wrapc[SG], x[SG], kj = 0, ki = 0, kw = 0;
    bool act = false, hasj = false;
    int cidx = 0, wcur = 0;
#pragma unroll
    for (int k = 0; k < SG; ++k) { carry[k] = 0; wrapc[k] = 0; x[k] = 0; iD[k] = 0; acc[k] = 0; }
    auto setup = [&](int q) {
      cp_async_wait<D - 1>();
      if (BLK) __syncthreads(); else __syncwarp();
      const int h = hof(q), i = h - j;
      act = row && q <= H && i >= 0 && i < ni;
      const int jj = j - hs;
      hasj = act && jj >= 0 && jj < nj;
      if (!act) return;
      const T* me = sm.ring[q % kWaveSlots][t + 1];
      cidx = i + ni * j;
      wcur = __ldg(&g.woff[h]) + (j - wave_jlo(h, ni));
      const bool prev_exists = fwd ? i > 0 : i < ni - 1;
      const bool wrap = per && (fwd ? i == ni - 1 : i == 0);
#pragma unroll
      for (int k = 0; k < SG; ++k) {
        iD[k] = me[RS_ID + k];
        acc[k] = fwd ? me[RS_RHS + k] : T(0);
        if (prev_exists) acc[k] += carry[k];
        if (wrap) acc[k] += wrapc[k];
      }
      if (hasj) {
        const T* nb = sm.ring[(q + kWaveSlots - 1) % kWaveSlots][fwd ? t : t + 2];
        kj = wave_coef<T>(nb + RS_U, nb[RS_L1], me + (fwd ? RS_SJM : RS_SJP), fwd ? -1 : +1);
      }
      ki = wave_coef<T>(me + RS_U, me[RS_L0], me + (fwd ? RS_SIP : RS_SIM), fwd ? -1 : +1);
      kw = wave_coef<T>(me + RS_U, me[RS_L0], me + (fwd ? RS_SIM : RS_SIP), fwd ? +1 : -1);
    };
    setup(0);
    for (int q = 0; q <= H; ++q) {
      const int h = hof(q), i = h - j;
      if (!BLK && q > 0) cluster_wait();
      if (act) {
        if (hasj) {
          const bool remote = fwd ? t == 0 : t == R - 1;
          const T* src = remote ? sm.mbox[(q - 1) & 1] : sm.x[(q - 1) & 1][fwd ? t - 1 : t + 1];
#pragma unroll
          for (int k = 0; k < SG; ++k) acc[k] += kj * src[k];
        }
        const T* bse = sm.base[q % kWaveSlots][t + 1];
#pragma unroll
        for (int k = 0; k < SG; ++k) {
          x[k] = fwd ? acc[k] * iD[k] : bse[k] + acc[k] * iD[k];
          sm.x[q & 1][t][k] = x[k];
        }
        if (fwd ? (t == R - 1 && rank + 1 < C) : (t == 0 && rank > 0)) {
          T* dst = dsmem(&sm.mbox[q & 1][0], fwd ? rank + 1 : rank - 1);
#pragma unroll
          for (int k = 0; k < SG; ++k) dst[k] = x[k];
        }
      }
      if (!BLK) cluster_arrive();
      if (act) {
        double* out = fwd ? g.dQs : g.dQ;
#pragma unroll
        for (int k = 0; k < SG; ++k)
          if (k < ns) out[(size_t)(NF + s0 + k) * N + cidx] = (double)x[k];
        if (fwd) {
          T* b = base + (size_t)wcur * SG;
#pragma unroll
          for (int k = 0; k < SG; ++k) b[k] = x[k];
        }
#pragma unroll
        for (int k = 0; k < SG; ++k) carry[k] = ki * x[k];
        if (per && i == (fwd ? 0 : ni - 1))
#pragma unroll
          for (int k = 0; k < SG; ++k) wrapc[k] = kw * x[k];
      }
      if (q + D <= H) {
        wave_fetch<T>(rec, kRecS, g.woff, hof(q + D), H, ni, nj, j0, R,
                      &sm.ring[(q + D) % kWaveSlots][0][0]);
        if (!fwd)
          wave_fetch<T>(base, SG, g.woff, hof(q + D), H, ni, nj, j0, R,
                        &sm.base[(q + D) % kWaveSlots][0][0]);
      }
      cp_async_commit();
      setup(q + 1);
    }
    if (!BLK) cluster_wait();
    cp_async_wait<0>();
    if (BLK) __syncthreads(); else __syncwarp();
  }
}

template <class G, class T>
__global__ void __launch_bounds__(32) k_split_wave(DevGrid g, int R) {
  constexpr size_t BF = sizeof(WaveSmemF<G, T>), BS = sizeof(WaveSmemS<G, T>);
  __shared__ __align__(16) char smem[BF > BS ? BF : BS];
  const int comp = blockIdx.x / (int)cluster_nctarank();   // uniform within a cluster
  if (comp == 0) wave_flow<G, T>(g, R, *reinterpret_cast<WaveSmemF<G, T>*>(smem));
  else wave_species<G, T>(g, R, comp - 1, *reinterpret_cast<WaveSmemS<G, T>*>(smem));
}

template <class G>
constexpr int species_clusters() { return (G::NS + kSpeciesGroup - 1) / kSpeciesGroup; }
// species clusters of the direct-load cluster kernel k_split_cluster
template <class G>
constexpr int cluster_species_clusters() { return (G::NS + kClusterSpeciesGroup - 1) / kClusterSpeciesGroup; }

// K6d: 2D split sweeps in FP32 with one CTA per component (the flow block, then one per group
// of 4 species) holding every row of the grid: same records and arithmetic as K6c, with
// __syncthreads between hyperplanes instead of a cluster barrier (FP32 throughput lets one SM
// carry all rows).  nj <= kBlockRows.  With several warps the prefetch distance is 2 (4 ring
// slots): the slot that the fetch at the end of step q overwrites was last read in the setup of
// step q - 1, which every warp has left at the block barrier of the setup of step q.
constexpr int kBlockRows = 384;
template <class G>
constexpr size_t block_smem_bytes() {
  return sizeof(WaveSmemF<G, float, kBlockRows>) > sizeof(WaveSmemS<G, float, kBlockRows>)
             ? sizeof(WaveSmemF<G, float, kBlockRows>)
             : sizeof(WaveSmemS<G, float, kBlockRows>);
}
template <class G>
__global__ void __launch_bounds__(kBlockRows) k_split_block(DevGrid g) {
  extern __shared__ __align__(16) char bsm[];
  const int comp = blockIdx.x;
  if (comp == 0)
    wave_flow<G, float, kBlockRows, true>(g, g.nj, *reinterpret_cast<WaveSmemF<G, float, kBlockRows>*>(bsm));
  else
    wave_species<G, float, kBlockRows, true>(g, g.nj, comp - 1,
                                             *reinterpret_cast<WaveSmemS<G, float, kBlockRows>*>(bsm));
}

template <class G, class T, int W>
__global__ void __launch_bounds__(32 * W) k_split_cluster(DevGrid g, int R) {
  constexpr int NV = Aux<G, 2>::NF > kClusterSpeciesGroup ? Aux<G, 2>::NF : kClusterSpeciesGroup;
  __shared__ Xchg<G, NV, double> xf;   // sized for the widest use
  __shared__ double accI[kClusterRows][Aux<G, 2>::NF];
  const int comp = blockIdx.x / (int)cluster_nctarank();   // uniform within a cluster
  if (comp == 0) {
    if constexpr (W == 2)
      sweep_flow_cluster2<G, T>(g, R, *reinterpret_cast<Xchg<G, Aux<G, 2>::NF, T>*>(&xf),
                                *reinterpret_cast<T(*)[kClusterRows][Aux<G, 2>::NF]>(&accI));
    else
      sweep_flow_cluster1<G, T>(g, R, *reinterpret_cast<Xchg<G, Aux<G, 2>::NF, T>*>(&xf));
  }
  else sweep_species_cluster<G, T>(g, R, (comp - 1) * kClusterSpeciesGroup,
                                   *reinterpret_cast<Xchg<G, kClusterSpeciesGroup, T>*>(&xf));
}

// ---------------------------------------------------------------------------------------
// K6e: split sweeps of a 2D grid with the neighbour couplings assembled beforehand (FP64, or
// FP32 for the mixed-precision operator).
// The coupling of cell c with a neighbour nb across face S is the linear map
// x_nb -> D_c^-1 (+-1/2)(A_nb(S) x_nb +- lambda_nb x_nb) (Sec. 2.2, 2.3.1-2.3.2): it depends
// only on the state frozen for the iteration, not on the increments.  k_sweep_mat forms it for
// every cell and face in one fully parallel launch (the flow block as an NF x NF matrix, the
// species as one scalar shared by every species before the species' own D_s^-1), so the sweep
// itself is left with the dependent part alone: per cell and step a dot product of length NF
// per flow component.  GB300 issues one warp-wide FP64 FMA per SM sub-partition only every
// ~64 cycles, which made the matrix-free Jacobian product (tens of FP64 operations after every
// cluster barrier, on one or two sub-partitions) the bound of K6b; here each row of a CTA has
// kMatSlots threads, one per flow component (or species of the CTA's group), and a CTA's rows
// cover all four sub-partitions.
// Record of cell c (elements of the operator's type T, in which they are also formed: FP64, or
// FP32 for the mixed-precision operator): flow blocks [fwd i][fwd j][bwd i][bwd j], each NF
// rows of NP (NF rounded up to a whole 16-byte load, so that every row starts on 16 bytes),
// then the species coefficients in the same order.  Per row j after the N cell records: the
// periodic-i wrap couplings (forward: cell (ni-1, j) with (0, j); backward: (0, j) with
// (ni-1, j)), flow blocks then species coefficients.  k_split_mat (the cluster-barrier form)
// is FP64 only.
// ---------------------------------------------------------------------------------------
constexpr int kMatSlots = 8;       // threads per row of a CTA
constexpr int kMatSpecies = kMatSlots;

template <class G, class T = double>
struct MatRec {
  static constexpr int NF = Aux<G, 2>::NF;
  static constexpr int VEC = 16 / (int)sizeof(T);     // elements of one 16-byte load
  static constexpr int NP = (NF + VEC - 1) / VEC * VEC;
  static constexpr int BLK = NF * NP;
  static constexpr int CELL = 4 * BLK + 4;
  static constexpr int ROW = 2 * BLK + 4;
  static_assert(NF <= kMatSlots, "one thread per flow component");
  static_assert(CELL % VEC == 0, "cell records start on 16 bytes");
};
template <class T> struct Vec16;
template <> struct Vec16<double> {
  using type = double2;
  __device__ static void unpack(const double2& a, double* o) { o[0] = a.x; o[1] = a.y; }
};
template <> struct Vec16<float> {
  using type = float4;
  __device__ static void unpack(const float4& a, float* o) {
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  }
};
template <class G>
constexpr int mat_species_groups() { return (G::NS + kMatSpecies - 1) / kMatSpecies; }

// D_c^-1 (+-1/2)(A_nb(S) +- lambda I) of the flow block, written row-major with pitch NP
template <class G, class T>
__device__ __forceinline__ void mat_block(const DevGrid& g, int nb, const double* S, double lam,
                                          int side, double dF, double dEv, T* out) {
  constexpr int NF = MatRec<G, T>::NF, NP = MatRec<G, T>::NP;
  // formed in the operator's own type: FP64, or FP32 for the FP32 operator (whose sweep reads
  // the couplings as FP32 anyway)
  CellState<G, 2, T> w;
  load_state<G, 2, T>(g, nb, w);
  const T Sf[2] = {(T)S[0], (T)S[1]};
  const T lamT = (T)lam, dFT = (T)dF, dEvT = (T)dEv;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    T e[NF], a[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) e[q] = q == k ? T(1) : T(0);
    jvp_flow<G, 2, T>(w, Sf, e, a);
#pragma unroll
    for (int v = 0; v < NF; ++v) {
      const T l = v == k ? lamT : T(0);
      const T m = side < 0 ? T(0.5) * (a[v] + l) : T(-0.5) * (a[v] - l);
      out[v * NP + k] = ((G::NTEMP == 2 && v == NF - 1) ? dEvT : dFT) * m;
    }
  }
#pragma unroll
  for (int v = 0; v < NF; ++v)
#pragma unroll
    for (int k = NF; k < NP; ++k) out[v * NP + k] = T(0);
}

// species coupling (+-1/2)(U_nb +- lambda_C,nb) before D_s^-1, U_nb = u_nb . S
template <class G>
__device__ __forceinline__ double mat_coef(const DevGrid& g, int nb, const double* S, double lam, int side) {
  using A = Aux<G, 2>;
  const size_t N = g.N;
  const double U = g.W[A::U * N + nb] * S[0] + g.W[(A::U + 1) * N + nb] * S[1];
  return side < 0 ? 0.5 * (U + lam) : -0.5 * (U - lam);
}

template <class G, class T>
__global__ void __launch_bounds__(128) k_sweep_mat(DevGrid g) {
  using M = MatRec<G, T>;
  constexpr int BLK = M::BLK;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  const size_t N = g.N;
  const int ni = g.ni, nj = g.nj, i = c % ni, j = c / ni;
  const double dF = g.invD[c], dEv = g.invD[N + c];
  T* rec = reinterpret_cast<T*>(g.SMC) + (size_t)c * M::CELL;
  T* co = rec + 4 * BLK;
  const double* S;
  // a face on the grid's boundary couples nothing: its block and coefficient are zero
  if (i == 0 || j == 0 || i == ni - 1 || j == nj - 1) {
    for (int e = 0; e < M::CELL; ++e) rec[e] = T(0);
  }
  // forward: the lower neighbours (i-1, j) and (i, j-1); backward: the upper ones
  if (i > 0) {
    S = g.S[0] + 3 * (size_t)face_of(g, 0, i, j, 0);
    mat_block<G, T>(g, c - 1, S, g.lamF[c - 1], -1, dF, dEv, rec);
    co[0] = (T)mat_coef<G>(g, c - 1, S, g.lamC[c - 1], -1);
  }
  if (j > 0) {
    S = g.S[1] + 3 * (size_t)face_of(g, 1, i, j, 0);
    mat_block<G, T>(g, c - ni, S, g.lamF[N + c - ni], -1, dF, dEv, rec + BLK);
    co[1] = (T)mat_coef<G>(g, c - ni, S, g.lamC[N + c - ni], -1);
  }
  if (i < ni - 1) {
    S = g.S[0] + 3 * (size_t)face_of(g, 0, i + 1, j, 0);
    mat_block<G, T>(g, c + 1, S, g.lamF[c + 1], +1, dF, dEv, rec + 2 * BLK);
    co[2] = (T)mat_coef<G>(g, c + 1, S, g.lamC[c + 1], +1);
  }
  if (j < nj - 1) {
    S = g.S[1] + 3 * (size_t)face_of(g, 1, i, j + 1, 0);
    mat_block<G, T>(g, c + ni, S, g.lamF[N + c + ni], +1, dF, dEv, rec + 3 * BLK);
    co[3] = (T)mat_coef<G>(g, c + ni, S, g.lamC[N + c + ni], +1);
  }
  if (g.bc[0] == BC_PERIODIC) {
    T* pr = reinterpret_cast<T*>(g.SMC) + N * M::CELL + (size_t)j * M::ROW;
    if (i == ni - 1) {          // forward: (0, j) precedes (ni-1, j) and lies on its + side
      const int nb = ni * j;
      S = g.S[0] + 3 * (size_t)face_of(g, 0, ni, j, 0);
      mat_block<G, T>(g, nb, S, g.lamF[nb], +1, dF, dEv, pr);
      pr[2 * BLK] = (T)mat_coef<G>(g, nb, S, g.lamC[nb], +1);
    }
    if (i == 0) {               // backward: (ni-1, j) precedes (0, j) and lies on its - side
      const int nb = ni - 1 + ni * j;
      S = g.S[0] + 3 * (size_t)face_of(g, 0, 0, j, 0);
      mat_block<G, T>(g, nb, S, g.lamF[nb], -1, dF, dEv, pr + BLK);
      pr[2 * BLK + 1] = (T)mat_coef<G>(g, nb, S, g.lamC[nb], -1);
    }
  }
}

// inputs of one thread's cell at step q (loaded a step ahead)
template <class G, class T = double>
struct MatStep {
  // raw loads only (no arithmetic on them here, so that a prefetch does not wait for its own
  // loads): the coupling rows (species: the two coefficients before D_s^-1), the diagonal
  // inverse d and base = the right-hand side (forward) or the forward result (backward)
  T bi[MatRec<G, T>::NP], bj[MatRec<G, T>::NP], base, d;
  int c, i;
  bool act;
};

template <class G, class T = double>
__device__ __forceinline__ void mat_step_load(const DevGrid& g, int q, int j, bool on, bool fwd,
                                              bool flow, int v, int s, MatStep<G, T>& m) {
  using M = MatRec<G, T>;
  using V = typename Vec16<T>::type;
  constexpr int VEC = M::VEC;
  constexpr int NF = M::NF, NP = M::NP, BLK = M::BLK;
  const int ni = g.ni, H = ni + g.nj - 2;
  const int i = (fwd ? q : H - q) - j;
  m.act = on && q <= H && i >= 0 && i < ni;
  m.i = i;
  if (!m.act) return;
  const size_t N = g.N;
  const int c = i + ni * j;
  m.c = c;
  const T* rec = reinterpret_cast<const T*>(g.SMC) + (size_t)c * M::CELL;
  if (flow) {
    const V* ri = reinterpret_cast<const V*>(rec + (fwd ? 0 : 2 * BLK) + v * NP);
    const V* rj = reinterpret_cast<const V*>(rec + (fwd ? BLK : 3 * BLK) + v * NP);
#pragma unroll
    for (int k = 0; k < NP / VEC; ++k) {
      Vec16<T>::unpack(ri[k], m.bi + VEC * k);
      Vec16<T>::unpack(rj[k], m.bj + VEC * k);
    }
    m.d = (T)g.invD[((G::NTEMP == 2 && v == NF - 1) ? N : 0) + c];
    m.base = (T)(fwd ? g.rhsF[v * N + c] : g.dQs[v * N + c]);
  } else {
    m.d = (T)g.invD[(2 + s) * N + c];
    m.base = (T)(fwd ? -g.R[(size_t)s * N + c] : g.dQs[(size_t)(NF + s) * N + c]);
    const T* co = rec + 4 * BLK;
    m.bi[0] = co[fwd ? 0 : 2];
    m.bj[0] = co[fwd ? 1 : 3];
  }
}

template <class G>
__global__ void __launch_bounds__(kMatSlots * kClusterRows) k_split_mat(DevGrid g, int R) {
  using M = MatRec<G>;
  constexpr int NF = M::NF, NP = M::NP, BLK = M::BLK;
  __shared__ __align__(16) double xs[2][kClusterRows][kMatSlots];
  const size_t N = g.N;
  const int comp = blockIdx.x / (int)cluster_nctarank();   // 0: flow block, else a species group
  const unsigned rank = cluster_ctarank();
  const int t = threadIdx.x / kMatSlots, v = threadIdx.x % kMatSlots;
  const int j = rank * R + t;
  const int ni = g.ni, nj = g.nj, H = ni + nj - 2;
  const bool per = g.bc[0] == BC_PERIODIC;
  const bool flow = comp == 0;
  const int s = (comp - 1) * kMatSpecies + v;
  const bool on = t < R && j < nj && (flow ? v < NF : s < G::NS);
  for (int pass = 0; pass < 2; ++pass) {
    const bool fwd = pass == 0;
    double xp[NF], xf[NF], pw[NP];   // flow: the row's previous and first results, wrap block row
    double sp = 0.0, sf = 0.0, pc = 0.0;
#pragma unroll
    for (int k = 0; k < NF; ++k) xp[k] = xf[k] = 0.0;
#pragma unroll
    for (int k = 0; k < NP; ++k) pw[k] = 0.0;
    if (on && per) {
      const double* pr = g.SMC + N * M::CELL + (size_t)j * M::ROW;
      if (flow) {
#pragma unroll
        for (int k = 0; k < NP; ++k) pw[k] = pr[(fwd ? 0 : BLK) + v * NP + k];
      } else {
        pc = pr[2 * BLK + (fwd ? 0 : 1)];
      }
    }
    double* out = fwd ? g.dQs : g.dQ;
    const size_t orow = (size_t)(flow ? v : NF + s) * N;
    MatStep<G> cur, nxt;
    mat_step_load<G>(g, 0, j, on, fwd, flow, v, s, cur);
    for (int q = 0; q <= H; ++q) {
      mat_step_load<G>(g, q + 1, j, on, fwd, flow, v, s, nxt);     // prefetch the next step
      // the row's own earlier cells (and the periodic wrap) need no other CTA: coupled while the
      // cluster barrier is pending
      double acc = 0.0;
      if (cur.act) {
        const int i = cur.i;
        acc = fwd ? cur.d * cur.base : cur.base;
        const bool hasi = fwd ? i > 0 : i < ni - 1;
        const bool wrap = per && i == (fwd ? ni - 1 : 0);
        if (flow) {
          if (hasi) {
#pragma unroll
            for (int k = 0; k < NF; ++k) acc += cur.bi[k] * xp[k];
          }
          if (wrap) {
#pragma unroll
            for (int k = 0; k < NF; ++k) acc += pw[k] * xf[k];
          }
        } else {
          if (hasi) acc += (cur.d * cur.bi[0]) * sp;
          if (wrap) acc += cur.d * pc * sf;
        }
      }
      if (q > 0) cluster_wait();
      if (cur.act) {
        // the neighbouring row's result of step q-1: this CTA's shared memory or, across a CTA
        // boundary, the neighbour CTA's
        if (fwd ? j > 0 : j < nj - 1) {
          const int par = (q - 1) & 1;
          const double* src;
          if (fwd) src = (t > 0) ? xs[par][t - 1] : dsmem(&xs[par][R - 1][0], rank - 1);
          else src = (t < R - 1) ? xs[par][t + 1] : dsmem(&xs[par][0][0], rank + 1);
          if (flow) {
            // two partial sums: a shorter chain of dependent FP64 operations
            double a0 = acc, a1 = 0.0;
#pragma unroll
            for (int k = 0; k < NF; ++k) {
              if (k & 1) a1 += cur.bj[k] * src[k];
              else a0 += cur.bj[k] * src[k];
            }
            acc = a0 + a1;
          } else {
            acc += (cur.d * cur.bj[0]) * src[v];
          }
        }
        xs[q & 1][t][v] = acc;
      }
      __syncwarp();                    // a row's kMatSlots threads share one warp
      cluster_arrive();
      // after the arrive: its release then covers only the shared-memory exchange, not the
      // global store (which the next step's release finds long completed)
      if (cur.act) {
        out[orow + cur.c] = acc;
        if (flow) {
#pragma unroll
          for (int k = 0; k < NF; ++k) xp[k] = xs[q & 1][t][k];
        } else {
          sp = acc;
        }
        if (cur.i == (fwd ? 0 : ni - 1)) {
#pragma unroll
          for (int k = 0; k < NF; ++k) xf[k] = xp[k];
          sf = sp;
        }
      }
      cur = nxt;
    }
    cluster_wait();
  }
}

// Point-to-point form of K6e: the rows of a CTA step together (__syncthreads between
// hyperplanes) and only the row at a CTA boundary talks to the neighbouring CTA, by writing its
// result straight into that CTA's shared memory (st.async) and completing a per-hyperplane
// mbarrier there.  No cluster-wide barrier per step: a CTA waits only for the data it needs, so
// a CTA can run ahead of the ones downstream and the cross-CTA latency is paid once per CTA
// boundary rather than once per hyperplane.  The receiving ring holds one slot per hyperplane
// of a pass (its mbarrier completes one phase per pass; every slot's expected byte count is
// registered before a cluster barrier that precedes all sends of the pass).
constexpr long kP2PSpinLimit = 1L << 22;   // bounded waits (then ST_TIMEOUT)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t cluster_map(uint32_t a, unsigned rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ bool p2p_wait(uint32_t bar, uint32_t parity) {
  for (long it = 0; it < kP2PSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// Inputs of one thread for one hyperplane step of k_split_p2p, staged in shared memory by
// cp.async kP2PStageD steps ahead (one slot per thread and step, a ring of kP2PStageD + 1
// slots): the coupling rows bi, bj (NP elements of T each; species: the two coefficients), then
// the raw FP64 diagonal inverse d and base (right-hand side forward, forward result backward).
#ifndef CS_P2P_STAGE
#define CS_P2P_STAGE 6
#endif
constexpr int kP2PStageD = CS_P2P_STAGE;
template <class T, int NP>
struct P2PSlot {
  static constexpr int BYTES = 2 * NP * (int)sizeof(T) + 2 * (int)sizeof(double);
  static_assert(BYTES % 16 == 0, "slots start on 16 bytes");
};
// dynamic shared memory of k_split_p2p: the ring [H + 1][kMatSlots] of T, H + 1 mbarriers, then
// (from a 16-byte boundary) the staging ring [kP2PStageD + 1][threads] of slots
template <class T>
__host__ __device__ inline size_t p2p_ring_bytes(int ni, int nj) {
  return ((size_t)(ni + nj - 1) * (kMatSlots * sizeof(T) + sizeof(unsigned long long)) + 15) / 16 * 16;
}
template <class T, int NP>
__host__ __device__ inline size_t p2p_smem_bytes(int ni, int nj, int threads) {
  return p2p_ring_bytes<T>(ni, nj) + (size_t)(kP2PStageD + 1) * threads * P2PSlot<T, NP>::BYTES;
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

// Issue the copies of step q's inputs of this thread into its slot (nothing for a step whose
// cell does not exist; the caller commits one group per step).
template <class G, class T>
__device__ __forceinline__ void p2p_stage_issue(const DevGrid& g, int q, int j, bool on, bool fwd,
                                                bool flow, int v, int s, unsigned char* slot) {
  using M = MatRec<G, T>;
  constexpr int NF = M::NF, NP = M::NP, BLK = M::BLK;
  const int ni = g.ni, H = ni + g.nj - 2;
  const int i = (fwd ? q : H - q) - j;
  if (!(on && q <= H && i >= 0 && i < ni)) return;
  const size_t N = g.N;
  const int c = i + ni * j;
  const T* rec = reinterpret_cast<const T*>(g.SMC) + (size_t)c * M::CELL;
  T* bi = reinterpret_cast<T*>(slot);
  T* bj = bi + NP;
  double* db = reinterpret_cast<double*>(bj + NP);
  if (flow) {
    const T* ri = rec + (fwd ? 0 : 2 * BLK) + v * NP;
    const T* rj = rec + (fwd ? BLK : 3 * BLK) + v * NP;
#pragma unroll
    for (int k = 0; k < NP * (int)sizeof(T) / 16; ++k) {
      cp_async16(reinterpret_cast<char*>(bi) + 16 * k, reinterpret_cast<const char*>(ri) + 16 * k);
      cp_async16(reinterpret_cast<char*>(bj) + 16 * k, reinterpret_cast<const char*>(rj) + 16 * k);
    }
    cp_async8(db, g.invD + ((G::NTEMP == 2 && v == NF - 1) ? N : 0) + c);
    cp_async8(db + 1, fwd ? g.rhsF + v * N + c : g.dQs + v * N + c);
  } else {
    const T* co = rec + 4 * BLK + (fwd ? 0 : 2);
    if (sizeof(T) == 8) {
      cp_async16(bi, co);            // the two coefficients, one 16-byte piece
    } else {
      cp_async4(bi, co);
      cp_async4(bj, co + 1);
    }
    cp_async8(db, g.invD + (2 + s) * N + c);
    cp_async8(db + 1, fwd ? g.R + (size_t)s * N + c : g.dQs + (size_t)(NF + s) * N + c);
  }
}
// Step q's inputs from this thread's slot (valid once the slot's copies have completed)
template <class G, class T>
__device__ __forceinline__ void p2p_stage_read(const DevGrid& g, int q, int j, bool on, bool fwd,
                                               bool flow, const unsigned char* slot,
                                               MatStep<G, T>& m) {
  using M = MatRec<G, T>;
  constexpr int NP = M::NP;
  const int ni = g.ni, H = ni + g.nj - 2;
  const int i = (fwd ? q : H - q) - j;
  m.act = on && q <= H && i >= 0 && i < ni;
  m.i = i;
  if (!m.act) return;
  m.c = i + ni * j;
  const T* bi = reinterpret_cast<const T*>(slot);
  const T* bj = bi + NP;
  const double* db = reinterpret_cast<const double*>(bj + NP);
  if (flow) {
#pragma unroll
    for (int k = 0; k < NP; ++k) { m.bi[k] = bi[k]; m.bj[k] = bj[k]; }
    m.d = (T)db[0];
    m.base = (T)db[1];
  } else {
    if (sizeof(T) == 8) {
      m.bi[0] = bi[0];
      m.bj[0] = bi[1];
    } else {
      m.bi[0] = bi[0];
      m.bj[0] = bj[0];
    }
    m.d = (T)db[0];
    m.base = (T)(fwd ? -db[1] : db[1]);
  }
}
// one element into another CTA's shared memory, completing bytes on that CTA's mbarrier
__device__ __forceinline__ void st_async(uint32_t dst, double v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];\n"
               ::"r"(dst), "l"(__double_as_longlong(v)), "r"(bar) : "memory");
}
__device__ __forceinline__ void st_async(uint32_t dst, float v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];\n"
               ::"r"(dst), "r"(__float_as_uint(v)), "r"(bar) : "memory");
}

template <class G, class T>
__global__ void __launch_bounds__(kMatSlots * kClusterRows) k_split_p2p(DevGrid g, int R) {
  using M = MatRec<G, T>;
  constexpr int NF = M::NF, NP = M::NP, BLK = M::BLK;
  extern __shared__ __align__(16) unsigned char p2p_dyn[];
  __shared__ __align__(16) T xs[2][kClusterRows][kMatSlots];
  const int ni = g.ni, nj = g.nj, H = ni + nj - 2;
  T* ring = reinterpret_cast<T*>(p2p_dyn);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(ring + (size_t)(H + 1) * kMatSlots);
  constexpr int SB = P2PSlot<T, NP>::BYTES, S = kP2PStageD + 1;
  unsigned char* stage = p2p_dyn + p2p_ring_bytes<T>(ni, nj);
  auto slot_of = [&](int q) { return stage + ((size_t)(q % S) * blockDim.x + threadIdx.x) * SB; };
  const size_t N = g.N;
  const int comp = blockIdx.x / (int)cluster_nctarank();   // 0: flow block, else a species group
  const unsigned rank = cluster_ctarank();
  const int t = threadIdx.x / kMatSlots, v = threadIdx.x % kMatSlots;
  const int j = rank * R + t;
  const bool per = g.bc[0] == BC_PERIODIC;
  const bool flow = comp == 0;
  const int s = (comp - 1) * kMatSpecies + v;
  const bool on = t < R && j < nj && (flow ? v < NF : s < G::NS);
  // elements one boundary row sends per hyperplane: one per active slot
  const int nsend = flow ? NF : (G::NS - (comp - 1) * kMatSpecies < kMatSpecies ? G::NS - (comp - 1) * kMatSpecies : kMatSpecies);
  for (int q = threadIdx.x; q <= H; q += blockDim.x)
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar + q)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  __syncthreads();
  bool timed_out = false;
  for (int pass = 0; pass < 2; ++pass) {
    const bool fwd = pass == 0;
    // this pass's expected bytes per slot: the CTA's first (forward) or last (backward) row
    // receives its neighbouring row's result of the previous hyperplane from the next CTA
    if (threadIdx.x < 32) {
      const int jc = fwd ? (int)rank * R : (int)rank * R + R - 1;
      const bool row_ok = jc < nj && (fwd ? jc > 0 : jc + 1 < nj);
      for (int q = threadIdx.x; q <= H; q += 32) {
        const int ic = (fwd ? q : H - q) - jc;
        const uint32_t bytes = (row_ok && ic >= 0 && ic < ni) ? nsend * (uint32_t)sizeof(T) : 0u;
        unsigned long long st;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;\n"
                     : "=l"(st) : "r"(smem_u32(mbar + q)), "r"(bytes) : "memory");
      }
    }
    if (!fwd) __threadfence();   // forward results are read back through cp.async (L2)
    cluster_arrive();
    cluster_wait();
    T xp[NF], xf[NF], pw[NP];   // flow: the row's previous and first results, wrap block row
    T sp = 0, sf = 0, pc = 0;
#pragma unroll
    for (int k = 0; k < NF; ++k) xp[k] = xf[k] = T(0);
#pragma unroll
    for (int k = 0; k < NP; ++k) pw[k] = T(0);
    if (on && per) {
      const T* pr = reinterpret_cast<const T*>(g.SMC) + N * M::CELL + (size_t)j * M::ROW;
      if (flow) {
#pragma unroll
        for (int k = 0; k < NP; ++k) pw[k] = pr[(fwd ? 0 : BLK) + v * NP + k];
      } else {
        pc = pr[2 * BLK + (fwd ? 0 : 1)];
      }
    }
    double* out = fwd ? g.dQs : g.dQ;
    const size_t orow = (size_t)(flow ? v : NF + s) * N;
    // the row whose neighbour lives in the next CTA of this pass's direction, and the receiver
    const bool boundary_in = fwd ? t == 0 : t == R - 1;
    const bool boundary_out = fwd ? t == R - 1 : t == 0;
    const unsigned peer = fwd ? rank + 1 : rank - 1;
    const bool hasj = fwd ? j > 0 : j < nj - 1;
    const bool sends = fwd ? j + 1 < nj : j > 0;
    // the inputs of step q were copied kP2PStageD steps ahead into this thread's slot q mod S
    auto step = [&](int q) {
      cp_async_wait<kP2PStageD - 1>();    // this thread's copies of step q have landed
      MatStep<G, T> cur;
      p2p_stage_read<G, T>(g, q, j, on, fwd, flow, slot_of(q), cur);
      p2p_stage_issue<G, T>(g, q + kP2PStageD, j, on, fwd, flow, v, s, slot_of(q + kP2PStageD));
      cp_async_commit();                   // one group per step, possibly empty
      // the row's own earlier cells (and the periodic wrap) need no other row: coupled before
      // this step's synchronisation
      T acc = 0;
      if (cur.act) {
        acc = fwd ? cur.d * cur.base : cur.base;
        const bool hasi = fwd ? cur.i > 0 : cur.i < ni - 1;
        const bool wrap = per && cur.i == (fwd ? ni - 1 : 0);
        if (flow) {
          if (hasi) {
#pragma unroll
            for (int k = 0; k < NF; ++k) acc += cur.bi[k] * xp[k];
          }
          if (wrap) {
#pragma unroll
            for (int k = 0; k < NF; ++k) acc += pw[k] * xf[k];
          }
        } else {
          if (hasi) acc += (cur.d * cur.bi[0]) * sp;
          if (wrap) acc += cur.d * pc * sf;
        }
      }
      if (q > 0) __syncthreads();      // the CTA's results of step q-1 are in xs
      if (cur.act) {
        // the neighbouring row's result of step q-1; across a CTA boundary the neighbouring CTA
        // wrote it into ring slot q
        if (hasj) {
          const T* src;
          if (!boundary_in) {
            src = xs[(q - 1) & 1][fwd ? t - 1 : t + 1];
          } else {
            // after a wait has run out the results are invalid anyway: no further waits, so
            // that a failed exchange costs one wait bound, not one per step
            if (!timed_out && !p2p_wait(smem_u32(mbar + q), (uint32_t)pass)) {
              timed_out = true;
              set_status(g, ST_TIMEOUT, cur.c);
            }
            src = ring + (size_t)q * kMatSlots;
          }
          if (flow) {
#pragma unroll
            for (int k = 0; k < NF; ++k) acc += cur.bj[k] * src[k];
          } else {
            acc += (cur.d * cur.bj[0]) * src[v];
          }
        }
        xs[q & 1][t][v] = acc;
        if (boundary_out && sends) {
          const uint32_t dst = cluster_map(smem_u32(ring + (size_t)(q + 1) * kMatSlots + v), peer);
          st_async(dst, acc, cluster_map(smem_u32(mbar + q + 1), peer));
        }
        out[orow + cur.c] = (double)acc;
      }
      __syncwarp();                    // a row's kMatSlots threads share one warp
      if (cur.act) {
        if (flow) {
#pragma unroll
          for (int k = 0; k < NF; ++k) xp[k] = xs[q & 1][t][k];
        } else {
          sp = xs[q & 1][t][v];
        }
        if (cur.i == (fwd ? 0 : ni - 1)) {
#pragma unroll
          for (int k = 0; k < NF; ++k) xf[k] = xp[k];
          sf = sp;
        }
      }
    };
#pragma unroll 1
    for (int q = 0; q < kP2PStageD; ++q) {
      p2p_stage_issue<G, T>(g, q, j, on, fwd, flow, v, s, slot_of(q));
      cp_async_commit();
    }
#pragma unroll 1
    for (int q = 0; q <= H; ++q) step(q);
    cp_async_wait<0>();
    __syncthreads();
  }
  // no CTA leaves while a neighbour may still write into its shared memory
  cluster_arrive();
  cluster_wait();
}

// ---------------------------------------------------------------------------------------
// K7: consistency corrections and update (Sec. 2.3.3; CS-1 weight W_s = Y_s, negative
// densities clipped to 0 and counted).
// mode 1: CS-1, 2: CS-2 (dQ in split layout), 0: coupled update (CI layout).
// ---------------------------------------------------------------------------------------
// New conserved state qn of cell c for the increment alpha * dq with the correction of `mode`
// (rs: the cell's species densities, rho their sum); false for a non-physical result.
template <class G, int ND>
__device__ __forceinline__ bool cell_update(const DevGrid& g, int mode, int clip, const double* dq,
                                            int c, const double* rs, double rho, double alpha,
                                            double* qn, int& nclip) {
  using A = Aux<G, ND>;
  constexpr int NS = G::NS, NF = A::NF;
  const size_t N = g.N;
  nclip = 0;
  const double drho = alpha * dq[c];
  const double rnew = rho + drho;
  if (!(rnew > 0.0)) return false;
  double out[NS];
  if (mode == 1) {
    double sd = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) sd += alpha * dq[(NF + s) * N + c];
    const double irho = 1.0 / rho, rem = drho - sd;
#pragma unroll
    for (int s = 0; s < NS; ++s) out[s] = rs[s] + alpha * dq[(NF + s) * N + c] + rs[s] * irho * rem;
  } else if (mode == 2) {
    double t[NS], sum = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      t[s] = rs[s] + alpha * dq[(NF + s) * N + c];
      if (clip && t[s] < 0.0) { t[s] = 0.0; ++nclip; }
      sum += t[s];
    }
    if (!(sum > 0.0)) return false;
    const double f = rnew / sum;
#pragma unroll
    for (int s = 0; s < NS; ++s) out[s] = t[s] * f;
  } else {
    // coupled update: the first species is the remainder of the new total density
    double sum = 0.0;
#pragma unroll
    for (int s = 1; s < NS; ++s) {
      out[s] = rs[s] + alpha * dq[(NF + s - 1) * N + c];
      sum += out[s];
    }
    out[0] = rnew - sum;
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double v = out[s];
    if (clip && v < 0.0 && mode != 2) { v = 0.0; ++nclip; }
    qn[s] = v;
  }
#pragma unroll
  for (int q = 1; q < NF; ++q) {
    double v = g.Q[(NS + q - 1) * N + c] + alpha * dq[q * N + c];
    if (clip && G::NTEMP == 2 && q == NF - 1 && v < 0.0) { v = 0.0; ++nclip; }
    qn[NS + q - 1] = v;
  }
  return true;
}

// Specific energies of a conserved state: e0 = translational(-rotational) thermal energy per
// unit mass (formation, kinetic [and pool] energy taken out), e1 = pool energy per unit mass.
template <class G, int ND>
__device__ __forceinline__ void specific_thermal(const double* q, double& e0, double& e1) {
  constexpr int NS = G::NS;
  double rho = 0.0, m2 = 0.0, et = q[NS + ND];
#pragma unroll
  for (int s = 0; s < NS; ++s) rho += q[s];
#pragma unroll
  for (int d = 0; d < ND; ++d) m2 += q[NS + d] * q[NS + d];
  et -= 0.5 * m2 / rho;
#pragma unroll
  for (int s = 0; s < NS; ++s) et -= q[s] * hf<G>(s);
  e1 = 0.0;
  if (G::NTEMP == 2) {
    et -= q[NS + ND + 1];
    e1 = q[NS + ND + 1] / rho;
  }
  e0 = et / rho;
}

// Is the updated state qn inside the update limit's band around q0 (specific thermal energy
// within a factor 1 + f, pool energy gaining at most f of the old specific energies)?
template <class G, int ND>
__device__ __forceinline__ bool within_limit(const double* q0, const double* qn, double f) {
  double a0, a1, b0, b1;
  specific_thermal<G, ND>(q0, a0, a1);
  if (!(a0 > 0.0)) return true;
  specific_thermal<G, ND>(qn, b0, b1);
  if (!(b0 * (1.0 + f) >= a0 && b0 <= (1.0 + f) * a0)) return false;
  if (G::NTEMP == 2 && !(b1 <= a1 + f * (a0 + a1))) return false;
  return true;
}

// K7: consistency correction (CS-1 mode 1, CS-2 mode 2, coupled mode 0) and update, with the
// optional update limit: the cell's whole increment is scaled by alpha = min(1, ulim rho /
// |d rho|), then alpha is halved (at most 30 times) while the corrected state is non-physical
// or outside the band of within_limit.  alpha = 1 leaves every product exact, so with
// ulim = 0 this is the plain update.
template <class G, int ND>
__global__ void __launch_bounds__(256) k_correct(DevGrid g, int mode, int clip, const double* dq) {
  using A = Aux<G, ND>;
  constexpr int NS = G::NS, NQ = A::NQ;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  const size_t N = g.N;
  double q0[NQ], rho = 0.0;
#pragma unroll
  for (int v = 0; v < NQ; ++v) q0[v] = g.Q[v * N + c];
#pragma unroll
  for (int s = 0; s < NS; ++s) rho += q0[s];
  const double f = g.ulim;
  double alpha = 1.0;
  if (f > 0.0 && fabs(dq[c]) > f * rho) alpha = f * rho / fabs(dq[c]);
  double qn[NQ];
  int nclip = 0;
  bool ok = cell_update<G, ND>(g, mode, clip, dq, c, q0, rho, alpha, qn, nclip);
  if (f > 0.0) {
    for (int it = 0; it < 30 && (!ok || !within_limit<G, ND>(q0, qn, f)); ++it) {
      alpha *= 0.5;
      ok = cell_update<G, ND>(g, mode, clip, dq, c, q0, rho, alpha, qn, nclip);
    }
  }
  if (!ok) {
    set_status(g, ST_NONPHYSICAL, c);
    return;
  }
#pragma unroll
  for (int v = 0; v < NQ; ++v) g.Q[v * N + c] = qn[v];
  if (nclip) atomicAdd(&g.status[2], nclip);
}

// |A(S)| x in CI variables for the eigenvalue splitting A+- = (A +- |A|)/2 (Sec. 2.3): the
// acoustic waves U_n +- c carry alpha+- = (dp +- rho c dU_n) / (2 c^2) along (Y_s, u +- c n,
// H +- U_n c, e_v); every other wave moves with U_n:
//   |A| dq = |S| (|U_n| dq + (|U_n + c| - |U_n|) alpha+ r+ + (|U_n - c| - |U_n|) alpha- r-).
template <class G, int ND>
__device__ __forceinline__ void absjac_ci(const DevGrid& g, int nb, const double* S, const double* x,
                                          double* y) {
  using A = Aux<G, ND>;
  constexpr int NS = G::NS, NF = A::NF;
  const size_t N = g.N;
  const double* W = g.W;
  const double rho = W[A::RHO * N + nb], beta = W[A::BETA * N + nb], c = W[A::C * N + nb];
  double a2 = 0.0;
  for (int d = 0; d < ND; ++d) a2 += S[d] * S[d];
  const double area = sqrt(a2), ia = 1.0 / area;
  double u[ND], n[ND], Un = 0.0, ndm = 0.0, dp = 0.0;
  double first = x[0];
  for (int s = 1; s < NS; ++s) {
    dp += W[(A::PRS + s) * N + nb] * x[NF + s - 1];
    first -= x[NF + s - 1];
  }
  dp += W[(A::PRS + 0) * N + nb] * first;
  for (int d = 0; d < ND; ++d) {
    u[d] = W[(A::U + d) * N + nb];
    n[d] = S[d] * ia;
    Un += u[d] * n[d];
    ndm += n[d] * x[1 + d];
    dp -= beta * u[d] * x[1 + d];
  }
  dp += beta * x[ND + 1];
  if (G::NTEMP == 2) dp += W[A::PREV * N + nb] * x[NF - 1];
  const double dUn = (ndm - Un * x[0]) / rho;
  const double i2c2 = 0.5 / (c * c);
  const double ap = (dp + rho * c * dUn) * i2c2, am = (dp - rho * c * dUn) * i2c2;
  const double l0 = fabs(Un), lp = fabs(Un + c) - l0, lm = fabs(Un - c) - l0;
  const double H = W[A::H * N + nb];
  const double wsum = lp * ap + lm * am;          // coefficient of the (Y_s, e_v) parts
  y[0] = area * (l0 * x[0] + wsum);               // sum of the species rows (sum_s Y_s = 1)
  for (int d = 0; d < ND; ++d)
    y[1 + d] = area * (l0 * x[1 + d] + lp * ap * (u[d] + c * n[d]) + lm * am * (u[d] - c * n[d]));
  y[ND + 1] = area * (l0 * x[ND + 1] + lp * ap * (H + Un * c) + lm * am * (H - Un * c));
  if (G::NTEMP == 2) y[NF - 1] = area * (l0 * x[NF - 1] + wsum * W[A::EV * N + nb]);
  for (int s = 1; s < NS; ++s) y[NF + s - 1] = area * (l0 * x[NF + s - 1] + wsum * W[(A::Y + s) * N + nb]);
}

// ---------------------------------------------------------------------------------------
// Coupled (CI) operator: dense diagonal blocks (V/dtau + sum lambda) I - V dS/dQ_CI with one
// species eliminated through the total density (Sec. 2.2, Sec. 2.3.3; the eliminated species
// is the first of the list, N2, not the electron: see jvp_ci), LU with partial pivoting.
// ---------------------------------------------------------------------------------------
template <int NC>
__device__ __forceinline__ void lu_solve(const double* M, const int* piv, double* b) {
  for (int kk = 0; kk < NC; ++kk) {
    const int p = piv[kk];
    if (p != kk) { const double t = b[kk]; b[kk] = b[p]; b[p] = t; }
  }
  for (int r = 1; r < NC; ++r)
    for (int col = 0; col < r; ++col) b[r] -= M[r * NC + col] * b[col];
  for (int r = NC - 1; r >= 0; --r) {
    for (int col = r + 1; col < NC; ++col) b[r] -= M[r * NC + col] * b[col];
    b[r] /= M[r * NC + r];
  }
}

template <class G, int ND>
__global__ void __launch_bounds__(64) k_ci_block(DevGrid g) {
  using A = Aux<G, ND>;
  constexpr int NS = G::NS, NF = A::NF, NC = A::NCI, NQ = A::NQ;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  const size_t N = g.N;
  double* M = g.DLU + (size_t)c * NC * NC;
  const double diag = g.Vdt[c] + M[0];
  for (int e = 0; e < NC * NC; ++e) M[e] = 0.0;
  for (int e = 0; e < NC; ++e) M[e * NC + e] = diag;
  const double V = g.V[c];
  if (G::NTEMP == 2) M[(NF - 1) * NC + NF - 1] += V * g.W[A::RELAX * N + c];
  if (g.cisplit) {
    // eigenvalue splitting: + sum_d |A_c(S_d)|, S_d the mean of the cell's two d-faces
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    for (int d = 0; d < ND; ++d) {
      const double* Sm = face_vec(g, d, i, j, k, -1);
      const double* Sp = face_vec(g, d, i, j, k, +1);
      double Sb[ND];
      for (int q = 0; q < ND; ++q) Sb[q] = 0.5 * (Sm[q] + Sp[q]);
      for (int col = 0; col < NC; ++col) {
        double e[NC], a[NC];
        for (int q = 0; q < NC; ++q) e[q] = q == col ? 1.0 : 0.0;
        absjac_ci<G, ND>(g, c, Sb, e, a);
        for (int r = 0; r < NC; ++r) M[r * NC + col] += a[r];
      }
    }
  }
  if (g.react && G::NR > 0) {
    double q[NQ];
    for (int v = 0; v < NQ; ++v) q[v] = g.Q[v * N + c];
    Prim<G, ND> w;
    if (primitive<G, ND>(q, g.W[A::T * N + c], g.W[A::TV * N + c], w) != ST_OK) {
      set_status(g, ST_NONPHYSICAL, c);
      return;
    }
    double om[NS], jd[NS], J[NS * NS], wT[NS], wTv[NS], emT[NS], emTv[NS], rT[NS], rV[NS];
    vib_exp<G>(1.0 / w.T, emT);
    if (G::NTEMP == 2) vib_exp<G>(1.0 / w.Tv, emTv);
    else for (int s = 0; s < NS; ++s) emTv[s] = emT[s];
    vib_rcp<G>(emT, rT);
    vib_rcp<G>(emTv, rV);
    chemistry<G, true>(w.rhos, w.T, w.Tv, emT, emTv, rT, rV, om, jd, J, wT, wTv);
    // temperature derivatives with respect to the full conserved variables
    double dT[NQ], dTv[NQ];
    double ke = 0.0;
    for (int d = 0; d < ND; ++d) ke += 0.5 * w.u[d] * w.u[d];
    for (int s = 0; s < NS; ++s) {
      double ev = 0.0, cvv;
      if (G::NTEMP == 1) vib<G>(s, w.T, ev, cvv);
      else ev = (G::sp(s).kind == ELECTRON) ? 1.5 * Rs<G>(s) * w.Tv : w.eve[s];
      dT_drho<G, ND>(w, s, ev, dT[s], dTv[s]);
    }
    const double rc = w.rho * (G::NTEMP == 1 ? w.cv : w.cvtr);
    for (int d = 0; d < ND; ++d) dT[NS + d] = -w.u[d] / rc;
    dT[NS + ND] = 1.0 / rc;
    if (G::NTEMP == 1) {
      for (int v = NS; v < NQ; ++v) dTv[v] = dT[v];
    } else {
      for (int d = 0; d < ND; ++d) dTv[NS + d] = 0.0;
      dTv[NS + ND] = 0.0;
      dT[NQ - 1] = -1.0 / rc;
      dTv[NQ - 1] = (w.cvve > 0.0) ? 1.0 / (w.rho * w.cvve) : 0.0;
    }
    // rows: species s = 1..NS-1; the first species (N2) is the eliminated one,
    // rho_1st = rho - sum_{r>0} rho_r, so column rho is d/d rho_1st and column rho_r is
    // d/d rho_r - d/d rho_1st
    for (int s = 1; s < NS; ++s) {
      auto jq = [&](int kcol) {   // full-layout row of d omega_s / dQ
        double v = wT[s] * dT[kcol] + wTv[s] * dTv[kcol];
        if (kcol < NS) v += J[s * NS + kcol];
        return v;
      };
      const double first = jq(0);
      double* row = M + (NF + s - 1) * NC;
      row[0] -= V * first;
      for (int kk = 1; kk < NF; ++kk) row[kk] -= V * jq(NS + kk - 1);
      for (int r = 1; r < NS; ++r) row[NF + r - 1] -= V * (jq(r) - first);
    }
  }
  // LU with partial pivoting (ties: lowest row), in place
  int* piv = g.piv + (size_t)c * NC;
  for (int kk = 0; kk < NC; ++kk) {
    int p = kk;
    double best = fabs(M[kk * NC + kk]);
    for (int r = kk + 1; r < NC; ++r) {
      const double v = fabs(M[r * NC + kk]);
      if (v > best) { best = v; p = r; }
    }
    piv[kk] = p;
    if (best == 0.0) {
      set_status(g, ST_NONPHYSICAL, c);
      return;
    }
    if (p != kk)
      for (int col = 0; col < NC; ++col) {
        const double t = M[kk * NC + col];
        M[kk * NC + col] = M[p * NC + col];
        M[p * NC + col] = t;
      }
    const double inv = 1.0 / M[kk * NC + kk];
    for (int r = kk + 1; r < NC; ++r) {
      const double l = M[r * NC + kk] * inv;
      M[r * NC + kk] = l;
      for (int col = kk + 1; col < NC; ++col) M[r * NC + col] -= l * M[kk * NC + col];
    }
  }
  // the explicit inverse, column by column from the factors: the cluster sweep multiplies by
  // it (independent dot products) instead of running the two dependent substitutions per step
  if (g.DINV) {
    double* Dv = g.DINV + (size_t)c * NC * NC;
    for (int col = 0; col < NC; ++col) {
      double e[NC];
      for (int r = 0; r < NC; ++r) e[r] = r == col ? 1.0 : 0.0;
      lu_solve<NC>(M, g.piv + (size_t)c * NC, e);
      for (int r = 0; r < NC; ++r) Dv[r * NC + col] = e[r];
    }
  }
}


// coupled Jacobian-vector product in CI variables (rho, m, rhoE, [rho e_v], rho_2..rho_ns);
// the first species is eliminated: rho_1st = rho - sum of the others
template <class G, int ND>
__device__ __forceinline__ void jvp_ci(const DevGrid& g, int nb, const double* S, const double* x,
                                       double* y) {
  using A = Aux<G, ND>;
  constexpr int NS = G::NS, NF = A::NF;
  const size_t N = g.N;
  const double* W = g.W;
  const double rho = W[A::RHO * N + nb], beta = W[A::BETA * N + nb];
  double u[ND], U = 0.0, Sdm = 0.0, dp = 0.0;
  double first = x[0];
  for (int s = 1; s < NS; ++s) {
    dp += W[(A::PRS + s) * N + nb] * x[NF + s - 1];
    first -= x[NF + s - 1];
  }
  dp += W[(A::PRS + 0) * N + nb] * first;
  for (int d = 0; d < ND; ++d) {
    u[d] = W[(A::U + d) * N + nb];
    U += u[d] * S[d];
    Sdm += S[d] * x[1 + d];
    dp -= beta * u[d] * x[1 + d];
  }
  dp += beta * x[ND + 1];
  if (G::NTEMP == 2) dp += W[A::PREV * N + nb] * x[NF - 1];
  const double dU = (Sdm - U * x[0]) / rho;
  y[0] = Sdm;
  for (int d = 0; d < ND; ++d) y[1 + d] = x[1 + d] * U + rho * u[d] * dU + dp * S[d];
  const double rhoE = g.Q[(NS + ND) * N + nb], p = W[A::P * N + nb];
  y[ND + 1] = (x[ND + 1] + dp) * U + (rhoE + p) * dU;
  if (G::NTEMP == 2) y[NF - 1] = x[NF - 1] * U + g.Q[(A::NQ - 1) * N + nb] * dU;
  for (int s = 1; s < NS; ++s) y[NF + s - 1] = x[NF + s - 1] * U + rho * W[(A::Y + s) * N + nb] * dU;
}

template <class G, int ND, bool FWD>
__global__ void __launch_bounds__(64) k_sweep_coupled(DevGrid g, int h, int off, int cnt) {
  using A = Aux<G, ND>;
  constexpr int NS = G::NS, NF = A::NF, NC = A::NCI;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (t >= cnt || !hyperplane_cell<G, ND>(g, h, t + off, i, j, k)) return;
  const int c = cell_of(g, i, j, k);
  const size_t N = g.N;
  double acc[NC];
  if (FWD) {
    double rr = 0.0;
    for (int s = 0; s < NS; ++s) rr += g.R[s * N + c];
    acc[0] = -rr;
    for (int q = 1; q < NF; ++q) acc[q] = -g.R[(NS + q - 1) * N + c];
    for (int s = 1; s < NS; ++s) acc[NF + s - 1] = -g.R[s * N + c];
  } else {
    for (int q = 0; q < NC; ++q) acc[q] = 0.0;
  }
  const double* X = FWD ? g.dQcs : g.dQc;
  for (int d = 0; d < ND; ++d)
    for (int s = -1; s <= 1; s += 2) {
      bool lower;
      const int nb = neighbour(g, i, j, k, d, s, lower);
      if (nb < 0 || lower != FWD) continue;
      const double* Sf = face_vec(g, d, i, j, k, s);
      double xn[NC], ax[NC];
      for (int q = 0; q < NC; ++q) xn[q] = X[q * N + nb];
      jvp_ci<G, ND>(g, nb, Sf, xn, ax);
      // spectral splitting: lamCI = the coupled radius; eigenvalue splitting: lamCI = 2
      // lambda_vis and |A_nb(S_f)| x is added
      const double l = g.lamCI[d * N + nb];
      if (g.cisplit) {
        double bx[NC];
        absjac_ci<G, ND>(g, nb, Sf, xn, bx);
        for (int q = 0; q < NC; ++q) ax[q] += (s < 0 ? bx[q] : -bx[q]);
      }
      for (int q = 0; q < NC; ++q) {
        if (s < 0) acc[q] += 0.5 * (ax[q] + l * xn[q]);
        else acc[q] -= 0.5 * (ax[q] - l * xn[q]);
      }
    }
  lu_solve<NC>(g.DLU + (size_t)c * NC * NC, g.piv + (size_t)c * NC, acc);
  double* Y = FWD ? g.dQcs : g.dQc;
  for (int q = 0; q < NC; ++q) Y[q * N + c] = FWD ? acc[q] : g.dQcs[q * N + c] + acc[q];
}

// ---------------------------------------------------------------------------------------
// Coupled (CI) sweeps of a 2D grid in one thread-block-cluster launch: the same arithmetic as
// k_sweep_coupled, with the hyperplane loop inside the kernel (as in k_split_cluster): CTA r
// of the cluster owns rows [r R, (r+1) R), one lane per row; the row's previous cell (and the
// first one, for a periodic i) stay in registers, the neighbouring row's result comes from
// shared memory or, across a CTA boundary, distributed shared memory, and one cluster barrier
// separates consecutive hyperplanes.  Each cell applies the coupled Jacobian of its
// neighbours matrix-free and solves with its LU factors.
// ---------------------------------------------------------------------------------------
// one neighbour's coupling (spectral or eigenvalue splitting), as in k_sweep_coupled
template <class G>
__device__ __forceinline__ void ci_contrib(const DevGrid& g, int nb, int d, const double* Sf,
                                           const double* xn, int side, double* acc) {
  constexpr int NC = Aux<G, 2>::NCI;
  double ax[NC];
  jvp_ci<G, 2>(g, nb, Sf, xn, ax);
  if (g.cisplit) {
    double bx[NC];
    absjac_ci<G, 2>(g, nb, Sf, xn, bx);
    for (int q = 0; q < NC; ++q) ax[q] += (side < 0 ? bx[q] : -bx[q]);
  }
  const double l = g.lamCI[d * (size_t)g.N + nb];
  for (int q = 0; q < NC; ++q) {
    if (side < 0) acc[q] += 0.5 * (ax[q] + l * xn[q]);
    else acc[q] -= 0.5 * (ax[q] - l * xn[q]);
  }
}

template <class G>
__global__ void __launch_bounds__(32) k_ci_cluster(DevGrid g, int R) {
  using A = Aux<G, 2>;
  constexpr int NS = G::NS, NF = A::NF, NC = A::NCI;
  __shared__ double xv[2][kClusterRows][NC];
  const size_t N = g.N;
  const unsigned rank = cluster_ctarank();
  const int t = cluster_row(R);
  const int j = rank * R + t;
  const bool row = t >= 0 && j < g.nj;
  const bool per = g.bc[0] == BC_PERIODIC;
  const int ni = g.ni, nj = g.nj, H = ni + nj - 2;
  for (int pass = 0; pass < 2; ++pass) {
    const bool fwd = pass == 0;
    double prevx[NC], firstx[NC];
    int prevc = 0, firstc = 0;
    for (int q = 0; q <= H; ++q) {
      const int i = (fwd ? q : H - q) - j;
      const bool act = row && i >= 0 && i < ni;
      double acc[NC];
      int c = 0;
      if (act) {
        c = i + ni * j;
        if (fwd) {
          double rr = 0.0;
          for (int s = 0; s < NS; ++s) rr += g.R[s * N + c];
          acc[0] = -rr;
          for (int v = 1; v < NF; ++v) acc[v] = -g.R[(NS + v - 1) * N + c];
          for (int s = 1; s < NS; ++s) acc[NF + s - 1] = -g.R[s * N + c];
        } else {
          for (int v = 0; v < NC; ++v) acc[v] = 0.0;
        }
        // the row's own earlier cells: no other CTA involved, before the barrier
        if (fwd) {
          if (i > 0) ci_contrib<G>(g, prevc, 0, face_vec(g, 0, i, j, 0, -1), prevx, -1, acc);
          if (per && i == ni - 1) ci_contrib<G>(g, firstc, 0, face_vec(g, 0, i, j, 0, +1), firstx, +1, acc);
        } else {
          if (per && i == 0) ci_contrib<G>(g, firstc, 0, face_vec(g, 0, i, j, 0, -1), firstx, -1, acc);
          if (i < ni - 1) ci_contrib<G>(g, prevc, 0, face_vec(g, 0, i, j, 0, +1), prevx, +1, acc);
        }
      }
      if (q > 0) cluster_wait();
      if (act) {
        const int jj = fwd ? j - 1 : j + 1;
        if (jj >= 0 && jj < nj) {
          const int par = (q - 1) & 1;
          const double* src;
          if (fwd) src = (t > 0) ? xv[par][t - 1] : dsmem(&xv[par][R - 1][0], rank - 1);
          else src = (t < R - 1) ? xv[par][t + 1] : dsmem(&xv[par][0][0], rank + 1);
          double xn[NC];
          for (int v = 0; v < NC; ++v) xn[v] = src[v];
          ci_contrib<G>(g, i + ni * jj, 1, face_vec(g, 1, i, j, 0, fwd ? -1 : +1), xn, fwd ? -1 : +1, acc);
        }
        {
          const double* Dv = g.DINV + (size_t)c * NC * NC;
          double y[NC];
#pragma unroll
          for (int r = 0; r < NC; ++r) {
            double a = 0.0;
#pragma unroll
            for (int k = 0; k < NC; ++k) a += Dv[r * NC + k] * acc[k];
            y[r] = a;
          }
#pragma unroll
          for (int r = 0; r < NC; ++r) acc[r] = y[r];
        }
        double* out = fwd ? g.dQcs : g.dQc;
        for (int v = 0; v < NC; ++v) {
          const double x = fwd ? acc[v] : g.dQcs[v * N + c] + acc[v];
          out[v * N + c] = x;
          xv[q & 1][t][v] = x;
          prevx[v] = x;
        }
        prevc = c;
        if (i == (fwd ? 0 : ni - 1)) {
          for (int v = 0; v < NC; ++v) firstx[v] = prevx[v];
          firstc = c;
        }
      }
      cluster_arrive();
    }
    cluster_wait();
  }
}

// ---------------------------------------------------------------------------------------
// Coupled (CI) sweeps of a 2D grid over assembled neighbour blocks.  k_ci_mat forms, for every
// cell, the coupling blocks of its four neighbours in CI variables,
// (+-1/2)(A_nb(S) [+- |A_nb(S)|] +- lambda_nb I), column by column from jvp_ci / absjac_ci (the
// products k_ci_cluster applies one lane per row), and the cell's right-hand side.
// k_ci_mat_sweep then runs both sweeps in one cluster launch with kCISlots threads per row, one
// per CI variable: per hyperplane step a thread takes one row of each neighbour block (dot
// products of length NC) and, once the row's threads have exchanged their right-hand sides
// through shared memory, one row of the diagonal block's inverse.  The FP64 work of a cell is
// spread over NC threads (and the four SM sub-partitions) instead of one lane.
// Record of cell c (doubles): blocks [fwd i][fwd j][bwd i][bwd j], NC rows of NP (NC rounded up
// to even), then the forward right-hand side (NP); per row j after the N cell records: the
// periodic-i wrap blocks (forward, backward).
// ---------------------------------------------------------------------------------------
constexpr int kCISlots = 16;
constexpr int kCIRows = 16;     // rows per CTA at most (kCISlots x kCIRows threads)

template <class G>
struct CIRec {
  static constexpr int NC = Aux<G, 2>::NCI;
  static constexpr int NP = (NC + 1) / 2 * 2;
  static constexpr int BLK = NC * NP;
  static constexpr int CELL = 4 * BLK + NP;
  static constexpr int ROW = 2 * BLK;
  static_assert(NC <= kCISlots, "one thread per CI variable");
};

// the block of neighbour nb across face Sf on side `side` (direction d for its radius)
template <class G>
__device__ __forceinline__ void ci_block_of(const DevGrid& g, int nb, int d, const double* Sf, int side,
                                            double* out) {
  constexpr int NC = CIRec<G>::NC, NP = CIRec<G>::NP;
  const double l = g.lamCI[d * (size_t)g.N + nb];
#pragma unroll 1
  for (int k = 0; k < NC; ++k) {
    double e[NC], ax[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) e[q] = q == k ? 1.0 : 0.0;
    jvp_ci<G, 2>(g, nb, Sf, e, ax);
    if (g.cisplit) {
      double bx[NC];
      absjac_ci<G, 2>(g, nb, Sf, e, bx);
#pragma unroll
      for (int q = 0; q < NC; ++q) ax[q] += (side < 0 ? bx[q] : -bx[q]);
    }
#pragma unroll
    for (int v = 0; v < NC; ++v) {
      const double lv = v == k ? l : 0.0;
      out[v * NP + k] = side < 0 ? 0.5 * (ax[v] + lv) : -0.5 * (ax[v] - lv);
    }
  }
#pragma unroll
  for (int v = 0; v < NC; ++v)
#pragma unroll
    for (int k = NC; k < NP; ++k) out[v * NP + k] = 0.0;
}

template <class G>
__global__ void __launch_bounds__(64) k_ci_mat(DevGrid g) {
  using M = CIRec<G>;
  using A = Aux<G, 2>;
  constexpr int NS = G::NS, NF = A::NF, NC = M::NC, NP = M::NP, BLK = M::BLK;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  const size_t N = g.N;
  const int ni = g.ni, nj = g.nj, i = c % ni, j = c / ni;
  double* rec = g.CIM + (size_t)c * M::CELL;
  // a face on the grid's boundary couples nothing: its block is zero
  if (i == 0 || j == 0 || i == ni - 1 || j == nj - 1) {
    for (int e = 0; e < 4 * BLK; ++e) rec[e] = 0.0;
  }
  if (i > 0) ci_block_of<G>(g, c - 1, 0, face_vec(g, 0, i, j, 0, -1), -1, rec);
  if (j > 0) ci_block_of<G>(g, c - ni, 1, face_vec(g, 1, i, j, 0, -1), -1, rec + BLK);
  if (i < ni - 1) ci_block_of<G>(g, c + 1, 0, face_vec(g, 0, i, j, 0, +1), +1, rec + 2 * BLK);
  if (j < nj - 1) ci_block_of<G>(g, c + ni, 1, face_vec(g, 1, i, j, 0, +1), +1, rec + 3 * BLK);
  // forward right-hand side in CI variables: -(sum_s R_s, R_m, R_E[, R_ev], R_2 .. R_ns)
  double* rhs = rec + 4 * BLK;
  double rr = 0.0;
  for (int s = 0; s < NS; ++s) rr += g.R[s * N + c];
  rhs[0] = -rr;
  for (int v = 1; v < NF; ++v) rhs[v] = -g.R[(NS + v - 1) * N + c];
  for (int s = 1; s < NS; ++s) rhs[NF + s - 1] = -g.R[s * N + c];
  for (int v = NC; v < NP; ++v) rhs[v] = 0.0;
  if (g.bc[0] == BC_PERIODIC) {
    double* pr = g.CIM + N * M::CELL + (size_t)j * M::ROW;
    // forward: (0, j) precedes (ni-1, j) across the cut, on its + side; backward: (ni-1, j)
    // precedes (0, j), on its - side
    if (i == ni - 1) ci_block_of<G>(g, ni * j, 0, face_vec(g, 0, i, j, 0, +1), +1, pr);
    if (i == 0) ci_block_of<G>(g, ni - 1 + ni * j, 0, face_vec(g, 0, i, j, 0, -1), -1, pr + BLK);
  }
}

// inputs of one thread's cell at step q (raw loads, one step ahead; the inverse's row is loaded
// at the start of its own step, ahead of the cluster barrier)
template <class G>
struct CIStep {
  double bi[CIRec<G>::NP], bj[CIRec<G>::NP], base;
  int c, i;
  bool act;
};

template <class G>
__device__ __forceinline__ void ci_step_load(const DevGrid& g, int q, int j, bool on, bool fwd, int v,
                                             CIStep<G>& m) {
  using M = CIRec<G>;
  constexpr int NP = M::NP, BLK = M::BLK;
  const int ni = g.ni, H = ni + g.nj - 2;
  const int i = (fwd ? q : H - q) - j;
  m.act = on && q <= H && i >= 0 && i < ni;
  m.i = i;
  if (!m.act) return;
  const int c = i + ni * j;
  m.c = c;
  const double* rec = g.CIM + (size_t)c * M::CELL;
  const double2* ri = reinterpret_cast<const double2*>(rec + (fwd ? 0 : 2 * BLK) + v * NP);
  const double2* rj = reinterpret_cast<const double2*>(rec + (fwd ? BLK : 3 * BLK) + v * NP);
#pragma unroll
  for (int k = 0; k < NP / 2; ++k) {
    const double2 a = ri[k], b = rj[k];
    m.bi[2 * k] = a.x;
    m.bi[2 * k + 1] = a.y;
    m.bj[2 * k] = b.x;
    m.bj[2 * k + 1] = b.y;
  }
  m.base = fwd ? rec[4 * BLK + v] : g.dQcs[(size_t)v * g.N + c];
}

template <class G>
__global__ void __launch_bounds__(kCISlots * kCIRows) k_ci_mat_sweep(DevGrid g, int R) {
  using M = CIRec<G>;
  constexpr int NC = M::NC, BLK = M::BLK, NP = M::NP;
  __shared__ __align__(16) double xv[2][kCIRows][kCISlots];   // results of the last two steps
  __shared__ __align__(16) double ac[kCIRows][kCISlots];      // a row's right-hand sides
  __shared__ __align__(16) double xf[kCIRows][kCISlots];      // a row's first result of the pass
  const size_t N = g.N;
  const unsigned rank = cluster_ctarank();
  const int t = threadIdx.x / kCISlots, v = threadIdx.x % kCISlots;
  const int j = rank * R + t;
  const int ni = g.ni, nj = g.nj, H = ni + nj - 2;
  const bool per = g.bc[0] == BC_PERIODIC;
  const bool on = t < R && j < nj && v < NC;
  for (int pass = 0; pass < 2; ++pass) {
    const bool fwd = pass == 0;
    double* out = fwd ? g.dQcs : g.dQc;
    const bool hasj = fwd ? j > 0 : j < nj - 1;
    xf[t][v] = 0.0;
    __syncwarp();
    CIStep<G> cur, nxt;
    ci_step_load<G>(g, 0, j, on, fwd, v, cur);
    for (int q = 0; q <= H; ++q) {
      ci_step_load<G>(g, q + 1, j, on, fwd, v, nxt);     // prefetch the next step
      // the row's own previous cell (and the periodic wrap): no other row involved, coupled
      // while the cluster barrier is pending
      double acc = 0.0, dinv[NC];
      if (cur.act) {
        const double* Dv = g.DINV + (size_t)cur.c * NC * NC + v * NC;
#pragma unroll
        for (int k = 0; k < NC; ++k) dinv[k] = Dv[k];
        const int i = cur.i;
        if (fwd) acc = cur.base;
        if (fwd ? i > 0 : i < ni - 1) {
          const double* xp = xv[(q - 1) & 1][t];
#pragma unroll
          for (int k = 0; k < NC; ++k) acc += cur.bi[k] * xp[k];
        }
        if (per && i == (fwd ? ni - 1 : 0)) {
          const double* pw = g.CIM + N * M::CELL + (size_t)j * M::ROW + (fwd ? 0 : BLK) + v * NP;
#pragma unroll
          for (int k = 0; k < NC; ++k) acc += pw[k] * xf[t][k];
        }
      }
      if (q > 0) cluster_wait();
      if (cur.act) {
        if (hasj) {
          const int par = (q - 1) & 1;
          const double* src;
          if (fwd) src = (t > 0) ? xv[par][t - 1] : dsmem(&xv[par][R - 1][0], rank - 1);
          else src = (t < R - 1) ? xv[par][t + 1] : dsmem(&xv[par][0][0], rank + 1);
#pragma unroll
          for (int k = 0; k < NC; ++k) acc += cur.bj[k] * src[k];
        }
        ac[t][v] = acc;
      }
      __syncwarp();                    // a row's kCISlots threads share one warp
      if (cur.act) {
        double y = 0.0;
#pragma unroll
        for (int k = 0; k < NC; ++k) y += dinv[k] * ac[t][k];
        const double x = fwd ? y : cur.base + y;
        out[(size_t)v * N + cur.c] = x;
        xv[q & 1][t][v] = x;
        if (cur.i == (fwd ? 0 : ni - 1)) xf[t][v] = x;
      }
      __syncwarp();
      cluster_arrive();
      cur = nxt;
    }
    cluster_wait();
  }
}

// ---------------------------------------------------------------------------------------
// Freestream: density from p, T, Y; velocity = Mach * frozen sound speed; conserved state and
// auxiliary record (one thread).
// ---------------------------------------------------------------------------------------
template <class G, int ND>
__global__ void k_freestream(DevGrid g, const double* in, double* fsQ) {
  // in: [T, Tv, p, mach, dir[3], Y[NS]]
  using A = Aux<G, ND>;
  constexpr int NS = G::NS, NQ = A::NQ;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double T = in[0], Tv = (G::NTEMP == 2) ? in[1] : in[0], p = in[2], mach = in[3];
  const double* Y = in + 7;
  double Rm = 0.0;
  for (int s = 0; s < NS; ++s)
    Rm += Y[s] * Rs<G>(s) * ((G::NTEMP == 2 && G::sp(s).kind == ELECTRON) ? Tv / T : 1.0);
  const double rho = p / (Rm * T);
  double q[NQ];
  double e = 0.0, ev = 0.0;
  for (int s = 0; s < NS; ++s) {
    q[s] = rho * Y[s];
    double evs, cvv;
    if (G::sp(s).kind == ELECTRON && G::NTEMP == 2) evs = 1.5 * Rs<G>(s) * Tv;
    else vib<G>(s, G::NTEMP == 2 ? Tv : T, evs, cvv);
    e += q[s] * (cvtr<G>(s) * T + evs + hf<G>(s));
    ev += q[s] * evs;
  }
  for (int d = 0; d < ND; ++d) q[NS + d] = 0.0;
  q[NS + ND] = e;
  if (G::NTEMP == 2) q[NQ - 1] = ev;
  Prim<G, ND> w;
  if (primitive<G, ND>(q, T, Tv, w) != ST_OK) { set_status(g, ST_NONPHYSICAL, -1); return; }
  double dn = 0.0;
  for (int d = 0; d < ND; ++d) dn += in[4 + d] * in[4 + d];
  dn = sqrt(dn);
  double ke = 0.0;
  for (int d = 0; d < ND; ++d) {
    const double u = mach * w.c * in[4 + d] / dn;
    q[NS + d] = rho * u;
    ke += 0.5 * u * u;
  }
  q[NS + ND] = e + rho * ke;
  if (primitive<G, ND>(q, T, Tv, w) != ST_OK) { set_status(g, ST_NONPHYSICAL, -1); return; }
  for (int v = 0; v < NQ; ++v) fsQ[v] = q[v];
  DevGrid one = g;
  one.W = g.fsW;
  one.N = 1;
  store_prim<G, ND>(one, 0, w);
}

template <class G, int ND>
__global__ void __launch_bounds__(256) k_fill(DevGrid g, const double* fsQ) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  for (int v = 0; v < Aux<G, ND>::NQ; ++v) g.Q[(size_t)v * g.N + c] = fsQ[v];
}


// ---------------------------------------------------------------------------------------
// Chemistry surrogate coupling.  Raw features of a cell: log10 rho, T / 1e4, Tv / 1e4 and the
// mass fractions Y_1..Y_11 (zero beyond the model's species); raw targets: asinh(omega_s) and
// asinh(d omega_s / d rho_s) (SI units; zero beyond the model's species).  The network works
// on standardised values, x = (f - mean) / std; norm = [mean_f[14], std_f[14], mean_t[22],
// std_t[22]].
// ---------------------------------------------------------------------------------------
constexpr int kSurrIn = 14, kSurrOut = 22, kSurrNS = 11;

template <class G, int ND>
__device__ __forceinline__ void surr_raw_features(const DevGrid& g, int c, float* f) {
  using A = Aux<G, ND>;
  const size_t N = g.N;
  // logarithms throughout: the rates are Arrhenius in T and mass-action in the densities, and
  // trace species span many decades (1e-10 floors the mass fractions).  The network's inputs
  // are FP32, so the logarithms are taken in FP32 (an FP64 logarithm per input cost more than
  // the network itself)
  f[0] = log10f((float)g.W[A::RHO * N + c]);
  f[1] = log10f((float)g.W[A::T * N + c]);
  f[2] = log10f((float)g.W[A::TV * N + c]);
#pragma unroll
  for (int s = 0; s < kSurrNS; ++s)
    f[3 + s] = s < G::NS ? log10f(fmaxf((float)g.W[(A::Y + s) * N + c], 0.f) + 1e-10f) : -10.f;
}

// raw features [N][14] and raw targets [N][22] of every cell (from the auxiliary fields of the
// last primitive evaluation, exact chemistry)
template <class G, int ND>
__global__ void __launch_bounds__(128) k_surr_sample(DevGrid g, float* X, float* T) {
  using A = Aux<G, ND>;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  const size_t N = g.N;
  float f[kSurrIn];
  surr_raw_features<G, ND>(g, c, f);
#pragma unroll
  for (int k = 0; k < kSurrIn; ++k) X[(size_t)c * kSurrIn + k] = f[k];
#pragma unroll
  for (int s = 0; s < kSurrNS; ++s) {
    T[(size_t)c * kSurrOut + s] = s < G::NS ? (float)asinh(g.W[(A::OM + s) * N + c]) : 0.f;
    // the part of d omega_s / d rho_s the operator uses: its stiffness max(0, -d omega / d rho)
    T[(size_t)c * kSurrOut + kSurrNS + s] =
        s < G::NS ? (float)asinh(fmax(0.0, -g.W[(A::DOM + s) * N + c])) : 0.f;
  }
}

// standardised network inputs [N][14]
template <class G, int ND>
__global__ void __launch_bounds__(128) k_surr_features(DevGrid g, float* X, const double* norm) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  float f[kSurrIn];
  surr_raw_features<G, ND>(g, c, f);
  // standardised, and held to the range the training data spans (|x| <= 8) so that a state
  // unlike any the network saw cannot drive it far outside
#pragma unroll
  for (int k = 0; k < kSurrIn; ++k)
    X[(size_t)c * kSurrIn + k] = (float)fmin(fmax((f[k] - norm[k]) / norm[kSurrIn + k], -8.0), 8.0);
}

// network outputs [N][22] -> the species Jacobian diagonal d omega_s / d rho_s of the operator
template <class G, int ND>
__global__ void __launch_bounds__(128) k_surr_decode(DevGrid g, const float* Y, const double* norm) {
  using A = Aux<G, ND>;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  const size_t N = g.N;
  const double* mt = norm + 2 * kSurrIn;
  const double* st = mt + kSurrOut;
#pragma unroll
  for (int s = 0; s < G::NS; ++s) {
    const int o = kSurrNS + s;
    // de-standardised stiffness asinh(max(0, -d omega / d rho)), held to the span of the
    // training targets (mean +- 8 standard deviations, and >= 0); a non-finite output maps to
    // the upper bound, which only adds to the operator's diagonal
    // (FP32 arithmetic: the network's output carries FP32 / bf16 precision)
    const float y = Y[(size_t)c * kSurrOut + o] * (float)st[o] + (float)mt[o];
    const float hi = (float)(mt[o] + 8.0 * st[o]);
    const float t = y == y ? fminf(fmaxf(y, fmaxf(0.f, (float)(mt[o] - 8.0 * st[o]))), hi) : hi;
    g.W[(A::DOM + s) * N + c] = -(double)sinhf(t);
  }
}

}  // namespace cs
