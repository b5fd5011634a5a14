// Host-side launch sequences for one gas model and dimension.  Each instantiation lives in
// its own translation unit (launch_<model>.cu) so the three models compile in parallel.
#pragma once
#include <cstring>
#include <type_traits>

#include "kernels.cuh"

namespace cs {

struct Launcher {
  virtual ~Launcher() {}
  int ns, ntemp, nq, nF, nci, ng, naux, nd;
  virtual cudaError_t init_constants() = 0;
  virtual void freestream(const DevGrid& g, cudaStream_t st, const double* in, double* fsQ) = 0;
  virtual void fill(const DevGrid& g, cudaStream_t st, const double* fsQ) = 0;
  // residual: primitives + gradients + face fluxes + assembly + norms (out[3] on device)
  void residual(const DevGrid& g, cudaStream_t st, int stag, double* out) {
    primitive(g, st);
    gradient(g, st);
    flux(g, st);
    assemble(g, st, stag, out);
  }
  // primitive() = primitive_state() (temperature solves, primitives, transport) + chem()
  // (chemistry, its Jacobian diagonal, vibrational relaxation)
  void primitive(const DevGrid& g, cudaStream_t st) {
    primitive_state(g, st);
    chem(g, st);
  }
  virtual void primitive_state(const DevGrid& g, cudaStream_t st) = 0;
  virtual void chem(const DevGrid& g, cudaStream_t st) = 0;
  virtual void gradient(const DevGrid& g, cudaStream_t st) = 0;
  virtual void flux(const DevGrid& g, cudaStream_t st) = 0;
  virtual void assemble(const DevGrid& g, cudaStream_t st, int stag, double* out) = 0;
  virtual void spectral(const DevGrid& g, cudaStream_t st) = 0;
  // both sweeps; returns launches (the cluster path does both in one launch when available)
  // mixed = true: the sweeps compute in FP32 (from FP64 inputs, into FP64 increments)
  int sweep_split(const DevGrid& g, cudaStream_t st, bool mixed = false) {
    const int n = use_cluster ? sweep_split_cluster(g, st, mixed) : 0;
    if (n) return n;
    return sweep_split_dir(g, st, true, mixed) + sweep_split_dir(g, st, false, mixed);
  }
  virtual int sweep_split_cluster(const DevGrid& g, cudaStream_t st, bool mixed = false) = 0;
  bool use_cluster = true;
  int cluster_kind = 0;    // 0: by precision, 1: direct-load cluster kernel, 2: wavefront records,
                           // 3: one CTA per component (FP32), 4: assembled couplings exchanged
                           // point to point where the ring fits (FP64 or FP32), 5: the FP64
                           // assembled couplings with a cluster barrier
  int force_C = 0;         // CTAs per cluster chosen by the batch tuner (0: largest that fits)
  int cluster_warps = 2;   // warps per CTA of the direct-load cluster kernel (batches: 1)
  bool sweep_split_cluster_ok = false;   // set by the last sweep_split_cluster call
  // kernel of the last split sweep, numbered as the "cluster_sweep" option (0 one launch per
  // hyperplane, 1 direct loads, 2 wavefront records, 4 one CTA per component, 5 assembled
  // couplings point to point, 6 assembled couplings with a cluster barrier; -1 none yet) and
  // its CTAs per cluster
  int last_sweep = -1, last_sweep_C = 0;
  // bit C of the result is set when the cluster sweep of `kind` (1 direct, 2 wavefront
  // records) can run with C CTAs per component on this grid and device
  virtual int cluster_sizes(const DevGrid& g, int kind, bool mixed) = 0;
  // does the FP32 one-CTA-per-component sweep apply to this grid?
  virtual bool block_available(const DevGrid& g) = 0;
  // run the cluster-size probes of the current choice (host-side calls that must not happen
  // inside a stream capture)
  virtual void prepare(const DevGrid& g, bool mixed) = 0;
  virtual int sweep_split_dir(const DevGrid& g, cudaStream_t st, bool fwd, bool mixed = false) = 0;
  // doubles of DevGrid::SMC, the coupling records of the 2D split sweep (0: not used)
  virtual size_t mat_doubles(const DevGrid& g) const = 0;
  // does a split sweep of this precision use the records on this grid and device?
  virtual bool mat_usable(const DevGrid& g, bool mixed) = 0;
  virtual void ci_block(const DevGrid& g, cudaStream_t st) = 0;
  void sweep_coupled(const DevGrid& g, cudaStream_t st) {
    if (use_cluster && sweep_coupled_cluster(g, st)) return;
    sweep_coupled_dir(g, st, true);
    sweep_coupled_dir(g, st, false);
  }
  virtual int sweep_coupled_dir(const DevGrid& g, cudaStream_t st, bool fwd) = 0;
  // both coupled sweeps of a 2D grid in one cluster launch; 0 where it does not apply
  virtual int sweep_coupled_cluster(const DevGrid& g, cudaStream_t st) = 0;
  // doubles of DevGrid::CIM, the 2D coupled neighbour blocks (0: not used)
  virtual size_t ci_mat_doubles(const DevGrid& g) const = 0;
  virtual void correct(const DevGrid& g, cudaStream_t st, int mode, int clip, const double* dq) = 0;
  // chemistry surrogate coupling (raw samples; standardised inputs; decoded diagonal)
  virtual void surr_sample(const DevGrid& g, cudaStream_t st, float* X, float* T) = 0;
  virtual void surr_features(const DevGrid& g, cudaStream_t st, float* X, const double* norm) = 0;
  virtual void surr_decode(const DevGrid& g, cudaStream_t st, const float* Y, const double* norm) = 0;
  // offset (in units of N) and count of a named auxiliary field, or -1
  virtual int aux_field(const char* name, int* count) const = 0;
  static int blocks(long n, int t) { return (int)((n + t - 1) / t); }
};

template <class G, int ND>
struct LauncherT : Launcher {
  using A = Aux<G, ND>;
  LauncherT() {
    ns = G::NS;
    ntemp = G::NTEMP;
    nq = A::NQ;
    nF = A::NF;
    nci = A::NCI;
    ng = A::NG;
    naux = A::COUNT;
    nd = ND;
  }

  cudaError_t init_constants() override {
    ReactionData h[21];
    std::memset(h, 0, sizeof h);
    static const double effs[4][11] = {{0}, CS_EFF_N2, CS_EFF_O2, CS_EFF_NO};
    for (int r = 0; r < 21; ++r) {
      const ReactionInit& x = kReactionInit[r];
      h[r].nr = x.nr;
      h[r].r[0] = x.r0;
      h[r].r[1] = x.r1;
      h[r].np = x.np;
      h[r].p[0] = x.p0;
      h[r].p[1] = x.p1;
      h[r].p[2] = x.p2;
      h[r].third = x.third;
      h[r].lnA = log(x.A_cgs * 1e-3);   // cm^3/(mol s) -> m^3/(kmol s)
      h[r].n = x.n;
      h[r].theta = x.theta;
      h[r].tf = x.tf;
      h[r].tb = x.tb;
      for (int s = 0; s < 11; ++s) h[r].eff[s] = effs[x.effset][s];
    }
    cudaError_t e = cudaMemcpyToSymbol(c_reactions, h, sizeof h);
    if (e != cudaSuccess) return e;
    // species-derived constants (see GasConst)
    GasConst gc;
    std::memset(&gc, 0, sizeof gc);
    static const SpeciesData kPerfectHost = {DIATOMIC, 28.9647, 0.0, 2.88, 2, 1, 0.0};
    const SpeciesData* sp = G::PERFECT ? &kPerfectHost : kSpeciesHost;
    for (int s = 0; s < G::NS; ++s) {
      gc.Rs[s] = kRu / sp[s].M;
      gc.hf[s] = sp[s].h0 / sp[s].M;
      gc.invM[s] = 1.0 / sp[s].M;
    }
    for (int s = 0; s < G::NS && !G::PERFECT; ++s) {
      const double m = sp[s].M / kNa;
      double v = -1.5 * log(2.0 * kPi * m * kKb / (kH * kH)) - log(kKb / kPref) - log(sp[s].g0);
      if (sp[s].kind == DIATOMIC) v += log(sp[s].sigma * sp[s].thr);
      gc.gc0[s] = v;
      gc.cbk[s] = sqrt(8.0 * kRu / (kPi * sp[s].M));
      gc.icbk[s] = 1.0 / gc.cbk[s];
      for (int q = 0; q < G::NS; ++q) {
        if (sp[s].kind != DIATOMIC || sp[s].thv <= 0.0 || sp[q].kind == ELECTRON) continue;
        const double mu = sp[s].M * sp[q].M / (sp[s].M + sp[q].M);
        const double A = 1.16e-3 * sqrt(mu) * pow(sp[s].thv, 4.0 / 3.0);
        const double B = 0.015 * pow(mu, 0.25);
        // tau_sq p = exp(A (T^-1/3 - B) - 18.42); store the exponent of 1/(tau_sq p)
        gc.mwA[s][q] = A;
        gc.mwAB[s][q] = A * B + 18.42;
      }
    }
    gc.lnPRu = log(kPref / kRu);
    for (int s = 0; s < G::NS && !G::PERFECT; ++s) {
      gc.blA[s] = kBlottnerHost[s][0];
      gc.blB[s] = kBlottnerHost[s][1];
      gc.blC[s] = kBlottnerHost[s][2];
      const double ms = sp[s].M / kNa;
      gc.hsd[s] = (5.0 / 16.0) * sqrt(kPi * ms * kKb) / kPi;
      gc.ipm[s] = kNa / sp[s].M;
      for (int r = 0; r < G::NS; ++r) {
        const double mr = sp[r].M / kNa, msr = ms * mr / (ms + mr);
        gc.wm[s][r] = pow(sp[r].M / sp[s].M, 0.25);
        gc.wd[s][r] = 1.0 / sqrt(8.0 * (1.0 + sp[s].M / sp[r].M));
        gc.dsr[s][r] = 3.0 / 8.0 * sqrt(kKb / (2.0 * kPi * msr));
      }
    }
    for (int s = 0; s < G::NS; ++s) {
      gc.Rsf[s] = (float)gc.Rs[s];
      gc.hff[s] = (float)gc.hf[s];
      gc.thvf[s] = (float)sp[s].thv;
    }
    double tab[64];
    for (int j = 0; j < 64; ++j) tab[j] = exp2(j / 64.0);
    e = cudaMemcpyToSymbol(g_exp2_64, tab, sizeof tab);
    if (e != cudaSuccess) return e;
    double lnF[256], invF[256];
    for (int j = 0; j < 256; ++j) {
      lnF[j] = log1p(j / 256.0);
      invF[j] = 1.0 / (1.0 + j / 256.0);
    }
    if ((e = cudaMemcpyToSymbol(g_lnF_256, lnF, sizeof lnF)) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(g_invF_256, invF, sizeof invF)) != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_gas, &gc, sizeof gc);
  }

  void freestream(const DevGrid& g, cudaStream_t st, const double* in, double* fsQ) override {
    k_freestream<G, ND><<<1, 1, 0, st>>>(g, in, fsQ);
  }
  void fill(const DevGrid& g, cudaStream_t st, const double* fsQ) override {
    k_fill<G, ND><<<blocks(g.N, 256), 256, 0, st>>>(g, fsQ);
  }

  void primitive_state(const DevGrid& g, cudaStream_t st) override {
    k_primitive<G, ND><<<blocks(g.N, CS_PRIM_THREADS), CS_PRIM_THREADS, 0, st>>>(g);
    if (g.transport) k_transport<G, ND><<<blocks(g.N, 128), 128, 0, st>>>(g);
  }
  void chem(const DevGrid& g, cudaStream_t st) override {
    k_chem<G, ND><<<blocks(g.N, 128), 128, 0, st>>>(g);
  }
  void gradient(const DevGrid& g, cudaStream_t st) override {
    k_gradient<G, ND><<<blocks(g.N, 128), 128, 0, st>>>(g);
  }
  void flux(const DevGrid& g, cudaStream_t st) override {
    if (g.hcorr) {
      k_eta<G, ND, 0><<<blocks(g.nf[0], 256), 256, 0, st>>>(g);
      k_eta<G, ND, 1><<<blocks(g.nf[1], 256), 256, 0, st>>>(g);
      if (ND == 3) k_eta<G, ND, (ND == 3 ? 2 : 1)><<<blocks(g.nf[2], 256), 256, 0, st>>>(g);
    }
    k_flux<G, ND, 0><<<blocks(g.nf[0], 128), 128, 0, st>>>(g);
    k_flux<G, ND, 1><<<blocks(g.nf[1], 128), 128, 0, st>>>(g);
    if (ND == 3) k_flux<G, ND, (ND == 3 ? 2 : 1)><<<blocks(g.nf[2], 128), 128, 0, st>>>(g);
  }
  void assemble(const DevGrid& g, cudaStream_t st, int stag, double* out) override {
    const int nb = blocks(g.N, 256);
    k_assemble<G, ND><<<nb, 256, 0, st>>>(g);
    k_norms<G, ND><<<1, 256, 0, st>>>(g, nb, stag, out);
  }

  void spectral(const DevGrid& g, cudaStream_t st) override {
    k_spectral<G, ND><<<blocks(g.N, 128), 128, 0, st>>>(g);
  }

  // cells of hyperplane h: 2D j in [max(0, h-ni+1), min(h, nj-1)]; 3D all (j, k) pairs
  void plane_range(const DevGrid& g, int h, int& off, int& count) const {
    if (ND == 2) {
      const int jlo = h - g.ni + 1 > 0 ? h - g.ni + 1 : 0;
      const int jhi = h < g.nj - 1 ? h : g.nj - 1;
      off = jlo;
      count = jhi - jlo + 1;
    } else {
      off = 0;
      count = g.nj * g.nk;
    }
  }

  // Can `kern` run as clusters of C CTAs (32 x warps threads each), one cluster per component
  // (the flow block and `groups` species groups), with dyn_smem bytes of dynamic shared memory?
  // The opt-in limit is a property of the kernel, shared by every grid of the process, so it is
  // set to attr_smem, the largest size any grid launches the kernel with (a probe of a smaller
  // grid must not lower the limit a larger grid's launches rely on).
  template <class K>
  bool cluster_fits(K kern, int C, int warps, int groups, size_t dyn_smem = 0, size_t attr_smem = 0) {
    if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (attr_smem < dyn_smem) attr_smem = dyn_smem;
    // static plus dynamic shared memory above 48 KiB needs the opt-in
    if (attr_smem > 0 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)attr_smem) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3(C * (1 + groups));
    cfg.blockDim = dim3(32 * warps);
    cfg.dynamicSmemBytes = dyn_smem;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n >= 1) return true;
    cudaGetLastError();
    return false;
  }

  // The direct-load cluster kernel fits with C CTAs per cluster (checked for its two-warp form,
  // the one with more registers per CTA); clusters above 8 CTAs are allowed for both forms.
  template <class T>
  bool direct_fits(int C) {
    if (C > 8 && cudaFuncSetAttribute(k_split_cluster<G, T, 1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return cluster_fits(k_split_cluster<G, T, 2>, C, 2, cluster_species_clusters<G>());
  }

  // Cluster size for the direct-load cluster sweep (0: not available for this grid / device).
  template <class T>
  int cluster_size(const DevGrid& g, int& probed) {
    if (ND != 2 || g.bc[2] == BC_PERIODIC) return 0;
    if (force_C > 0) return (g.nj + force_C - 1) / force_C <= kClusterRows ? force_C : 0;
    if (probed >= 0) return probed;
    probed = 0;
    for (int C : {16, 8, 4, 2}) {
      if ((g.nj + C - 1) / C > kClusterRows) continue;
      if (direct_fits<T>(C)) {
        probed = C;
        break;
      }
    }
    return probed;
  }
  int probed64_ = -1, probed32_ = -1;

  // one launch: both sweeps of the flow block and of every species (returns launches)
  int sweep_split_cluster(const DevGrid& g, cudaStream_t st, bool mixed) override {
    // measured on GB300: the assembled couplings exchanged point to point (both precisions),
    // then in FP32 the one-CTA-per-component kernel (where nj fits) and the wavefront-record
    // kernel, in FP64 the assembled couplings with a cluster barrier and the direct-load kernel
    const int kind = cluster_kind ? cluster_kind : 4;
    if (kind >= 4) {
      // 4: point to point, then (FP64) the cluster barrier; 5: the barrier
      const int n = mixed ? (kind != 5 ? sweep_mat<float>(g, st, true) : 0)
                          : sweep_mat<double>(g, st, kind != 5);
      if (n) return n;
    }
    const int alt = kind >= 4 ? (mixed ? 3 : 1) : kind;
    if (alt == 3 && mixed && g.wrec) {
      const int n = sweep_block(g, st);
      if (n) return n;
    }
    if ((alt == 2 || alt == 3) && g.wrec) {
      const int n = mixed ? sweep_wave_t<float>(g, st, wprobed32_) : sweep_wave_t<double>(g, st, wprobed64_);
      if (n) return n;
    }
    return mixed ? sweep_cluster_t<float>(g, st, probed32_) : sweep_cluster_t<double>(g, st, probed64_);
  }
  int wprobed64_ = -1, wprobed32_ = -1;

  // wavefront-record kernel: cluster size with at most kWaveRows rows per CTA
  template <class T>
  int wave_cluster_size(const DevGrid& g, int& probed) {
    if (ND != 2 || g.bc[2] == BC_PERIODIC) return 0;
    if (force_C > 0) return (g.nj + force_C - 1) / force_C <= kWaveRows ? force_C : 0;
    if (probed >= 0) return probed;
    probed = 0;
    for (int C : {16, 8, 4, 2, 1}) {
      if ((g.nj + C - 1) / C > kWaveRows) continue;
      if (cluster_fits(k_split_wave<G, T>, C, 1, species_clusters<G>())) {
        probed = C;
        break;
      }
    }
    return probed;
  }

  int cluster_sizes(const DevGrid& g, int kind, bool mixed) override {
    if (ND != 2 || g.bc[2] == BC_PERIODIC) return 0;
    int mask = 0;
    for (int C : {1, 2, 4, 8, 16}) {
      bool ok;
      if (kind == 2) {
        ok = (g.nj + C - 1) / C <= kWaveRows && g.wrec &&
             (mixed ? cluster_fits(k_split_wave<G, float>, C, 1, species_clusters<G>()) : cluster_fits(k_split_wave<G, double>, C, 1, species_clusters<G>()));
      } else {
        ok = C >= 2 && (g.nj + C - 1) / C <= kClusterRows &&
             (mixed ? direct_fits<float>(C) : direct_fits<double>(C));
      }
      if (ok) mask |= 1 << C;
    }
    return mask;
  }

  void prepare(const DevGrid& g, bool mixed) override {
    const int kind = cluster_kind ? cluster_kind : 4;
    if (kind >= 4 && g.SMC) {
      if (mixed) {
        if (kind != 5) mat_cluster_size<float>(g, true);
      } else {
        mat_cluster_size<double>(g, false);
        if (kind != 5) mat_cluster_size<double>(g, true);
      }
    }
    const int alt = kind >= 4 ? (mixed ? 3 : 1) : kind;
    if (alt == 3 && mixed) block_ok(g);   // (fallbacks of the assembled-coupling sweeps)
    if (alt == 2 || alt == 3) {
      if (mixed) wave_cluster_size<float>(g, wprobed32_);
      else wave_cluster_size<double>(g, wprobed64_);
    }
    if (mixed) cluster_size<float>(g, probed32_);
    else cluster_size<double>(g, probed64_);
  }

  // FP32 block kernel: one CTA per component with every row (0 when it does not apply)
  bool block_ok(const DevGrid& g) {
    if (ND != 2 || g.bc[2] == BC_PERIODIC || g.nj > kBlockRows) return false;
    if (block_probed_ < 0) {
      block_probed_ = cudaFuncSetAttribute(k_split_block<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)block_smem_bytes<G>()) == cudaSuccess ? 1 : 0;
      cudaGetLastError();
    }
    return block_probed_ == 1;
  }
  int block_probed_ = -1;
  bool block_available(const DevGrid& g) override { return block_ok(g); }
  int sweep_block(const DevGrid& g, cudaStream_t st) {
    sweep_split_cluster_ok = false;
    if (!block_ok(g)) return 0;
    k_pack_wave<G, float><<<blocks(g.N, 128), 128, 0, st>>>(g);
    const int threads = ((g.nj + 31) / 32) * 32;
    k_split_block<G><<<1 + species_clusters<G>(), threads, block_smem_bytes<G>(), st>>>(g);
    if (cudaGetLastError() != cudaSuccess) return 0;
    sweep_split_cluster_ok = true;
    last_sweep = 4;
    last_sweep_C = 1;
    return 2;
  }

  template <class T>
  int sweep_wave_t(const DevGrid& g, cudaStream_t st, int& probed) {
    sweep_split_cluster_ok = false;
    const int C = wave_cluster_size<T>(g, probed);
    if (C == 0) return 0;
    k_pack_wave<G, T><<<blocks(g.N, 128), 128, 0, st>>>(g);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3(C * (1 + species_clusters<G>()));
    cfg.blockDim = dim3(32);
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const int R = (g.nj + C - 1) / C;
    if (cudaLaunchKernelEx(&cfg, k_split_wave<G, T>, g, R) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    sweep_split_cluster_ok = true;
    last_sweep = 2;
    last_sweep_C = C;
    return 2;
  }
  template <class T>
  int sweep_cluster_t(const DevGrid& g, cudaStream_t st, int& probed) {
    sweep_split_cluster_ok = false;
    if (ND != 2) return 0;
    const int C = cluster_size<T>(g, probed);
    if (C == 0) return 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3(C * (1 + cluster_species_clusters<G>()));
    const int W = cluster_warps == 1 ? 1 : 2;
    cfg.blockDim = dim3(32 * W);
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const int R = (g.nj + C - 1) / C;
    const cudaError_t e = W == 1 ? cudaLaunchKernelEx(&cfg, k_split_cluster<G, T, 1>, g, R)
                                 : cudaLaunchKernelEx(&cfg, k_split_cluster<G, T, 2>, g, R);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    sweep_split_cluster_ok = true;
    last_sweep = 1;
    last_sweep_C = C;
    return 1;
  }

  // 2D sweeps over assembled couplings (K6e): k_sweep_mat, then one cluster launch with
  // kMatSlots threads per row, point to point between CTAs (k_split_p2p) where its ring fits in
  // shared memory, else (FP64 only) with a cluster barrier per hyperplane (k_split_mat).  T is
  // the operator's type (FP64, or FP32 for the mixed-precision operator).  Single grids only: a
  // batch keeps the one-warp direct kernel, whose CTAs need fewer registers and no records.
  size_t mat_doubles(const DevGrid& g) const override {
    // only where a cluster of at most 16 CTAs can hold the rows
    if (ND != 2 || g.bc[2] == BC_PERIODIC || g.nj > 16 * kClusterRows) return 0;
    const size_t d = (size_t)g.N * MatRec<G, double>::CELL + (size_t)g.nj * MatRec<G, double>::ROW;
    const size_t f = ((size_t)g.N * MatRec<G, float>::CELL + (size_t)g.nj * MatRec<G, float>::ROW + 1) / 2;
    return d > f ? d : f;
  }
  static constexpr size_t kP2PMaxSmem = 200 * 1024;
  // will a split sweep of this precision read the coupling records?  (The records are
  // allocated only then: for the FP32 operator they serve only k_split_p2p, whose ring may not
  // fit the grid.)
  bool mat_usable(const DevGrid& g, bool mixed) override {
    const int kind = cluster_kind ? cluster_kind : 4;
    if (ND != 2 || !use_cluster || cluster_warps == 1 || kind < 4) return false;
    if (mixed) return kind != 5 && mat_cluster_size<float>(g, true) > 0;
    return (kind != 5 && mat_cluster_size<double>(g, true) > 0) || mat_cluster_size<double>(g, false) > 0;
  }
  template <class T>
  bool mat_fits(const DevGrid& g, int C, bool p2p) {
    const int R = (g.nj + C - 1) / C;
    if (R > kClusterRows) return false;
    const int warps = (kMatSlots * R + 31) / 32;
    if (!p2p) return std::is_same<T, double>::value && cluster_fits(k_split_mat<G>, C, warps, mat_species_groups<G>());
    const size_t smem = p2p_smem_bytes<T, MatRec<G, T>::NP>(g.ni, g.nj, 32 * warps);
    return smem <= kP2PMaxSmem && cluster_fits(k_split_p2p<G, T>, C, warps, mat_species_groups<G>(), smem, kP2PMaxSmem);
  }
  template <class T>
  int mat_cluster_size(const DevGrid& g, bool p2p) {
    if (ND != 2 || g.bc[2] == BC_PERIODIC) return 0;
    const int m = (p2p ? 1 : 0) + (std::is_same<T, float>::value ? 2 : 0);
    if (force_C > 0) {
      if (mat_forced_C_[m] != force_C) {
        mat_forced_C_[m] = force_C;
        mat_forced_ok_[m] = mat_fits<T>(g, force_C, p2p);
      }
      return mat_forced_ok_[m] ? force_C : 0;
    }
    if (mat_probed_[m] >= 0) return mat_probed_[m];
    mat_probed_[m] = 0;
    for (int C : {16, 8, 4, 2}) {
      if (mat_fits<T>(g, C, p2p)) {
        mat_probed_[m] = C;
        break;
      }
    }
    return mat_probed_[m];
  }
  int mat_probed_[4] = {-1, -1, -1, -1}, mat_forced_C_[4] = {0, 0, 0, 0};
  bool mat_forced_ok_[4] = {false, false, false, false};
  template <class T>
  int sweep_mat(const DevGrid& g, cudaStream_t st, bool allow_p2p) {
    sweep_split_cluster_ok = false;
    if constexpr (ND != 2) {
      return 0;
    } else {
      if (cluster_warps == 1 || !g.SMC) return 0;
      int C = allow_p2p ? mat_cluster_size<T>(g, true) : 0;
      const bool p2p = C > 0;
      if (!p2p) C = std::is_same<T, double>::value ? mat_cluster_size<T>(g, false) : 0;
      if (C == 0) return 0;
      const int R = (g.nj + C - 1) / C;
      k_sweep_mat<G, T><<<blocks(g.N, 128), 128, 0, st>>>(g);
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      cfg.gridDim = dim3(C * (1 + mat_species_groups<G>()));
      cfg.blockDim = dim3((kMatSlots * R + 31) / 32 * 32);
      cfg.dynamicSmemBytes = p2p ? p2p_smem_bytes<T, MatRec<G, T>::NP>(g.ni, g.nj, (kMatSlots * R + 31) / 32 * 32) : 0;
      cfg.stream = st;
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      const cudaError_t e = p2p ? cudaLaunchKernelEx(&cfg, k_split_p2p<G, T>, g, R)
                                : cudaLaunchKernelEx(&cfg, k_split_mat<G>, g, R);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      sweep_split_cluster_ok = true;
      last_sweep = p2p ? 5 : 6;
      last_sweep_C = C;
      return 2;
    }
  }

  int sweep_split_dir(const DevGrid& g, cudaStream_t st, bool fwd, bool mixed) override {
    const int H = g.ni + g.nj + (ND == 3 ? g.nk : 1) - 2;
    int launches = 0;
    last_sweep = 0;
    last_sweep_C = 0;
    for (int t = 0; t <= H; ++t) {
      const int h = fwd ? t : H - t;
      int off, cnt;
      plane_range(g, h, off, cnt);
      if (cnt <= 0) continue;
      const int nb = blocks(cnt, 32);
      if (mixed) {
        if (fwd) k_sweep_split<G, ND, true, float><<<nb, 32, 0, st>>>(g, h, off, cnt);
        else k_sweep_split<G, ND, false, float><<<nb, 32, 0, st>>>(g, h, off, cnt);
      } else {
        if (fwd) k_sweep_split<G, ND, true, double><<<nb, 32, 0, st>>>(g, h, off, cnt);
        else k_sweep_split<G, ND, false, double><<<nb, 32, 0, st>>>(g, h, off, cnt);
      }
      ++launches;
    }
    return launches;
  }

  void ci_block(const DevGrid& g, cudaStream_t st) override {
    k_ci_block<G, ND><<<blocks(g.N, 64), 64, 0, st>>>(g);
  }

  size_t ci_mat_doubles(const DevGrid& g) const override {
    // only where a cluster of at most 16 CTAs can hold the rows
    if (ND != 2 || g.bc[2] == BC_PERIODIC || g.nj > 16 * kCIRows) return 0;
    return (size_t)g.N * CIRec<G>::CELL + (size_t)g.nj * CIRec<G>::ROW;
  }
  // both coupled sweeps over assembled neighbour blocks (k_ci_mat, then k_ci_mat_sweep with
  // kCISlots threads per row); 0 where the blocks are not allocated or no cluster fits
  int ci_mat_probed_ = -1;
  int sweep_coupled_mat(const DevGrid& g, cudaStream_t st) {
    if constexpr (ND != 2) {
      return 0;
    } else {
      if (!g.CIM || g.bc[2] == BC_PERIODIC) return 0;
      if (ci_mat_probed_ < 0) {
        ci_mat_probed_ = 0;
        for (int C : {16, 8, 4, 2}) {
          const int R = (g.nj + C - 1) / C;
          if (R > kCIRows) continue;
          if (cluster_fits(k_ci_mat_sweep<G>, C, (kCISlots * R + 31) / 32, 0)) {
            ci_mat_probed_ = C;
            break;
          }
        }
      }
      const int C = ci_mat_probed_;
      if (C == 0) return 0;
      const int R = (g.nj + C - 1) / C;
      k_ci_mat<G><<<blocks(g.N, 64), 64, 0, st>>>(g);
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      cfg.gridDim = dim3(C);
      cfg.blockDim = dim3((kCISlots * R + 31) / 32 * 32);
      cfg.stream = st;
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      if (cudaLaunchKernelEx(&cfg, k_ci_mat_sweep<G>, g, R) != cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      return 2;
    }
  }
  int ci_probed_ = -1;
  int sweep_coupled_cluster(const DevGrid& g, cudaStream_t st) override {
    if constexpr (ND != 2) {
      return 0;
    } else {
      if (g.bc[2] == BC_PERIODIC) return 0;
      if (const int n = sweep_coupled_mat(g, st)) return n;
      if (ci_probed_ < 0) {
        ci_probed_ = 0;
        for (int C : {16, 8, 4, 2}) {
          if ((g.nj + C - 1) / C > kClusterRows) continue;
          if (cluster_fits(k_ci_cluster<G>, C, 1, 0)) { ci_probed_ = C; break; }
        }
      }
      const int C = ci_probed_;
      if (C == 0) return 0;
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      cfg.gridDim = dim3(C);
      cfg.blockDim = dim3(32);
      cfg.stream = st;
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      const int R = (g.nj + C - 1) / C;
      if (cudaLaunchKernelEx(&cfg, k_ci_cluster<G>, g, R) != cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      return 1;
    }
  }

  int sweep_coupled_dir(const DevGrid& g, cudaStream_t st, bool fwd) override {
    const int H = g.ni + g.nj + (ND == 3 ? g.nk : 1) - 2;
    int launches = 0;
    for (int t = 0; t <= H; ++t) {
      const int h = fwd ? t : H - t;
      int off, cnt;
      plane_range(g, h, off, cnt);
      if (cnt <= 0) continue;
      if (fwd) k_sweep_coupled<G, ND, true><<<blocks(cnt, 32), 32, 0, st>>>(g, h, off, cnt);
      else k_sweep_coupled<G, ND, false><<<blocks(cnt, 32), 32, 0, st>>>(g, h, off, cnt);
      ++launches;
    }
    return launches;
  }

  void surr_sample(const DevGrid& g, cudaStream_t st, float* X, float* T) override {
    k_surr_sample<G, ND><<<blocks(g.N, 128), 128, 0, st>>>(g, X, T);
  }
  void surr_features(const DevGrid& g, cudaStream_t st, float* X, const double* norm) override {
    k_surr_features<G, ND><<<blocks(g.N, 128), 128, 0, st>>>(g, X, norm);
  }
  void surr_decode(const DevGrid& g, cudaStream_t st, const float* Y, const double* norm) override {
    k_surr_decode<G, ND><<<blocks(g.N, 128), 128, 0, st>>>(g, Y, norm);
  }

  void correct(const DevGrid& g, cudaStream_t st, int mode, int clip, const double* dq) override {
    k_correct<G, ND><<<blocks(g.N, 256), 256, 0, st>>>(g, mode, clip, dq);
  }

  int aux_field(const char* name, int* count) const override {
    struct E { const char* n; int off, cnt; };
    const E tab[] = {{"rho", A::RHO, 1}, {"u", A::U, ND}, {"T", A::T, 1}, {"Tv", A::TV, 1},
                     {"p", A::P, 1}, {"c", A::C, 1}, {"beta", A::BETA, 1}, {"Gam", A::GAM, 1},
                     {"H", A::H, 1}, {"mu", A::MU, 1}, {"kt", A::KT, 1}, {"kv", A::KV, 1},
                     {"rhoD", A::RHOD, 1}, {"rhoDs", A::RHODS, G::NS}, {"relax", A::RELAX, 1},
                     {"omega_v", A::OMV, 1}, {"cv", A::CV, 1}, {"cvtr", A::CVTR, 1}, {"cvve", A::CVVE, 1},
                     {"omega", A::OM, G::NS}, {"dom", A::DOM, G::NS}, {"prs", A::PRS, G::NS}};
    for (const E& e : tab)
      if (!std::strcmp(e.n, name)) { *count = e.cnt; return e.off; }
    return -1;
  }
};

Launcher* make_launcher_perfect_2d();
Launcher* make_launcher_perfect_3d();
Launcher* make_launcher_air5_2d();
Launcher* make_launcher_air5_3d();
Launcher* make_launcher_air11_2d();
Launcher* make_launcher_air11_3d();

}  // namespace cs
