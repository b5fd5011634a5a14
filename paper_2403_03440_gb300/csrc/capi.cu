// C ABI of the library (include/cs.h): grid objects, device memory, geometry kernels and the
// host-side sequencing of the iteration (Sec. 2.2-2.3 of arXiv:2403.03440).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "../../include/cs.h"
#include "launcher.cuh"

using namespace cs;

// the chemistry surrogate network (mlp.cu)
int mlp_max_batch(cs_mlp m);
void mlp_forward_on(cs_mlp m, const float* X, int n, float* Y, cudaStream_t st);

// phases timed by cs_profile: primitive, gradient, flux, assemble, spectral (+CI blocks),
// forward sweep, backward sweep, correction
#define CS_NPHASE 8

// ---------------------------------------------------------------------------------------
// Geometry (a1; Sec. 2.2 metrics in finite-volume form): face area vectors oriented along +d,
// face centroids, cell volumes and centroids.
// ---------------------------------------------------------------------------------------
struct GeomArgs {
  int nd, ni, nj, nk;
  const double* node[3];
  double* S[3];
  double* fc[3];
  int nf[3];
  double* V;
  double* xc;
};

__device__ __forceinline__ void node_at(const GeomArgs& a, int i, int j, int k, double* x) {
  const size_t n = i + (size_t)(a.ni + 1) * (j + (size_t)(a.nj + 1) * k);
  for (int d = 0; d < 3; ++d) x[d] = d < a.nd ? a.node[d][n] : 0.0;
}

__global__ void k_geom_faces(GeomArgs a, int d) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= a.nf[d]) return;
  const int fi = a.ni + (d == 0), fj = a.nj + (d == 1);
  const int i = f % fi, j = (f / fi) % fj, k = f / (fi * fj);
  double* S = a.S[d] + 3 * (size_t)f;
  double* c = a.fc[d] + 3 * (size_t)f;
  if (a.nd == 2) {
    double p[3], q[3];
    node_at(a, i, j, 0, p);
    if (d == 0) node_at(a, i, j + 1, 0, q); else node_at(a, i + 1, j, 0, q);
    const double ex = q[0] - p[0], ey = q[1] - p[1];
    // +i face: (ey, -ex); +j face: (-ey, ex)  (right-handed (i, j))
    S[0] = d == 0 ? ey : -ey;
    S[1] = d == 0 ? -ex : ex;
    S[2] = 0.0;
    for (int q2 = 0; q2 < 3; ++q2) c[q2] = 0.5 * (p[q2] + q[q2]);
  } else {
    // quad spanned by the two cyclic axes ea, eb: S = (P_ab - P_0) x (P_b - P_a) / 2
    const int ea = (d + 1) % 3, eb = (d + 2) % 3;
    int o[3] = {i, j, k}, pa[3] = {i, j, k}, pb[3] = {i, j, k}, pab[3] = {i, j, k};
    pa[ea]++; pb[eb]++; pab[ea]++; pab[eb]++;
    double x0[3], xa[3], xb[3], xab[3];
    node_at(a, o[0], o[1], o[2], x0);
    node_at(a, pa[0], pa[1], pa[2], xa);
    node_at(a, pb[0], pb[1], pb[2], xb);
    node_at(a, pab[0], pab[1], pab[2], xab);
    const double d1[3] = {xab[0] - x0[0], xab[1] - x0[1], xab[2] - x0[2]};
    const double d2[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
    S[0] = 0.5 * (d1[1] * d2[2] - d1[2] * d2[1]);
    S[1] = 0.5 * (d1[2] * d2[0] - d1[0] * d2[2]);
    S[2] = 0.5 * (d1[0] * d2[1] - d1[1] * d2[0]);
    for (int q2 = 0; q2 < 3; ++q2) c[q2] = 0.25 * (x0[q2] + xa[q2] + xb[q2] + xab[q2]);
  }
}

__global__ void k_geom_cells(GeomArgs a) {
  const long N = (long)a.ni * a.nj * (a.nd == 3 ? a.nk : 1);
  const long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  const int i = c % a.ni, j = (c / a.ni) % a.nj, k = c / ((long)a.ni * a.nj);
  if (a.nd == 2) {
    double p0[3], p1[3], p2[3], p3[3];
    node_at(a, i, j, 0, p0);
    node_at(a, i + 1, j, 0, p1);
    node_at(a, i + 1, j + 1, 0, p2);
    node_at(a, i, j + 1, 0, p3);
    const double a1 = 0.5 * ((p1[0] - p0[0]) * (p2[1] - p0[1]) - (p2[0] - p0[0]) * (p1[1] - p0[1]));
    const double a2 = 0.5 * ((p2[0] - p0[0]) * (p3[1] - p0[1]) - (p3[0] - p0[0]) * (p2[1] - p0[1]));
    a.V[c] = a1 + a2;
    for (int q = 0; q < 2; ++q)
      a.xc[q * N + c] = (a1 * (p0[q] + p1[q] + p2[q]) + a2 * (p0[q] + p2[q] + p3[q])) / (3.0 * (a1 + a2));
    a.xc[2 * N + c] = 0.0;
  } else {
    double v = 0.0;
    for (int d = 0; d < 3; ++d) {
      const int fi = a.ni + (d == 0), fj = a.nj + (d == 1);
      int hi[3] = {i, j, k};
      hi[d]++;
      const size_t fl = i + (size_t)fi * (j + (size_t)fj * k);
      const size_t fh = hi[0] + (size_t)fi * (hi[1] + (size_t)fj * hi[2]);
      for (int q = 0; q < 3; ++q)
        v += a.fc[d][3 * fh + q] * a.S[d][3 * fh + q] - a.fc[d][3 * fl + q] * a.S[d][3 * fl + q];
    }
    a.V[c] = v / 3.0;
    double x[3] = {0, 0, 0};
    for (int e = 0; e < 8; ++e) {
      double p[3];
      node_at(a, i + (e & 1), j + ((e >> 1) & 1), k + ((e >> 2) & 1), p);
      for (int q = 0; q < 3; ++q) x[q] += 0.125 * p[q];
    }
    for (int q = 0; q < 3; ++q) a.xc[q * N + c] = x[q];
  }
}

// Stagnation wall cell: j = 0 wall face whose normal is most nearly opposite to dir
// (ties within 1e-12 go to the lower index).  One block.
__global__ void k_stagnation(const double* Sj, int ni, int nj, int nk, int nd, double dx,
                             double dy, double dz, int* out) {
  __shared__ double bv[256];
  __shared__ int bi[256];
  const double dn = sqrt(dx * dx + dy * dy + dz * dz);
  double best = 1e300;
  int besti = -1;
  const int nw = ni * nk;
  for (int t = threadIdx.x; t < nw; t += blockDim.x) {
    const int i = t % ni, k = t / ni;
    const double* S = Sj + 3 * ((size_t)i + (size_t)ni * (nj + 1) * k);
    const double a = S[0] * S[0] + S[1] * S[1] + (nd == 3 ? S[2] * S[2] : 0.0);
    if (a <= 0.0) continue;
    const double v = (S[0] * dx + S[1] * dy + (nd == 3 ? S[2] * dz : 0.0)) / (sqrt(a) * dn);
    const int c = i + ni * nj * k;
    if (v < best - 1e-12 || (fabs(v - best) <= 1e-12 && c < besti)) { best = v; besti = c; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = besti;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 1e300;
    int c = -1;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      if (bi[t] < 0) continue;
      if (bv[t] < b - 1e-12 || (fabs(bv[t] - b) <= 1e-12 && bi[t] < c)) { b = bv[t]; c = bi[t]; }
    }
    *out = c;
  }
}

// ---------------------------------------------------------------------------------------
// Grid object
// ---------------------------------------------------------------------------------------
struct cs_grid_s {
  cs_grid_desc desc;
  cudaStream_t stream = nullptr;
  std::unique_ptr<Launcher> L;
  DevGrid g{};
  std::vector<void*> allocs;
  double* node[3] = {nullptr, nullptr, nullptr};
  double* fsQ = nullptr;      // device [nq]
  double* fsin = nullptr;     // device freestream description
  double* norms = nullptr;    // device [3]
  int* stag_dev = nullptr;
  double* params = nullptr;   // device [4]
  int* iter_dev = nullptr;    // device iteration counter of the CFL ramp in captured iterations
  cs_mlp surr = nullptr;      // attached surrogate network (species Jacobian diagonal)
  float *sx = nullptr, *sy = nullptr;   // its inputs [N][14] and outputs [N][22]
  double* snorm = nullptr;    // standardisation [14 + 14 + 22 + 22]
  double* h_pin = nullptr;    // pinned host scratch [64]
  double dual_dt = 0.0, dual_theta = 0.0;   // dual time stepping (dt 0: steady)
  int dual_levels = 0;        // physical levels stored (0, 1, 2)
  int* h_status = nullptr;    // pinned [4]
  int stag = -1;
  int have_R = 0, have_bc = 0, iter = 0;
  int last_op = -1;           // 0 split, 1 coupled
  bool mat_refused = false;   // the coupling records of the 2D split sweep could not be allocated
  char err[512] = {0};
  // second stream of the iteration: the chemistry beside the gradient and fluxes (created on
  // first use; the fork and join events order it within the grid's stream)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // per-phase CUDA-event timing of cs_step (enabled by cs_profile)
  bool prof = false;
  cudaEvent_t ev[8][CS_NPHASE + 1];
  int ev_used = 0;
  double prof_ms[CS_NPHASE] = {0};
  long prof_launches[CS_NPHASE] = {0};
};

static cs_status fail(cs_grid g, cs_status st, const char* fmt, ...) {
  if (g) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g->err, sizeof g->err, fmt, ap);
    va_end(ap);
  }
  return st;
}

#define CUDA_TRY(g, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail(g, CS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <class T>
static cudaError_t dalloc(cs_grid g, T** p, size_t n) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, n * sizeof(T) > 0 ? n * sizeof(T) : 8);
  if (e != cudaSuccess) return e;
  g->allocs.push_back(v);
  *p = (T*)v;
  return cudaMemsetAsync(v, 0, n * sizeof(T) > 0 ? n * sizeof(T) : 8, g->stream);
}

// zero the device status, run, then read the status back (synchronises the stream)
static cs_status begin(cs_grid g) {
  CUDA_TRY(g, cudaMemsetAsync(g->g.status, 0, 4 * sizeof(int), g->stream));
  return CS_OK;
}
static cs_status finish(cs_grid g, const char* what) {
  CUDA_TRY(g, cudaGetLastError());
  CUDA_TRY(g, cudaMemcpyAsync(g->h_status, g->g.status, 4 * sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(g, cudaStreamSynchronize(g->stream));
  const int code = g->h_status[0];
  if (code == ST_NONPHYSICAL)
    return fail(g, CS_ERR_NONPHYSICAL, "%s: non-physical state at cell %d", what, g->h_status[1]);
  if (code == ST_NEWTON)
    return fail(g, CS_ERR_NEWTON, "%s: temperature solve failed at cell %d", what, g->h_status[1]);
  if (code == ST_TIMEOUT) return fail(g, CS_ERR_TIMEOUT, "%s: device wait timed out", what);
  if (code != 0) return fail(g, CS_ERR_CUDA, "%s: device status %d", what, code);
  return CS_OK;
}

static void prof_record(cs_grid g, int slot, int phase) {
  if (g->prof) cudaEventRecord(g->ev[slot][phase], g->stream);
}
// accumulate the timings of the recorded iterations (stream already synchronised)
static void prof_resolve(cs_grid g) {
  if (!g->prof) return;
  for (int s = 0; s < g->ev_used; ++s)
    for (int p = 0; p < CS_NPHASE; ++p) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, g->ev[s][p], g->ev[s][p + 1]) == cudaSuccess) g->prof_ms[p] += ms;
    }
  g->ev_used = 0;
}

extern "C" cs_status cs_profile(cs_grid g, int enable, double* ms_out, long* launches_out) {
  if (!g) return CS_ERR_ARG;
  if (ms_out)
    for (int p = 0; p < CS_NPHASE; ++p) ms_out[p] = g->prof_ms[p];
  if (launches_out)
    for (int p = 0; p < CS_NPHASE; ++p) launches_out[p] = g->prof_launches[p];
  if (enable && !g->prof) {
    for (int s = 0; s < 8; ++s)
      for (int p = 0; p <= CS_NPHASE; ++p)
        if (cudaEventCreate(&g->ev[s][p]) != cudaSuccess) return fail(g, CS_ERR_CUDA, "event create");
  }
  if (!enable && g->prof) {
    cudaStreamSynchronize(g->stream);
    for (int s = 0; s < 8; ++s)
      for (int p = 0; p <= CS_NPHASE; ++p) cudaEventDestroy(g->ev[s][p]);
  }
  g->prof = enable != 0;
  g->ev_used = 0;
  for (int p = 0; p < CS_NPHASE; ++p) { g->prof_ms[p] = 0.0; g->prof_launches[p] = 0; }
  return CS_OK;
}

extern "C" cs_status cs_sweep_info(cs_grid g, int out[2]) {
  if (!g || !out) return CS_ERR_ARG;
  out[0] = g->L->last_sweep;
  out[1] = g->L->last_sweep_C;
  return CS_OK;
}

extern "C" cs_status cs_gas_info(int mech, double* M, double* hf, int dims[3]) {
  static const double MN = CS_MN, MO = CS_MO, ME = CS_ME;
  static const double Mair[11] = {2 * MN, 2 * MO, MN + MO, MN, MO, MN + MO - ME, 2 * MN - ME,
                                  2 * MO - ME, MN - ME, MO - ME, ME};
  static const double h0[11] = {0.0, 0.0, 89.77e6, 470.82e6, 246.79e6, 983.6e6, 1503.3e6,
                                1164.5e6, 1873.1e6, 1560.7e6, 0.0};
  int ns, nr, nt;
  if (mech == CS_MECH_PERFECT) { ns = 1; nr = 0; nt = 1; }
  else if (mech == CS_MECH_AIR5) { ns = 5; nr = 5; nt = 1; }
  else if (mech == CS_MECH_AIR11) { ns = 11; nr = 21; nt = 2; }
  else return CS_ERR_ARG;
  for (int s = 0; s < ns; ++s) {
    M[s] = mech == CS_MECH_PERFECT ? 28.9647 : Mair[s];
    hf[s] = mech == CS_MECH_PERFECT ? 0.0 : h0[s] / Mair[s];
  }
  dims[0] = ns;
  dims[1] = nr;
  dims[2] = nt;
  return CS_OK;
}

static void make_side(cs_grid g);

extern "C" cs_status cs_grid_create(const cs_grid_desc* desc, const double* nodes_host,
                                    void* cuda_stream, cs_grid* out) {
  if (!desc || !nodes_host || !out) return CS_ERR_ARG;
  *out = nullptr;
  const int nd = desc->ndim;
  if (nd < 2 || nd > 3 || desc->ni < 2 || desc->nj < 1 || (nd == 3 && desc->nk < 1))
    return CS_ERR_ARG;
  for (int d = 0; d < nd; ++d) {
    const int lo = desc->bc[2 * d], hi = desc->bc[2 * d + 1];
    if (lo < 0 || lo > 4 || hi < 0 || hi > 4) return CS_ERR_ARG;
    if ((lo == CS_BC_PERIODIC) != (hi == CS_BC_PERIODIC)) return CS_ERR_ARG;
  }
  if (desc->limiter < 0 || desc->limiter > 2) return CS_ERR_ARG;
  std::unique_ptr<cs_grid_s> G(new cs_grid_s());
  cs_grid g = G.get();
  g->desc = *desc;
  g->stream = (cudaStream_t)cuda_stream;
  Launcher* L = nullptr;
  if (desc->mech == CS_MECH_PERFECT) L = nd == 2 ? make_launcher_perfect_2d() : make_launcher_perfect_3d();
  else if (desc->mech == CS_MECH_AIR5) L = nd == 2 ? make_launcher_air5_2d() : make_launcher_air5_3d();
  else if (desc->mech == CS_MECH_AIR11) L = nd == 2 ? make_launcher_air11_2d() : make_launcher_air11_3d();
  if (!L) return CS_ERR_ARG;
  g->L.reset(L);
  if (L->init_constants() != cudaSuccess) return CS_ERR_CUDA;

  DevGrid& d = g->g;
  d.nd = nd;
  d.ni = desc->ni;
  d.nj = desc->nj;
  d.nk = nd == 3 ? desc->nk : 1;
  const long N = (long)d.ni * d.nj * d.nk;
  if (N > 0x7fffffffL / 4) return CS_ERR_ARG;
  d.N = (int)N;
  for (int k = 0; k < 6; ++k) d.bc[k] = desc->bc[k];
  d.limiter = desc->limiter;
  d.react = desc->reacting;
  d.efix = desc->entropy_fix;
  d.hcorr = 1;
  d.ulim = 0.0;
  d.nojac = 0;
  d.Tw = 300.0;
  for (int k = 0; k < 3; ++k) d.nf[k] = 0;
  for (int k = 0; k < nd; ++k)
    d.nf[k] = (d.ni + (k == 0)) * (d.nj + (k == 1)) * (nd == 3 ? d.nk + (k == 2) : 1);
  const size_t nn = (size_t)(d.ni + 1) * (d.nj + 1) * (nd == 3 ? d.nk + 1 : 1);
  cudaError_t e = cudaSuccess;
#define ALLOC(p, n) do { if ((e = dalloc(g, &(p), (n))) != cudaSuccess) return e == cudaErrorMemoryAllocation ? CS_ERR_OOM : CS_ERR_CUDA; } while (0)
  for (int k = 0; k < nd; ++k) {
    ALLOC(g->node[k], nn);
    double* S;
    double* fc;
    ALLOC(S, 3 * (size_t)d.nf[k]);
    ALLOC(fc, 3 * (size_t)d.nf[k]);
    d.S[k] = S;
    d.fc[k] = fc;
    ALLOC(d.F[k], (size_t)L->nq * d.nf[k]);
    ALLOC(d.eta[k], (size_t)d.nf[k]);
  }
  for (int k = nd; k < 3; ++k) { d.S[k] = nullptr; d.fc[k] = nullptr; d.F[k] = nullptr; d.eta[k] = nullptr; }
  double *V, *xc;
  ALLOC(V, N);
  ALLOC(xc, 3 * N);
  d.V = V;
  d.xc = xc;
  ALLOC(d.Q, (size_t)L->nq * N);
  ALLOC(d.W, (size_t)L->naux * N);
  ALLOC(d.fsW, (size_t)L->naux);
  ALLOC(d.grad, (size_t)L->ng * 3 * N);
  ALLOC(d.R, (size_t)L->nq * N);
  ALLOC(d.lamF, 3 * N);
  ALLOC(d.lamC, 3 * N);
  ALLOC(d.lamCI, 3 * N);
  ALLOC(d.DF, N);
  ALLOC(d.DFev, N);
  ALLOC(d.Ds, (size_t)L->ns * N);
  ALLOC(d.Vdt, N);
  ALLOC(d.invD, (size_t)(2 + L->ns) * N);
  ALLOC(d.rhsF, (size_t)L->nF * N);
  d.woff = nullptr;
  d.wrec = d.wrecs = d.wbase = nullptr;
  if (nd == 2) {
    // hyperplane offsets of the wavefront-ordered sweep records (2D)
    const int H = d.ni + d.nj - 2;
    std::vector<int> off(H + 2, 0);
    for (int h = 0; h <= H; ++h) {
      const int jlo = h - d.ni + 1 > 0 ? h - d.ni + 1 : 0, jhi = h < d.nj - 1 ? h : d.nj - 1;
      off[h + 1] = off[h] + (jhi - jlo + 1);
    }
    int* woff;
    ALLOC(woff, H + 2);
    if (cudaMemcpyAsync(woff, off.data(), (H + 2) * sizeof(int), cudaMemcpyHostToDevice, g->stream) != cudaSuccess)
      return CS_ERR_CUDA;
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return CS_ERR_CUDA;
    d.woff = woff;
    const size_t groups = (L->ns + kSpeciesGroup - 1) / kSpeciesGroup;
    double *wr, *wrs, *wb;
    ALLOC(wr, (size_t)kRecF * N);
    ALLOC(wrs, groups * kRecS * N);
    ALLOC(wb, (8 + kSpeciesGroup * groups) * N);
    d.wrec = wr;
    d.wrecs = wrs;
    d.wbase = wb;
  }
  ALLOC(d.dQs, (size_t)(L->nF + L->ns) * N);
  ALLOC(d.dQ, (size_t)(L->nF + L->ns) * N);
  ALLOC(d.dQcs, (size_t)L->nci * N);
  ALLOC(d.dQc, (size_t)L->nci * N);
  ALLOC(d.red, 2 * (size_t)Launcher::blocks(N, 256) + 2);
  ALLOC(d.status, 4);
  ALLOC(g->fsQ, 32);
  ALLOC(g->fsin, 32);
  ALLOC(g->norms, 4);
  ALLOC(g->stag_dev, 1);
  ALLOC(g->params, 4);
  ALLOC(g->iter_dev, 1);
#undef ALLOC
  d.DLU = nullptr;
  d.DINV = nullptr;
  d.CIM = nullptr;
  d.piv = nullptr;
  d.params = g->params;
  if (cudaMallocHost(&g->h_pin, 64 * sizeof(double)) != cudaSuccess) return CS_ERR_OOM;
  if (cudaMallocHost(&g->h_status, 4 * sizeof(int)) != cudaSuccess) return CS_ERR_OOM;
  for (int k = 0; k < nd; ++k)
    if (cudaMemcpyAsync(g->node[k], nodes_host + k * nn, nn * sizeof(double),
                        cudaMemcpyHostToDevice, g->stream) != cudaSuccess)
      return CS_ERR_CUDA;
  GeomArgs ga;
  ga.nd = nd;
  ga.ni = d.ni;
  ga.nj = d.nj;
  ga.nk = d.nk;
  for (int k = 0; k < 3; ++k) {
    ga.node[k] = g->node[k];
    ga.S[k] = const_cast<double*>(d.S[k]);
    ga.fc[k] = const_cast<double*>(d.fc[k]);
    ga.nf[k] = d.nf[k];
  }
  ga.V = V;
  ga.xc = xc;
  for (int k = 0; k < nd; ++k) k_geom_faces<<<Launcher::blocks(d.nf[k], 128), 128, 0, g->stream>>>(ga, k);
  k_geom_cells<<<Launcher::blocks(N, 128), 128, 0, g->stream>>>(ga);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(g->stream) != cudaSuccess)
    return CS_ERR_CUDA;
  make_side(g);
  *out = G.release();
  return CS_OK;
}

extern "C" cs_status cs_grid_destroy(cs_grid g) {
  if (!g) return CS_ERR_ARG;
  cudaStreamSynchronize(g->stream);
  if (g->side) {
    cudaStreamSynchronize(g->side);
    cudaStreamDestroy(g->side);
  }
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_join) cudaEventDestroy(g->ev_join);
  for (void* p : g->allocs) cudaFree(p);
  if (g->g.DLU) cudaFree(g->g.DLU);
  if (g->g.DINV) cudaFree(g->g.DINV);
  if (g->g.CIM) cudaFree(g->g.CIM);
  if (g->g.piv) cudaFree(g->g.piv);
  if (g->h_pin) cudaFreeHost(g->h_pin);
  if (g->h_status) cudaFreeHost(g->h_status);
  delete g;
  return CS_OK;
}

extern "C" cs_status cs_grid_dims(cs_grid g, int out[8]) {
  if (!g || !out) return CS_ERR_ARG;
  const Launcher* L = g->L.get();
  out[0] = g->g.N;
  out[1] = L->nq;
  out[2] = L->nF + L->ns;
  out[3] = L->nci;
  out[4] = L->ns;
  out[5] = L->ntemp;
  out[6] = L->nF;
  out[7] = g->stag;
  return CS_OK;
}

extern "C" cs_status cs_set_boundary(cs_grid g, const cs_freestream* fs, const cs_wall* wall) {
  if (!g || !fs || !wall) return CS_ERR_ARG;
  if (wall->catalytic != 0) return fail(g, CS_ERR_ARG, "only non-catalytic walls");
  const int ns = g->L->ns;
  double* h = g->h_pin;
  h[0] = fs->T;
  h[1] = fs->Tv;
  h[2] = fs->p;
  h[3] = fs->mach;
  for (int q = 0; q < 3; ++q) h[4 + q] = fs->dir[q];
  for (int s = 0; s < ns; ++s) h[7 + s] = fs->Y[s];
  cs_status st = begin(g);
  if (st) return st;
  CUDA_TRY(g, cudaMemcpyAsync(g->fsin, h, (7 + ns) * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  g->g.Tw = wall->Tw;
  g->L->freestream(g->g, g->stream, g->fsin, g->fsQ);
  if (g->g.bc[2] == CS_BC_WALL) {
    k_stagnation<<<1, 256, 0, g->stream>>>(g->g.S[1], g->g.ni, g->g.nj, g->g.nk, g->g.nd,
                                            fs->dir[0], fs->dir[1], fs->dir[2], g->stag_dev);
    CUDA_TRY(g, cudaMemcpyAsync(&g->h_status[3], g->stag_dev, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  } else {
    g->h_status[3] = -1;
  }
  CUDA_TRY(g, cudaStreamSynchronize(g->stream));
  g->stag = g->h_status[3];
  st = finish(g, "cs_set_boundary");
  if (st) return st;
  g->have_bc = 1;
  return CS_OK;
}

static void reset_warm_start(cs_grid g) {
  // temperatures of the auxiliary array are the Newton warm starts: 0 = none
  int cnt;
  const int oT = g->L->aux_field("T", &cnt), oTv = g->L->aux_field("Tv", &cnt);
  cudaMemsetAsync(g->g.W + (size_t)oT * g->g.N, 0, g->g.N * sizeof(double), g->stream);
  cudaMemsetAsync(g->g.W + (size_t)oTv * g->g.N, 0, g->g.N * sizeof(double), g->stream);
}

extern "C" cs_status cs_set_state(cs_grid g, const double* Q) {
  if (!g || !Q) return CS_ERR_ARG;
  CUDA_TRY(g, cudaMemcpyAsync(g->g.Q, Q, (size_t)g->L->nq * g->g.N * sizeof(double),
                              cudaMemcpyDefault, g->stream));
  reset_warm_start(g);
  CUDA_TRY(g, cudaStreamSynchronize(g->stream));
  g->have_R = 0;
  g->iter = 0;
  return CS_OK;
}

extern "C" cs_status cs_load_state(cs_grid g, const double* Q) {
  if (!g || !Q) return CS_ERR_ARG;
  CUDA_TRY(g, cudaMemcpyAsync(g->g.Q, Q, (size_t)g->L->nq * g->g.N * sizeof(double),
                              cudaMemcpyDefault, g->stream));
  g->have_R = 0;
  return CS_OK;
}

extern "C" cs_status cs_init_freestream(cs_grid g) {
  if (!g) return CS_ERR_ARG;
  if (!g->have_bc) return fail(g, CS_ERR_STATE, "cs_init_freestream before cs_set_boundary");
  g->L->fill(g->g, g->stream, g->fsQ);
  reset_warm_start(g);
  CUDA_TRY(g, cudaGetLastError());
  CUDA_TRY(g, cudaStreamSynchronize(g->stream));
  g->have_R = 0;
  g->iter = 0;
  return CS_OK;
}

extern "C" cs_status cs_get_state(cs_grid g, double* Q_out) {
  if (!g || !Q_out) return CS_ERR_ARG;
  CUDA_TRY(g, cudaMemcpyAsync(Q_out, g->g.Q, (size_t)g->L->nq * g->g.N * sizeof(double),
                              cudaMemcpyDefault, g->stream));
  CUDA_TRY(g, cudaStreamSynchronize(g->stream));
  return CS_OK;
}

// enqueue the residual (no synchronisation)
// the species Jacobian diagonal of the operator from the attached network (after primitives)
static void enqueue_surrogate(cs_grid g) {
  if (!g->surr) return;
  g->L->surr_features(g->g, g->stream, g->sx, g->snorm);
  mlp_forward_on(g->surr, g->sx, g->g.N, g->sy, g->stream);
  g->L->surr_decode(g->g, g->stream, g->sy, g->snorm);
}

static void enqueue_residual(cs_grid g) {
  g->L->residual(g->g, g->stream, g->stag, g->norms);
  enqueue_surrogate(g);
}

extern "C" cs_status cs_residual(cs_grid g, double* R_out, double norms_host[3]) {
  if (!g) return CS_ERR_ARG;
  if (!g->have_bc) return fail(g, CS_ERR_STATE, "cs_residual before cs_set_boundary");
  cs_status st = begin(g);
  if (st) return st;
  enqueue_residual(g);
  if (R_out)
    CUDA_TRY(g, cudaMemcpyAsync(R_out, g->g.R, (size_t)g->L->nq * g->g.N * sizeof(double),
                                cudaMemcpyDefault, g->stream));
  CUDA_TRY(g, cudaMemcpyAsync(g->h_pin + 32, g->norms, 3 * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  st = finish(g, "cs_residual");
  if (st) return st;
  if (norms_host)
    for (int k = 0; k < 3; ++k) norms_host[k] = g->h_pin[32 + k];
  g->have_R = 1;
  return CS_OK;
}

// coupling records of the 2D split sweep over assembled couplings (K6e; FP64 or FP32 records in
// the same buffer), allocated only when a sweep of this precision will read them; without them
// (allocation refused) the sweep falls back to the other cluster kernels
static void ensure_mat(cs_grid g, bool mixed) {
  if (g->g.SMC || g->mat_refused) return;
  if (!g->L->mat_usable(g->g, mixed)) return;   // not sticky: another precision may use them
  const size_t n = g->L->mat_doubles(g->g);
  if (n == 0 || dalloc(g, &g->g.SMC, n) != cudaSuccess) {
    cudaGetLastError();
    g->g.SMC = nullptr;
    g->mat_refused = true;
  }
}

static cs_status set_cfl(cs_grid g, double cfl) {
  if (!(cfl > 0.0)) return fail(g, CS_ERR_ARG, "cfl must be positive");
  g->h_pin[40] = cfl;
  CUDA_TRY(g, cudaMemcpyAsync(g->params, g->h_pin + 40, sizeof(double), cudaMemcpyHostToDevice, g->stream));
  return CS_OK;
}

extern "C" cs_status cs_lusgs_split(cs_grid g, double cfl, int precision, double* dQ_out) {
  if (!g) return CS_ERR_ARG;
  if (precision != CS_FP64 && precision != CS_MIXED)
    return fail(g, CS_ERR_ARG, "unsupported precision %d", precision);
  if (!g->have_R) return fail(g, CS_ERR_STATE, "cs_lusgs_split before cs_residual");
  cs_status st = begin(g);
  if (st) return st;
  if ((st = set_cfl(g, cfl))) return st;
  ensure_mat(g, precision == CS_MIXED);
  g->L->spectral(g->g, g->stream);
  g->L->sweep_split(g->g, g->stream, precision == CS_MIXED);
  if (dQ_out)
    CUDA_TRY(g, cudaMemcpyAsync(dQ_out, g->g.dQ, (size_t)(g->L->nF + g->L->ns) * g->g.N * sizeof(double),
                                cudaMemcpyDefault, g->stream));
  st = finish(g, "cs_lusgs_split");
  if (st) return st;
  g->last_op = 0;
  return CS_OK;
}

static cs_status ensure_ci(cs_grid g) {
  if (g->g.DLU) return CS_OK;
  const size_t nc = g->L->nci;
  void *a = nullptr, *b = nullptr, *v = nullptr;
  if (cudaMalloc(&a, nc * nc * (size_t)g->g.N * sizeof(double)) != cudaSuccess) return CS_ERR_OOM;
  if (cudaMalloc(&b, nc * (size_t)g->g.N * sizeof(int)) != cudaSuccess) { cudaFree(a); return CS_ERR_OOM; }
  if (cudaMalloc(&v, nc * nc * (size_t)g->g.N * sizeof(double)) != cudaSuccess) {
    cudaFree(a);
    cudaFree(b);
    return CS_ERR_OOM;
  }
  g->g.DLU = (double*)a;
  g->g.piv = (int*)b;
  g->g.DINV = (double*)v;
  // 2D: the neighbour blocks of the assembled coupled sweep (without them, the one-lane-per-row
  // cluster sweep runs)
  const size_t nm = g->L->ci_mat_doubles(g->g);
  void* m = nullptr;
  if (nm > 0 && cudaMalloc(&m, nm * sizeof(double)) == cudaSuccess) g->g.CIM = (double*)m;
  else cudaGetLastError();
  return CS_OK;
}

extern "C" cs_status cs_lusgs_coupled(cs_grid g, double cfl, double* dQ_out) {
  if (!g) return CS_ERR_ARG;
  if (!g->have_R) return fail(g, CS_ERR_STATE, "cs_lusgs_coupled before cs_residual");
  cs_status st = ensure_ci(g);
  if (st) return fail(g, st, "coupled block allocation failed");
  if ((st = begin(g))) return st;
  if ((st = set_cfl(g, cfl))) return st;
  g->L->spectral(g->g, g->stream);
  g->L->ci_block(g->g, g->stream);
  g->L->sweep_coupled(g->g, g->stream);
  if (dQ_out)
    CUDA_TRY(g, cudaMemcpyAsync(dQ_out, g->g.dQc, (size_t)g->L->nci * g->g.N * sizeof(double),
                                cudaMemcpyDefault, g->stream));
  st = finish(g, "cs_lusgs_coupled");
  if (st) return st;
  g->last_op = 1;
  return CS_OK;
}

extern "C" cs_status cs_correct(cs_grid g, int mode, int clip, const double* dQ, int* nclip_out) {
  if (!g) return CS_ERR_ARG;
  if (mode < 0 || mode > 2) return fail(g, CS_ERR_ARG, "correction mode %d", mode);
  const double* src;
  const size_t n = (size_t)(mode == 0 ? g->L->nci : g->L->nF + g->L->ns) * g->g.N;
  cs_status st = begin(g);
  if (st) return st;
  if (dQ) {
    // caller's increments are copied into the matching internal buffer first
    double* dst = mode == 0 ? g->g.dQc : g->g.dQ;
    CUDA_TRY(g, cudaMemcpyAsync(dst, dQ, n * sizeof(double), cudaMemcpyDefault, g->stream));
    src = dst;
  } else {
    if ((mode == 0 && g->last_op != 1) || (mode != 0 && g->last_op != 0))
      return fail(g, CS_ERR_STATE, "cs_correct: no increments of the matching operator");
    src = mode == 0 ? g->g.dQc : g->g.dQ;
  }
  g->L->correct(g->g, g->stream, mode, clip, src);
  st = finish(g, "cs_correct");
  if (nclip_out) *nclip_out = g->h_status[2];
  if (st) return st;
  g->have_R = 0;
  return CS_OK;
}

// CFL of the current iteration computed on the device (the geometric ramp of cs_step from a
// device iteration counter), so that a captured iteration replays with the right CFL.
__global__ void k_cfl(double* params, int* iter, double cfl, double cfl_start, int ramp) {
  const int it = *iter;
  double c = cfl;
  if (ramp > 0 && it < ramp && cfl_start > 0.0) c = cfl_start * pow(cfl / cfl_start, (double)it / (double)ramp);
  params[0] = c;
  *iter = it + 1;
}
__global__ void k_set_int(int* p, int v) { *p = v; }

static cs_status check_opts(const cs_step_opts* o) {
  if (!o) return CS_ERR_ARG;
  if (o->scheme != CS_SCHEME_SPLIT && o->scheme != CS_SCHEME_COUPLED) return CS_ERR_ARG;
  if (o->scheme == CS_SCHEME_SPLIT && o->correction != 1 && o->correction != 2) return CS_ERR_ARG;
  if ((o->precision != CS_FP64 && o->precision != CS_MIXED) || o->iters < 0) return CS_ERR_ARG;
  if (!(o->cfl > 0.0)) return CS_ERR_ARG;
  return CS_OK;
}

// The chemistry of an iteration (k_chem: source, Jacobian diagonal, relaxation) reads only the
// state and the primitives and is read first by the assembly, so it runs on a second stream
// beside the gradient and flux kernels (which fill the SMs its last wave of CTAs leaves idle).
// Returns false (the caller then runs it in order) if the stream or events cannot be made.
static void make_side(cs_grid g) {   // at grid creation (not during a stream capture)
  if (cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (g->side) cudaStreamDestroy(g->side);
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    g->side = nullptr;
    g->ev_fork = g->ev_join = nullptr;
  }
}
static bool fork_chem(cs_grid g) {
  if (!g->side) return false;
  if (cudaEventRecord(g->ev_fork, g->stream) != cudaSuccess ||
      cudaStreamWaitEvent(g->side, g->ev_fork, 0) != cudaSuccess)
    return false;
  g->L->chem(g->g, g->side);
  return cudaEventRecord(g->ev_join, g->side) == cudaSuccess;
}

// Enqueue one pseudo-time iteration on g->stream (no host synchronisation).  device_cfl: the
// CFL comes from k_cfl and the device iteration counter and no profiling events are recorded
// (stream capture); otherwise the CFL of iteration g->iter is copied from pinned memory slot
// `slot`.  *nf / *nb receive the forward / backward sweep launch counts.
static cs_status enqueue_iteration(cs_grid g, const cs_step_opts* o, int slot, bool device_cfl,
                                   int* nf_out, int* nb_out) {
  const bool mixed = o->precision == CS_MIXED;
  CUDA_TRY(g, cudaMemsetAsync(&g->g.status[2], 0, sizeof(int), g->stream));
  if (device_cfl) {
    k_cfl<<<1, 1, 0, g->stream>>>(g->params, g->iter_dev, o->cfl, o->cfl_start, o->ramp_iters);
  } else {
    double cfl = o->cfl;
    if (o->ramp_iters > 0 && g->iter < o->ramp_iters && o->cfl_start > 0.0)
      cfl = o->cfl_start * pow(o->cfl / o->cfl_start, (double)g->iter / (double)o->ramp_iters);
    g->h_pin[41 + slot] = cfl;
    CUDA_TRY(g, cudaMemcpyAsync(g->params, g->h_pin + 41 + slot, sizeof(double),
                                cudaMemcpyHostToDevice, g->stream));
  }
  const bool rec = !device_cfl;
  const DevGrid& d = g->g;
  if (rec) prof_record(g, slot, 0);
  g->L->primitive_state(d, g->stream);
  const bool side = fork_chem(g);
  if (!side) g->L->chem(d, g->stream);
  if (rec) prof_record(g, slot, 1);
  g->L->gradient(d, g->stream);
  if (rec) prof_record(g, slot, 2);
  g->L->flux(d, g->stream);
  // join: the assembly reads the chemistry (the flux phase ends when both are done)
  if (side) CUDA_TRY(g, cudaStreamWaitEvent(g->stream, g->ev_join, 0));
  if (rec) prof_record(g, slot, 3);
  g->L->assemble(d, g->stream, g->stag, g->norms);
  if (rec) prof_record(g, slot, 4);
  // the species Jacobian diagonal of the operator from the network, when one is attached (the
  // exact source stays in the residual); timed with the spectral phase
  enqueue_surrogate(g);
  g->L->spectral(d, g->stream);
  int nf, nb;
  if (o->scheme == CS_SCHEME_SPLIT) {
    if (rec) prof_record(g, slot, 5);
    // the cluster path runs both sweeps in one launch (timed as phase 5)
    nf = g->L->use_cluster ? g->L->sweep_split_cluster(d, g->stream, mixed) : 0;
    nb = 0;
    if (!nf) nf = g->L->sweep_split_dir(d, g->stream, true, mixed);
    if (rec) prof_record(g, slot, 6);
    if (!g->L->use_cluster || !g->L->sweep_split_cluster_ok) nb = g->L->sweep_split_dir(d, g->stream, false, mixed);
    if (rec) prof_record(g, slot, 7);
    g->L->correct(d, g->stream, o->correction, o->clip, d.dQ);
  } else {
    g->L->ci_block(d, g->stream);
    if (rec) prof_record(g, slot, 5);
    // both sweeps in one cluster launch where it applies (2D), else one launch per hyperplane
    const int nc = g->L->use_cluster ? g->L->sweep_coupled_cluster(d, g->stream) : 0;
    const bool one = nc > 0;
    nf = one ? nc : g->L->sweep_coupled_dir(d, g->stream, true);
    if (rec) prof_record(g, slot, 6);
    nb = one ? 0 : g->L->sweep_coupled_dir(d, g->stream, false);
    if (rec) prof_record(g, slot, 7);
    g->L->correct(d, g->stream, 0, o->clip, d.dQc);
  }
  if (rec) prof_record(g, slot, 8);
  CUDA_TRY(g, cudaGetLastError());
  *nf_out = nf;
  *nb_out = nb;
  return CS_OK;
}

extern "C" cs_status cs_step(cs_grid g, const cs_step_opts* o, cs_step_stats* stats) {
  if (!g || !o) return CS_ERR_ARG;
  if (!g->have_bc) return fail(g, CS_ERR_STATE, "cs_step before cs_set_boundary");
  cs_status st = check_opts(o);
  if (st) return st;
  if (o->scheme == CS_SCHEME_COUPLED && (st = ensure_ci(g))) return fail(g, st, "allocation");
  if (o->scheme == CS_SCHEME_SPLIT) ensure_mat(g, o->precision == CS_MIXED);
  if ((st = begin(g))) return st;
  int done = 0;
  for (int it = 0; it < o->iters; ++it) {
    const int slot = it & 7;
    int nf, nb;
    if ((st = enqueue_iteration(g, o, slot, false, &nf, &nb))) return st;
    if (g->prof) {
      const long per[CS_NPHASE] = {2L + g->g.transport, 1, (long)g->g.nd, 2, o->scheme == CS_SCHEME_SPLIT ? 1 : 2, nf, nb, 1};
      for (int p = 0; p < CS_NPHASE; ++p) g->prof_launches[p] += per[p];
      g->ev_used = slot + 1;
    }
    g->iter++;
    done++;
    // detect device errors every 8 iterations without stalling every step
    if (slot == 7 || it == o->iters - 1) {
      CUDA_TRY(g, cudaMemcpyAsync(g->h_status, g->g.status, 4 * sizeof(int), cudaMemcpyDeviceToHost, g->stream));
      CUDA_TRY(g, cudaStreamSynchronize(g->stream));
      prof_resolve(g);
      if (g->h_status[0] != 0) break;
    }
  }
  CUDA_TRY(g, cudaMemcpyAsync(g->h_pin + 32, g->norms, 3 * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  st = finish(g, "cs_step");
  if (stats) {
    stats->iters_done = done;
    stats->r_species = g->h_pin[32];
    stats->r_energy = g->h_pin[33];
    stats->q_stag = g->h_pin[34];
    stats->nclip = g->h_status[2];
    stats->status_cell = st ? g->h_status[1] : -1;
  }
  g->have_R = 0;
  return st;
}

extern "C" cs_status cs_get_field(cs_grid g, const char* name, double* out, int* count_out) {
  if (!g || !name || !out) return CS_ERR_ARG;
  const size_t N = g->g.N;
  const double* src = nullptr;
  size_t n = 0;
  int cnt = 0;
  const int off = g->L->aux_field(name, &cnt);
  if (off >= 0) { src = g->g.W + (size_t)off * N; n = cnt * N; }
  else if (!strcmp(name, "lamF")) { src = g->g.lamF; n = g->L->nd * N; }
  else if (!strcmp(name, "lamC")) { src = g->g.lamC; n = g->L->nd * N; }
  else if (!strcmp(name, "lamCI")) { src = g->g.lamCI; n = g->L->nd * N; }
  else if (!strcmp(name, "DF")) { src = g->g.DF; n = N; }
  else if (!strcmp(name, "DFev")) { src = g->g.DFev; n = N; }
  else if (!strcmp(name, "Ds")) { src = g->g.Ds; n = g->L->ns * N; }
  else if (!strcmp(name, "V")) { src = g->g.V; n = N; }
  else if (!strcmp(name, "xc")) { src = g->g.xc; n = 3 * N; }
  else if (!strcmp(name, "grad")) { src = g->g.grad; n = (size_t)g->L->ng * 3 * N; }
  else if (!strcmp(name, "dQstar")) { src = g->g.dQs; n = (size_t)(g->L->nF + g->L->ns) * N; }
  else if (!strcmp(name, "S0") || !strcmp(name, "S1") || !strcmp(name, "S2")) {
    const int d = name[1] - '0';
    if (d >= g->L->nd) return fail(g, CS_ERR_ARG, "no field %s", name);
    src = g->g.S[d]; n = 3 * (size_t)g->g.nf[d];
  } else if (!strcmp(name, "F0") || !strcmp(name, "F1") || !strcmp(name, "F2")) {
    const int d = name[1] - '0';
    if (d >= g->L->nd) return fail(g, CS_ERR_ARG, "no field %s", name);
    src = g->g.F[d]; n = (size_t)g->L->nq * g->g.nf[d];
  } else {
    return fail(g, CS_ERR_ARG, "unknown field %s", name);
  }
  CUDA_TRY(g, cudaMemcpyAsync(out, src, n * sizeof(double), cudaMemcpyDefault, g->stream));
  CUDA_TRY(g, cudaStreamSynchronize(g->stream));
  if (count_out) *count_out = (int)n;
  return CS_OK;
}

extern "C" cs_status cs_set_option(cs_grid g, const char* name, double value) {
  if (!g || !name) return CS_ERR_ARG;
  if (!strcmp(name, "cluster_sweep")) {
    // 0 per hyperplane, 1 direct-load cluster kernel, 2 record cluster kernel, 3 default (by
    // precision), 4 one CTA per component (FP32 operator only; the others fall back to 2),
    // 5 assembled couplings exchanged point to point between CTAs where the ring fits (else
    // FP64: 6 then 1, FP32: 4 then 2), 6 the same FP64 couplings with a cluster barrier per
    // hyperplane (the FP32 operator falls back to 4 then 2); 7 (a retired systolic-warp form)
    // runs as 5
    g->L->use_cluster = value != 0.0;
    g->L->cluster_kind = value >= 6.0 && value < 7.0 ? 5 : value >= 5.0 ? 4 : value >= 4.0 ? 3 : (value >= 3.0 ? 0 : (value >= 2.0 ? 2 : 1));
    return CS_OK;
  }
  if (!strcmp(name, "cluster_size")) {
    const int C = (int)value;
    if ((double)C != value || (C != 0 && C != 1 && C != 2 && C != 4 && C != 8 && C != 16))
      return fail(g, CS_ERR_ARG, "cluster_size must be 0, 1, 2, 4, 8 or 16");
    // the probes set the kernels' non-portable cluster attribute where it is needed
    for (int kind : {1, 2})
      for (bool mixed : {false, true}) g->L->cluster_sizes(g->g, kind, mixed);
    g->L->force_C = C;
    return CS_OK;
  }
  if (!strcmp(name, "update_limit")) {
    if (!(value >= 0.0)) return fail(g, CS_ERR_ARG, "update_limit must be >= 0");
    g->g.ulim = value;
    return CS_OK;
  }
  if (!strcmp(name, "h_correction")) {
    g->g.hcorr = value != 0.0;
    return CS_OK;
  }
  if (!strcmp(name, "ci_splitting")) {
    if (value != 0.0 && value != 1.0) return fail(g, CS_ERR_ARG, "ci_splitting must be 0 or 1");
    g->g.cisplit = (int)value;
    return CS_OK;
  }
  if (!strcmp(name, "dtau_source")) {
    if (value != 0.0 && value != 1.0) return fail(g, CS_ERR_ARG, "dtau_source must be 0 or 1");
    g->g.dtau_src = (int)value;
    return CS_OK;
  }
  if (!strcmp(name, "transport")) {
    if (value != 0.0 && value != 1.0) return fail(g, CS_ERR_ARG, "transport must be 0 or 1");
    if (value == 1.0 && g->L->ns < 5) return fail(g, CS_ERR_ARG, "the species transport model needs an air mixture");
    g->g.transport = (int)value;
    g->have_R = 0;
    return CS_OK;
  }
  return fail(g, CS_ERR_ARG, "unknown option %s", name);
}

// Dual time stepping (Sec. 2.3): the coefficients (1+theta)/dt and theta/dt live in device
// memory (params[1], params[2]) so that captured iterations read the current values; theta
// takes effect from the second physical step on (the first has no Q^{n-1}).
__global__ void k_set_dual(double* params, double a, double b) {
  params[1] = a;
  params[2] = b;
}

static cs_status upload_dual(cs_grid g) {
  double a = 0.0, b = 0.0;
  if (g->dual_dt > 0.0 && g->dual_levels >= 1) {
    const double th = g->dual_levels >= 2 ? g->dual_theta : 0.0;
    a = (1.0 + th) / g->dual_dt;
    b = th / g->dual_dt;
  }
  k_set_dual<<<1, 1, 0, g->stream>>>(g->params, a, b);
  CUDA_TRY(g, cudaGetLastError());
  g->have_R = 0;
  return CS_OK;
}

extern "C" cs_status cs_set_dual(cs_grid g, double dt, double theta) {
  if (!g) return CS_ERR_ARG;
  if (!(dt >= 0.0) || !(theta >= 0.0) || !std::isfinite(dt) || !std::isfinite(theta))
    return fail(g, CS_ERR_ARG, "dual time step %g and theta %g must be finite and >= 0", dt, theta);
  if (dt > 0.0 && !g->g.Qn) {
    const size_t n = (size_t)g->L->nq * g->g.N;
    double *a = nullptr, *b = nullptr;
    if (dalloc(g, &a, n) != cudaSuccess || dalloc(g, &b, n) != cudaSuccess)
      return fail(g, CS_ERR_OOM, "dual time levels");
    g->g.Qn = a;
    g->g.Qnm1 = b;
  }
  g->dual_dt = dt;
  g->dual_theta = theta;
  g->dual_levels = 0;
  return upload_dual(g);
}

extern "C" cs_status cs_dual_advance(cs_grid g) {
  if (!g) return CS_ERR_ARG;
  if (!(g->dual_dt > 0.0) || !g->g.Qn) return fail(g, CS_ERR_STATE, "dual time stepping is off");
  const size_t bytes = (size_t)g->L->nq * g->g.N * sizeof(double);
  CUDA_TRY(g, cudaMemcpyAsync(const_cast<double*>(g->g.Qnm1), g->g.Qn, bytes, cudaMemcpyDeviceToDevice, g->stream));
  CUDA_TRY(g, cudaMemcpyAsync(const_cast<double*>(g->g.Qn), g->g.Q, bytes, cudaMemcpyDeviceToDevice, g->stream));
  if (g->dual_levels < 2) ++g->dual_levels;
  return upload_dual(g);
}

extern "C" const char* cs_last_error(cs_grid g) { return g ? g->err : "null grid"; }

// ---------------------------------------------------------------------------------------
// Batches of independent cases (many grids stepped together): K iterations of every case are
// captured once into one CUDA graph, each case on its own stream between a fork and a join
// event, and the graph is replayed; one graph launch then issues K iterations of all cases,
// which run concurrently on the GPU.  Per-case CFL ramps are evaluated on the device.  The
// tuner times each case's split sweep over the cluster sizes and the two cluster kernels.
// ---------------------------------------------------------------------------------------
struct cs_batch_s {
  std::vector<cs_grid> grids;
  std::vector<cudaStream_t> streams;   // one per case (library-owned, non-blocking)
  std::vector<cudaEvent_t> ready, join;
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cs_step_opts> key;       // options the graph was captured with
  std::vector<cs_mlp> key_surr;        // and the networks attached then
  std::vector<const double*> key_dual; // and the dual-time level buffers then
  std::vector<int> key_split;          // and the coupled operator's splitting then
  int key_k = 0;
  char err[512] = {0};
};

static cs_status bfail(cs_batch b, cs_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b->err, sizeof b->err, fmt, ap);
  va_end(ap);
  return st;
}
#define BCUDA_TRY(b, call)                                                                  \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return bfail(b, CS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static void batch_release(cs_batch b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto e : b->ready) cudaEventDestroy(e);
  for (auto e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
}

extern "C" cs_status cs_batch_create(int ncases, const cs_grid* grids, cs_batch* out) {
  if (!out || !grids || ncases < 1) return CS_ERR_ARG;
  *out = nullptr;
  for (int c = 0; c < ncases; ++c)
    if (!grids[c] || !grids[c]->have_bc) return CS_ERR_ARG;
  std::unique_ptr<cs_batch_s> b(new cs_batch_s);
  b->grids.assign(grids, grids + ncases);
  auto cleanup = [&](cs_status st) {
    batch_release(b.get());
    b->streams.clear(); b->ready.clear(); b->join.clear();
    b->fork = nullptr; b->origin = nullptr;
    return st;
  };
  if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(CS_ERR_CUDA);
  for (int c = 0; c < ncases; ++c) {
    cudaStream_t s;
    cudaEvent_t e1, e2;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return cleanup(CS_ERR_CUDA);
    b->streams.push_back(s);
    if (cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess) return cleanup(CS_ERR_CUDA);
    b->ready.push_back(e1);
    if (cudaEventCreateWithFlags(&e2, cudaEventDisableTiming) != cudaSuccess) return cleanup(CS_ERR_CUDA);
    b->join.push_back(e2);
  }
  *out = b.release();
  return CS_OK;
}

extern "C" cs_status cs_batch_destroy(cs_batch b) {
  if (!b) return CS_ERR_ARG;
  cudaStreamSynchronize(b->origin);
  batch_release(b);
  delete b;
  return CS_OK;
}

// run fn with every grid's stream replaced by its batch stream (restored afterwards)
template <class F>
static cs_status with_batch_streams(cs_batch b, F fn) {
  const int n = (int)b->grids.size();
  std::vector<cudaStream_t> saved(n);
  std::vector<int> warps(n);
  for (int c = 0; c < n; ++c) {
    // work the caller queued on the grid's own stream comes first
    BCUDA_TRY(b, cudaStreamSynchronize(b->grids[c]->stream));
    saved[c] = b->grids[c]->stream;
    b->grids[c]->stream = b->streams[c];
    // many grids share the GPU: the one-warp form of the cluster sweep keeps twice as many
    // CTAs resident
    warps[c] = b->grids[c]->L->cluster_warps;
    b->grids[c]->L->cluster_warps = 1;
  }
  const cs_status st = fn();
  for (int c = 0; c < n; ++c) {
    cudaStreamSynchronize(b->streams[c]);
    b->grids[c]->stream = saved[c];
    b->grids[c]->L->cluster_warps = warps[c];
  }
  return st;
}

extern "C" cs_status cs_batch_tune(cs_batch b, int precision, int trials, int* choice_out) {
  if (!b || (precision != CS_FP64 && precision != CS_MIXED) || trials < 1) return CS_ERR_ARG;
  const bool mixed = precision == CS_MIXED;
  return with_batch_streams(b, [&]() -> cs_status {
    cudaEvent_t e0, e1;
    BCUDA_TRY(b, cudaEventCreate(&e0));
    BCUDA_TRY(b, cudaEventCreate(&e1));
    cs_status result = CS_OK;
    for (size_t c = 0; c < b->grids.size() && !result; ++c) {
      cs_grid g = b->grids[c];
      Launcher* L = g->L.get();
      const DevGrid& d = g->g;
      // operator inputs of the current state (no update: the state does not change)
      g->h_pin[40] = 1.0;
      if (cudaMemcpyAsync(g->params, g->h_pin + 40, sizeof(double), cudaMemcpyHostToDevice, g->stream) != cudaSuccess ||
          begin(g)) { result = bfail(b, CS_ERR_CUDA, "case %zu: setup", c); break; }
      L->residual(d, g->stream, g->stag, g->norms);
      L->spectral(d, g->stream);
      float best = 1e30f;
      int best_kind = 0, best_C = 0;
      const int keep_kind = L->cluster_kind, keep_C = L->force_C;
      for (int kind : {1, 2, 3}) {
        // kind 3 (one CTA per component, FP32 only) has no cluster size: timed once as C = 1
        const int mask = kind == 3 ? (mixed && L->block_available(d) ? 2 : 0) : L->cluster_sizes(d, kind, mixed);
        for (int C : {1, 2, 4, 8, 16}) {
          if (!(mask & (1 << C))) continue;
          L->cluster_kind = kind;
          L->force_C = C;
          L->sweep_split_cluster(d, g->stream, mixed);      // warm
          cudaEventRecord(e0, g->stream);
          for (int t = 0; t < trials; ++t) L->sweep_split_cluster(d, g->stream, mixed);
          cudaEventRecord(e1, g->stream);
          if (cudaEventSynchronize(e1) != cudaSuccess) { result = bfail(b, CS_ERR_CUDA, "case %zu: timing", c); break; }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          // prefer fewer CTAs unless the larger cluster is > 3 % faster
          if (ms < 0.97f * best || (ms < best && C < best_C)) { best = ms; best_kind = kind; best_C = C; }
        }
        if (result) break;
      }
      if (result) break;
      if (best_C) {
        L->cluster_kind = best_kind;
        L->force_C = best_C;
      } else {
        L->cluster_kind = keep_kind;
        L->force_C = keep_C;
      }
      if (choice_out) {
        choice_out[2 * c] = best_kind;
        choice_out[2 * c + 1] = best_C;
      }
      if (finish(g, "cs_batch_tune")) result = bfail(b, CS_ERR_CUDA, "case %zu: %s", c, g->err);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (b->exec) {   // the captured graph used the old choices
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
      b->key.clear();
    }
    return result;
  });
}

static bool same_opts(const cs_step_opts& a, const cs_step_opts& b) {
  return a.scheme == b.scheme && a.correction == b.correction && a.clip == b.clip && a.cfl == b.cfl &&
         a.cfl_start == b.cfl_start && a.ramp_iters == b.ramp_iters && a.precision == b.precision;
}

extern "C" cs_status cs_batch_step(cs_batch b, const cs_step_opts* opts, int iters, int iters_per_graph,
                                   cs_step_stats* stats) {
  if (!b || !opts || iters < 0 || iters_per_graph < 1 || iters % iters_per_graph) return CS_ERR_ARG;
  const int n = (int)b->grids.size();
  for (int c = 0; c < n; ++c)
    if (check_opts(&opts[c])) return bfail(b, CS_ERR_ARG, "case %d: invalid options", c);
  if (iters == 0) return CS_OK;
  return with_batch_streams(b, [&]() -> cs_status {
    for (int c = 0; c < n; ++c) {
      cs_grid g = b->grids[c];
      if (opts[c].scheme == CS_SCHEME_COUPLED && ensure_ci(g)) return bfail(b, CS_ERR_OOM, "case %d: allocation", c);
      g->L->prepare(g->g, opts[c].precision == CS_MIXED);
    }
    bool recapture = !b->exec || b->key_k != iters_per_graph || (int)b->key.size() != n;
    for (int c = 0; c < n && !recapture; ++c)
      recapture = !same_opts(b->key[c], opts[c]) || b->key_surr[c] != b->grids[c]->surr ||
                  b->key_dual[c] != b->grids[c]->g.Qn || b->key_split[c] != b->grids[c]->g.cisplit;
    if (recapture) {
      if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
      BCUDA_TRY(b, cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
      cs_status st = CS_OK;
      if (cudaEventRecord(b->fork, b->origin) != cudaSuccess) st = CS_ERR_CUDA;
      for (int c = 0; c < n && !st; ++c)
        if (cudaStreamWaitEvent(b->streams[c], b->fork, 0) != cudaSuccess) st = CS_ERR_CUDA;
      for (int c = 0; c < n && !st; ++c) {
        for (int k = 0; k < iters_per_graph && !st; ++k) {
          int nf, nb;
          st = enqueue_iteration(b->grids[c], &opts[c], 0, true, &nf, &nb);
          if (st) bfail(b, st, "case %d: capture: %s", c, b->grids[c]->err);
        }
        if (!st && (cudaEventRecord(b->join[c], b->streams[c]) != cudaSuccess ||
                    cudaStreamWaitEvent(b->origin, b->join[c], 0) != cudaSuccess))
          st = CS_ERR_CUDA;
      }
      cudaGraph_t graph = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(b->origin, &graph);
      if (st || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return st ? st : bfail(b, CS_ERR_CUDA, "stream capture: %s", cudaGetErrorString(ee));
      }
      const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess) { b->exec = nullptr; return bfail(b, CS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ei)); }
      b->key.assign(opts, opts + n);
      b->key_surr.clear();
      for (int c = 0; c < n; ++c) b->key_surr.push_back(b->grids[c]->surr);
      b->key_dual.clear();
      for (int c = 0; c < n; ++c) b->key_dual.push_back(b->grids[c]->g.Qn);
      b->key_split.clear();
      for (int c = 0; c < n; ++c) b->key_split.push_back(b->grids[c]->g.cisplit);
      b->key_k = iters_per_graph;
    }
    // per-case setup on the case streams: status cleared, ramp counter = iterations done
    for (int c = 0; c < n; ++c) {
      cs_grid g = b->grids[c];
      if (begin(g)) return bfail(b, CS_ERR_CUDA, "case %d: %s", c, g->err);
      k_set_int<<<1, 1, 0, g->stream>>>(g->iter_dev, g->iter);
      BCUDA_TRY(b, cudaEventRecord(b->ready[c], g->stream));
      BCUDA_TRY(b, cudaStreamWaitEvent(b->origin, b->ready[c], 0));
    }
    for (int r = 0; r < iters / iters_per_graph; ++r) BCUDA_TRY(b, cudaGraphLaunch(b->exec, b->origin));
    BCUDA_TRY(b, cudaStreamSynchronize(b->origin));
    cs_status worst = CS_OK;
    for (int c = 0; c < n; ++c) {
      cs_grid g = b->grids[c];
      BCUDA_TRY(b, cudaMemcpyAsync(g->h_pin + 32, g->norms, 3 * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
      const cs_status st = finish(g, "cs_batch_step");
      g->iter += iters;
      g->have_R = 0;
      if (stats) {
        stats[c].iters_done = st ? 0 : iters;
        stats[c].r_species = g->h_pin[32];
        stats[c].r_energy = g->h_pin[33];
        stats[c].q_stag = g->h_pin[34];
        stats[c].nclip = g->h_status[2];
        stats[c].status_cell = st ? g->h_status[1] : -1;
      }
      if (st && !worst) {
        worst = st;
        bfail(b, st, "case %d: %s", c, g->err);
      }
    }
    return worst;
  });
}

extern "C" cs_status cs_batch_stream(cs_batch b, void** stream_out) {
  if (!b || !stream_out) return CS_ERR_ARG;
  *stream_out = (void*)b->origin;
  return CS_OK;
}

extern "C" const char* cs_batch_last_error(cs_batch b) { return b ? b->err : "null batch"; }

// ---------------------------------------------------------------------------------------
// Chemistry surrogate coupling
// ---------------------------------------------------------------------------------------
extern "C" cs_status cs_surrogate_sample(cs_grid g, float* X_dev, float* T_dev) {
  if (!g || !X_dev || !T_dev) return CS_ERR_ARG;
  cs_status st = begin(g);
  if (st) return st;
  g->L->surr_sample(g->g, g->stream, X_dev, T_dev);
  return finish(g, "cs_surrogate_sample");
}

extern "C" cs_status cs_surrogate_attach(cs_grid g, cs_mlp m, const double* norm_host) {
  if (!g || !m || !norm_host) return CS_ERR_ARG;
  if (mlp_max_batch(m) < g->g.N) return fail(g, CS_ERR_ARG, "network batch %d < %d cells", mlp_max_batch(m), g->g.N);
  for (int k = 0; k < 14; ++k)
    if (!(norm_host[14 + k] > 0.0)) return fail(g, CS_ERR_ARG, "input std %d must be > 0", k);
  for (int k = 0; k < 22; ++k)
    if (!(norm_host[2 * 14 + 22 + k] > 0.0)) return fail(g, CS_ERR_ARG, "target std %d must be > 0", k);
  cudaError_t e = cudaSuccess;
  if (!g->sx) e = dalloc(g, &g->sx, (size_t)14 * g->g.N);
  if (e == cudaSuccess && !g->sy) e = dalloc(g, &g->sy, (size_t)22 * g->g.N);
  if (e == cudaSuccess && !g->snorm) e = dalloc(g, &g->snorm, 2 * (14 + 22));
  if (e != cudaSuccess) return fail(g, CS_ERR_OOM, "surrogate buffers");
  CUDA_TRY(g, cudaMemcpyAsync(g->snorm, norm_host, sizeof(double) * 2 * (14 + 22), cudaMemcpyHostToDevice, g->stream));
  CUDA_TRY(g, cudaStreamSynchronize(g->stream));
  g->surr = m;
  g->g.nojac = 1;
  return CS_OK;
}

extern "C" cs_status cs_surrogate_detach(cs_grid g) {
  if (!g) return CS_ERR_ARG;
  g->surr = nullptr;
  g->g.nojac = 0;
  return CS_OK;
}
