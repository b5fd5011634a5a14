// Species-count scaling test (Sec. 3.1, the time-acceleration test): one implicit LU-SGS step
// of the split (CS) and coupled (CI) operators for a uniform, non-reacting flow of ns species
// in a Cartesian box with far field on every side, for any ns (the 2D/3D solver's kernels fix
// ns at compile time; these take it at run time).
//
// Gas: species s is calorically perfect with R_s = R_u / M_s and c_v,s = (f_s / 2) R_s; no
// vibrational or formation energy.  State layout (rho_1 .. rho_ns, m_x, m_y, m_z, rho E) x
// cells, cell c = i + ni (j + nj k).  Radii are the inviscid ones (the flow is uniform):
// lambda_F,d = |u.S_d| + c |S_d|, lambda_C,d = |u.S_d|, V/dtau = sum_d lambda_F,d / CFL,
// D_F = D_CI = V/dtau + sum_d lambda_F,d, D_s = V/dtau + sum_d lambda_C,d.
//
//  CS (Sec. 2.3.1-2.3.2): a 5-unknown flow block (rho, m, rho E) with the frozen-composition
//   flux Jacobian, and ns independent scalar species equations with the Jacobian U I.  One
//   launch: CTA 0 sweeps the flow block through every hyperplane i+j+k (forward, then
//   backward), the other CTAs each sweep a group of species; hyperplanes are separated by
//   __syncthreads, and no CTA waits for another (the species sweeps use only the flow
//   quantities of the state, not the flow increments).
//  CI (Sec. 2.2, Sec. 2.3.3): n_c = ns + 4 unknowns (rho, m, rho E, rho_2 .. rho_ns).  The
//   diagonal block (V/dtau + sum lambda) I - V dS/dQ is assembled densely per cell and LU-
//   factorised with partial pivoting, as for a reacting flow (here dS/dQ = 0, but the cost of
//   the general operator is what the test measures); the sweeps apply the coupled flux
//   Jacobian matrix-free and solve with the factors, one launch per hyperplane and one CTA
//   per cell of it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/cs.h"

namespace csbox {

constexpr double kRu = 8314.462618;   // J/(kmol K)
constexpr int kSweepThreads = 256;
constexpr int kGroup = 8;             // species per CTA of the split sweep
constexpr int kCiThreads = 256;
constexpr double kMaxFactorBytes = 32.0 * (1ull << 30);   // largest CI factor storage allowed

struct Box {
  int ns, ni, nj, nk, N, H;          // H hyperplanes
  double S[3][3];                    // face vectors of the three face families
  double V;
  const double* Rs;                  // [ns]
  const double* cvs;                 // [ns]
  const double* Q;                   // [ns + 4][N]
  double* aux;                       // [kAux][N]
  const int* hp_off;                 // [H + 1]
  const int* hp_cell;                // [N] cells in hyperplane order
};
// per-cell auxiliary record: primitives, radii, diagonals and their reciprocals, and the
// species sweep's neighbour coefficients 1/2 (U_d + lambda_C,d), 1/2 (U_d - lambda_C,d)
// (computed once per cell, not once per species)
enum { A_RHO = 0, A_U = 1, A_P = 4, A_C = 5, A_GM1 = 6, A_T = 7, A_LF = 8, A_LC = 11, A_DF = 14,
       A_DS = 15, A_IRHO = 16, A_IDF = 17, A_IDS = 18, A_KF = 19, A_KB = 22, kAux = 25 };

__device__ __forceinline__ void cell_ijk(const Box& b, int c, int& i, int& j, int& k) {
  i = c % b.ni;
  j = (c / b.ni) % b.nj;
  k = c / (b.ni * b.nj);
}
// neighbour across side s of direction d, or -1 at the box's boundary
__device__ __forceinline__ int neighbour(const Box& b, int c, int d, int s) {
  int o[3];
  cell_ijk(b, c, o[0], o[1], o[2]);
  o[d] += s;
  const int n = d == 0 ? b.ni : (d == 1 ? b.nj : b.nk);
  if (o[d] < 0 || o[d] >= n) return -1;
  return o[0] + b.ni * (o[1] + b.nj * o[2]);
}

// uniform conserved state from (T, p, u, Y)
__global__ void k_state(Box b, const double* Y, double T, double p, double u0, double u1, double u2,
                        double* Q) {
  // one warp per cell: mixture gas constant and heat capacity, then the cell's state
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= b.N) return;
  double R = 0.0, cv = 0.0;
  for (int s = lane; s < b.ns; s += 32) {
    R += Y[s] * b.Rs[s];
    cv += Y[s] * b.cvs[s];
  }
  for (int o = 16; o > 0; o >>= 1) {
    R += __shfl_xor_sync(0xffffffffu, R, o);
    cv += __shfl_xor_sync(0xffffffffu, cv, o);
  }
  const double rho = p / (R * T);
  const size_t N = b.N;
  for (int s = lane; s < b.ns; s += 32) Q[s * N + warp] = rho * Y[s];
  if (lane == 0) {
    Q[(b.ns + 0) * N + warp] = rho * u0;
    Q[(b.ns + 1) * N + warp] = rho * u1;
    Q[(b.ns + 2) * N + warp] = rho * u2;
    Q[(b.ns + 3) * N + warp] = rho * cv * T + 0.5 * rho * (u0 * u0 + u1 * u1 + u2 * u2);
  }
}

// primitives, radii and diagonals of every cell (one warp per cell)
__global__ void k_aux(Box b, double cfl) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (c >= b.N) return;
  const size_t N = b.N;
  double rho = 0.0, rR = 0.0, rcv = 0.0;
  for (int s = lane; s < b.ns; s += 32) {
    const double r = b.Q[s * N + c];
    rho += r;
    rR += r * b.Rs[s];
    rcv += r * b.cvs[s];
  }
  for (int o = 16; o > 0; o >>= 1) {
    rho += __shfl_xor_sync(0xffffffffu, rho, o);
    rR += __shfl_xor_sync(0xffffffffu, rR, o);
    rcv += __shfl_xor_sync(0xffffffffu, rcv, o);
  }
  if (lane != 0) return;
  const double u[3] = {b.Q[(b.ns + 0) * N + c] / rho, b.Q[(b.ns + 1) * N + c] / rho,
                       b.Q[(b.ns + 2) * N + c] / rho};
  const double k = 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  const double T = (b.Q[(b.ns + 3) * N + c] - rho * k) / rcv;
  const double p = rR * T;
  const double gm1 = rR / rcv;
  const double cs = sqrt((1.0 + gm1) * p / rho);
  double* a = b.aux;
  a[A_RHO * N + c] = rho;
  for (int q = 0; q < 3; ++q) a[(A_U + q) * N + c] = u[q];
  a[A_P * N + c] = p;
  a[A_C * N + c] = cs;
  a[A_GM1 * N + c] = gm1;
  a[A_T * N + c] = T;
  double sF = 0.0, sC = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double* S = b.S[d];        // the mean of the cell's two d-faces (uniform box)
    const double U = u[0] * S[0] + u[1] * S[1] + u[2] * S[2];
    const double lF = fabs(U) + cs * sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    const double lC = fabs(U);
    a[(A_LF + d) * N + c] = lF;
    a[(A_LC + d) * N + c] = lC;
    a[(A_KF + d) * N + c] = 0.5 * (U + lC);
    a[(A_KB + d) * N + c] = 0.5 * (U - lC);
    sF += lF;
    sC += lC;
  }
  const double Vdt = sF / cfl;
  a[A_DF * N + c] = Vdt + sF;
  a[A_DS * N + c] = Vdt + sC;
  a[A_IRHO * N + c] = 1.0 / rho;
  a[A_IDF * N + c] = 1.0 / (Vdt + sF);
  a[A_IDS * N + c] = 1.0 / (Vdt + sC);
}

// flow-block right-hand side (sum_s rhs_s, rhs_m, rhs_E) [5][N] (one warp per cell)
__global__ void k_rhs_flow(Box b, const double* rhs, double* rf) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (c >= b.N) return;
  const size_t N = b.N;
  double r = 0.0;
  for (int s = lane; s < b.ns; s += 32) r += rhs[s * N + c];
  for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  if (lane == 0) {
    rf[c] = r;
    for (int v = 1; v < 5; ++v) rf[v * N + c] = rhs[(b.ns + v - 1) * N + c];
  }
}

// frozen-composition flow flux Jacobian of cell nb's state through S, applied to x (5)
// (a: the auxiliary records, rEv: rho E of every cell; in shared memory when staged)
__device__ __forceinline__ void jvp_flow(const Box& b, const double* a, const double* rEv, int nb,
                                         const double* S, const double* x, double* y) {
  const size_t N = b.N;
  const double rho = a[A_RHO * N + nb], p = a[A_P * N + nb], gm1 = a[A_GM1 * N + nb];
  const double u[3] = {a[A_U * N + nb], a[(A_U + 1) * N + nb], a[(A_U + 2) * N + nb]};
  const double rE = rEv[nb];
  const double U = u[0] * S[0] + u[1] * S[1] + u[2] * S[2];
  const double k = 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  const double Sm = S[0] * x[1] + S[1] * x[2] + S[2] * x[3];
  const double dU = (Sm - U * x[0]) * a[A_IRHO * N + nb];
  const double dp = gm1 * (k * x[0] - (u[0] * x[1] + u[1] * x[2] + u[2] * x[3]) + x[4]);
  y[0] = Sm;
  for (int q = 0; q < 3; ++q) y[1 + q] = x[1 + q] * U + rho * u[q] * dU + S[q] * dp;
  y[4] = (x[4] + dp) * U + (rE + p) * dU;
}

// CS: CTA 0 sweeps the flow block, CTA g >= 1 the species [kGroup (g-1), kGroup g).  xs is the
// species scratch in [cell][species] layout (contiguous across a CTA's species of a cell).
// A species update is three multiply-adds with the neighbours' precomputed coefficients and
// one multiply by the cell's reciprocal diagonal.
__global__ void __launch_bounds__(kSweepThreads) k_cs_sweeps(Box b, const double* rhs, const double* rf,
                                                             double* xF, double* xs, double* dQ) {
  const size_t N = b.N;
  const double* a = b.aux;
  const double* rEv = b.Q + (size_t)(b.ns + 3) * N;
  if (blockIdx.x == 0) {
    for (int pass = 0; pass < 2; ++pass) {
      const bool fwd = pass == 0;
      for (int hh = 0; hh < b.H; ++hh) {
        const int h = fwd ? hh : b.H - 1 - hh;
        for (int t = b.hp_off[h] + threadIdx.x; t < b.hp_off[h + 1]; t += blockDim.x) {
          const int c = b.hp_cell[t];
          double acc[5];
          for (int v = 0; v < 5; ++v) acc[v] = fwd ? rf[v * N + c] : 0.0;
          for (int d = 0; d < 3; ++d) {
            const int s = fwd ? -1 : 1;
            const int nb = neighbour(b, c, d, s);
            if (nb < 0) continue;
            double xn[5], ax[5];
            for (int v = 0; v < 5; ++v) xn[v] = fwd ? xF[v * N + nb] : dQ[v * N + nb];
            jvp_flow(b, a, rEv, nb, b.S[d], xn, ax);
            const double l = a[(A_LF + d) * N + nb];
            for (int v = 0; v < 5; ++v) acc[v] += fwd ? 0.5 * (ax[v] + l * xn[v]) : -0.5 * (ax[v] - l * xn[v]);
          }
          const double iD = a[A_IDF * N + c];
          for (int v = 0; v < 5; ++v) {
            if (fwd) xF[v * N + c] = acc[v] * iD;
            else dQ[v * N + c] = xF[v * N + c] + acc[v] * iD;
          }
        }
        __syncthreads();
      }
    }
    return;
  }
  // species group
  const int G = b.ns < kGroup ? b.ns : kGroup;
  const int s = (blockIdx.x - 1) * G + (int)threadIdx.x % G;
  const int slot = threadIdx.x / G, nslot = blockDim.x / G;
  const bool active = s < b.ns && slot < nslot;
  const int ns = b.ns;
  for (int pass = 0; pass < 2; ++pass) {
    const bool fwd = pass == 0;
    for (int hh = 0; hh < b.H; ++hh) {
      const int h = fwd ? hh : b.H - 1 - hh;
      if (active) {
        for (int t = b.hp_off[h] + slot; t < b.hp_off[h + 1]; t += nslot) {
          const int c = b.hp_cell[t];
          double acc = fwd ? rhs[(size_t)s * N + c] : 0.0;
          for (int d = 0; d < 3; ++d) {
            const int nb = neighbour(b, c, d, fwd ? -1 : 1);
            if (nb < 0) continue;
            if (fwd) acc += a[(A_KF + d) * N + nb] * xs[(size_t)nb * ns + s];
            else acc -= a[(A_KB + d) * N + nb] * dQ[(size_t)(5 + s) * N + nb];
          }
          const double iD = a[A_IDS * N + c];
          if (fwd) xs[(size_t)c * ns + s] = acc * iD;
          else dQ[(size_t)(5 + s) * N + c] = xs[(size_t)c * ns + s] + acc * iD;
        }
      }
      __syncthreads();
    }
  }
}

// ---- CI ------------------------------------------------------------------------------------
// block reductions (blockDim = kCiThreads)
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  for (int k = 0; k < kCiThreads / 32; ++k) r += sh[k];
  return r;
}

// Dense diagonal block per cell, LU with partial pivoting in place, column-major (element
// (i, j) at j n + i); piv[k] = row swapped with row k.  One CTA per cell (grid-stride).
// Right-looking and blocked by panels of kPanel columns: (1) the panel is factorised column
// by column (pivot search, swap of the whole row, scaling, update inside the panel); (2) the
// panel's block row right of it is solved with the panel's unit lower triangle; (3) the
// trailing matrix takes the rank-kPanel update L21 U12 in 64 x 64 tiles staged through shared
// memory, each thread accumulating a 4 x 4 block in registers.  The same arithmetic as the
// unblocked algorithm up to the order of the sums in the trailing update.
constexpr int kPanel = 32, kTile = 64;

__global__ void __launch_bounds__(kCiThreads) k_ci_factor(Box b, double* LU, int* piv, int* err) {
  __shared__ double sv[kCiThreads];
  __shared__ int si[kCiThreads];
  __shared__ double sL[kPanel][kTile];   // L21 tile, column c of the panel x 64 rows
  __shared__ double sU[kPanel][kTile];   // U12 tile, row c of the panel x 64 columns
  const int n = b.ns + 4;
  const size_t nn = (size_t)n * n;
  const int tid = threadIdx.x;
  for (int c = blockIdx.x; c < b.N; c += gridDim.x) {
    double* A = LU + (size_t)c * nn;
    const double diag = b.aux[A_DF * (size_t)b.N + c];   // V/dtau + sum lambda (no source Jacobian)
    for (size_t e = tid; e < nn; e += blockDim.x) A[e] = (e % (n + 1) == 0) ? diag : 0.0;
    __syncthreads();
    bool singular = false;
    for (int k0 = 0; k0 < n && !singular; k0 += kPanel) {
      const int kb = n - k0 < kPanel ? n - k0 : kPanel, ke = k0 + kb;
      // (1) panel
      for (int k = k0; k < ke; ++k) {
        double best = -1.0;
        int bi = k;
        for (int i = k + tid; i < n; i += blockDim.x) {
          const double v = fabs(A[(size_t)k * n + i]);
          if (v > best) { best = v; bi = i; }
        }
        sv[tid] = best;
        si[tid] = bi;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
          if (tid < w) {
            const double o = sv[tid + w];
            const int oi = si[tid + w];
            if (o > sv[tid] || (o == sv[tid] && oi < si[tid])) { sv[tid] = o; si[tid] = oi; }
          }
          __syncthreads();
        }
        const int p = si[0];
        const double pv = sv[0];
        __syncthreads();
        if (tid == 0) piv[(size_t)c * n + k] = p;
        if (!(pv > 0.0)) {
          if (tid == 0) atomicExch(err, c + 1);
          singular = true;
          break;
        }
        if (p != k)
          for (int jj = tid; jj < n; jj += blockDim.x) {
            const double t = A[(size_t)jj * n + k];
            A[(size_t)jj * n + k] = A[(size_t)jj * n + p];
            A[(size_t)jj * n + p] = t;
          }
        __syncthreads();
        const double ip = 1.0 / A[(size_t)k * n + k];
        for (int i = k + 1 + tid; i < n; i += blockDim.x) A[(size_t)k * n + i] *= ip;
        __syncthreads();
        const int mr = n - k - 1, mc = ke - k - 1;       // rows below, panel columns right of k
        for (long e = tid; e < (long)mr * mc; e += blockDim.x) {
          const int i = k + 1 + (int)(e % mr), jj = k + 1 + (int)(e / mr);
          A[(size_t)jj * n + i] -= A[(size_t)k * n + i] * A[(size_t)jj * n + k];
        }
        __syncthreads();
      }
      if (singular || ke >= n) continue;
      // (2) U12 = L11^-1 A12, one thread per column right of the panel
      for (int jj = ke + tid; jj < n; jj += blockDim.x) {
        double* col = A + (size_t)jj * n;
        for (int r = k0 + 1; r < ke; ++r) {
          double acc = col[r];
          for (int cc = k0; cc < r; ++cc) acc -= A[(size_t)cc * n + r] * col[cc];
          col[r] = acc;
        }
      }
      __syncthreads();
      // (3) A22 -= L21 U12
      const int m = n - ke;
      const int tiles = (m + kTile - 1) / kTile;
      const int tx = tid % 16, ty = tid / 16;            // 4 x 4 block: rows 4 tx, columns 4 ty
      for (int tt = 0; tt < tiles * tiles; ++tt) {
        const int r0 = ke + (tt % tiles) * kTile, c0 = ke + (tt / tiles) * kTile;
        for (int e = tid; e < kPanel * kTile; e += blockDim.x) {
          const int cc = e / kTile, rr = e % kTile;
          const bool in = cc < kb;
          sL[cc][rr] = (in && r0 + rr < n) ? A[(size_t)(k0 + cc) * n + r0 + rr] : 0.0;
          sU[cc][rr] = (in && c0 + rr < n) ? A[(size_t)(c0 + rr) * n + k0 + cc] : 0.0;
        }
        __syncthreads();
        double acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[a][q] = 0.0;
        for (int cc = 0; cc < kb; ++cc) {
          double l[4], u[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) { l[a] = sL[cc][4 * tx + a]; u[a] = sU[cc][4 * ty + a]; }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[a][q] += l[a] * u[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int jj = c0 + 4 * ty + q;
          if (jj >= n) continue;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int i = r0 + 4 * tx + a;
            if (i < n) A[(size_t)jj * n + i] -= acc[a][q];
          }
        }
        __syncthreads();
      }
    }
    __syncthreads();
  }
}

// coupled flux Jacobian of cell nb's state through S applied to x (CI layout, n values in
// shared memory), added as sign * 1/2 (A x +- lambda x) into acc (shared)
__device__ void ci_gather(const Box& b, int nb, int d, bool lower, const double* x, double* acc,
                          double* red) {
  const size_t N = b.N;
  const int ns = b.ns, n = ns + 4;
  const double* a = b.aux;
  const double* S = b.S[d];
  const double rho = a[A_RHO * N + nb], p = a[A_P * N + nb], gm1 = a[A_GM1 * N + nb], T = a[A_T * N + nb];
  const double u[3] = {a[A_U * N + nb], a[(A_U + 1) * N + nb], a[(A_U + 2) * N + nb]};
  const double k = 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  const double rE = b.Q[(ns + 3) * N + nb];
  const double U = u[0] * S[0] + u[1] * S[1] + u[2] * S[2];
  const double l = a[(A_LF + d) * N + nb];
  // dp = sum_s p_s drho_s - gm1 u.dm + gm1 drhoE, p_s = T (R_s - gm1 cv_s) + gm1 k, with
  // drho_1 = drho - sum_{r>1} drho_r
  const double p1 = T * (b.Rs[0] - gm1 * b.cvs[0]) + gm1 * k;
  double part = 0.0;
  for (int r = 1 + threadIdx.x; r < ns; r += blockDim.x)
    part += (T * (b.Rs[r] - gm1 * b.cvs[r]) + gm1 * k - p1) * x[4 + r];
  const double sdp = block_sum(part, red);
  const double Sm = S[0] * x[1] + S[1] * x[2] + S[2] * x[3];
  const double dU = (Sm - U * x[0]) / rho;
  const double dp = p1 * x[0] + sdp - gm1 * (u[0] * x[1] + u[1] * x[2] + u[2] * x[3]) + gm1 * x[4];
  const double sg = lower ? 0.5 : -0.5, sl = lower ? l : -l;
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    double ax;
    if (v == 0) ax = Sm;
    else if (v < 4) ax = x[v] * U + rho * u[v - 1] * dU + S[v - 1] * dp;
    else if (v == 4) ax = (x[4] + dp) * U + (rE + p) * dU;
    else ax = x[v] * U + b.Q[(size_t)(v - 4) * N + nb] * dU;    // species r = v - 4 >= 1
    acc[v] += sg * (ax + sl * x[v]);
  }
  __syncthreads();
}

// solve LU z = acc in place (shared), with the row swaps of piv
__device__ void ci_solve(const double* A, const int* piv, int n, double* z) {
  for (int k = 0; k < n; ++k) {
    const int p = piv[k];
    if (p != k && threadIdx.x == 0) {
      const double t = z[k];
      z[k] = z[p];
      z[p] = t;
    }
    __syncthreads();
  }
  for (int k = 0; k < n; ++k) {                    // unit lower
    const double zk = z[k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) z[i] -= A[(size_t)k * n + i] * zk;
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {               // upper
    if (threadIdx.x == 0) z[k] /= A[(size_t)k * n + k];
    __syncthreads();
    const double zk = z[k];
    for (int i = threadIdx.x; i < k; i += blockDim.x) z[i] -= A[(size_t)k * n + i] * zk;
    __syncthreads();
  }
}

// one hyperplane of the CI forward (fwd) or backward sweep; one CTA per cell of it.
// Dynamic shared memory: 2 n doubles (neighbour vector, accumulator).
__global__ void __launch_bounds__(kCiThreads) k_ci_sweep(Box b, int h, bool fwd, const double* rhs,
                                                         const double* LU, const int* piv, double* x,
                                                         double* y) {
  extern __shared__ double sm[];
  __shared__ double red[kCiThreads / 32];
  const int t = b.hp_off[h] + blockIdx.x;
  if (t >= b.hp_off[h + 1]) return;
  const int c = b.hp_cell[t];
  const size_t N = b.N;
  const int ns = b.ns, n = ns + 4;
  double* xn = sm;
  double* acc = sm + n;
  if (fwd) {
    double part = 0.0;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) part += rhs[(size_t)s * N + c];
    const double rs = block_sum(part, red);
    for (int v = threadIdx.x; v < n; v += blockDim.x)
      acc[v] = v == 0 ? rs : (v < 5 ? rhs[(size_t)(ns + v - 1) * N + c] : rhs[(size_t)(v - 4) * N + c]);
  } else {
    for (int v = threadIdx.x; v < n; v += blockDim.x) acc[v] = 0.0;
  }
  __syncthreads();
  for (int d = 0; d < 3; ++d) {
    const int nb = neighbour(b, c, d, fwd ? -1 : 1);
    if (nb < 0) continue;
    const double* src = fwd ? x : y;
    for (int v = threadIdx.x; v < n; v += blockDim.x) xn[v] = src[(size_t)v * N + nb];
    __syncthreads();
    ci_gather(b, nb, d, fwd, xn, acc, red);
  }
  ci_solve(LU + (size_t)c * n * n, piv + (size_t)c * n, n, acc);
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    if (fwd) x[(size_t)v * N + c] = acc[v];
    else y[(size_t)v * N + c] = x[(size_t)v * N + c] + acc[v];
  }
}

}  // namespace csbox

using namespace csbox;

struct cs_species_box_s {
  Box b{};
  cudaStream_t st = nullptr;
  std::vector<void*> allocs;
  double* aux = nullptr;
  double* Q = nullptr;
  double* rf = nullptr;      // flow right-hand side [5][N]
  double* xF = nullptr;      // flow forward increments [5][N]
  double* xs = nullptr;      // species forward increments [N][ns]
  double* ci_x = nullptr;    // CI forward increments [n][N]
  double* LU = nullptr;      // CI factors [N][n][n] (allocated on first use)
  int* piv = nullptr;
  int* err = nullptr;
  std::vector<int> hp_off;
  char msg[256] = {0};
};

static cs_status bfail(cs_species_box b, cs_status s, const char* fmt, ...) {
  if (b) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->msg, sizeof b->msg, fmt, ap);
    va_end(ap);
  }
  return s;
}

template <class T>
static bool balloc(cs_species_box b, T** p, size_t n) {
  void* v = nullptr;
  if (cudaMalloc(&v, n * sizeof(T) > 0 ? n * sizeof(T) : 8) != cudaSuccess) return false;
  b->allocs.push_back(v);
  *p = (T*)v;
  return cudaMemsetAsync(v, 0, n * sizeof(T) > 0 ? n * sizeof(T) : 8, b->st) == cudaSuccess;
}

static bool device_ptr(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

extern "C" cs_status cs_species_box_create(int ns, int ni, int nj, int nk, const double* size_host,
                                           const double* M_host, const double* dof_host,
                                           const double* Y_host, double T, double p,
                                           const double* u_host, cs_species_box* out) {
  if (!out || !size_host || !M_host || !dof_host || !Y_host || !u_host) return CS_ERR_ARG;
  *out = nullptr;
  if (ns < 1 || ns > 65536 || ni < 1 || nj < 1 || nk < 1 || (long)ni * nj * nk > (1L << 24))
    return CS_ERR_ARG;
  if (!(T > 0.0) || !(p > 0.0)) return CS_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (!(size_host[d] > 0.0) || !std::isfinite(u_host[d])) return CS_ERR_ARG;
  for (int s = 0; s < ns; ++s)
    if (!(M_host[s] > 0.0) || !(dof_host[s] > 0.0) || !(Y_host[s] >= 0.0)) return CS_ERR_ARG;
  cs_species_box b = new cs_species_box_s();
  if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) { delete b; return CS_ERR_CUDA; }
  Box& x = b->b;
  x.ns = ns; x.ni = ni; x.nj = nj; x.nk = nk; x.N = ni * nj * nk; x.H = ni + nj + nk - 2;
  const double h[3] = {size_host[0] / ni, size_host[1] / nj, size_host[2] / nk};
  for (int d = 0; d < 3; ++d)
    for (int q = 0; q < 3; ++q) x.S[d][q] = 0.0;
  x.S[0][0] = h[1] * h[2];
  x.S[1][1] = h[0] * h[2];
  x.S[2][2] = h[0] * h[1];
  x.V = h[0] * h[1] * h[2];
  // hyperplane order of the cells (i + j + k ascending, cell index within)
  std::vector<int> cnt(x.H + 1, 0), cells(x.N);
  for (int c = 0; c < x.N; ++c) {
    const int i = c % ni, j = (c / ni) % nj, k = c / (ni * nj);
    cnt[i + j + k + 1]++;
  }
  for (int q = 0; q < x.H; ++q) cnt[q + 1] += cnt[q];
  b->hp_off = cnt;
  std::vector<int> fill(cnt.begin(), cnt.end() - 1);
  for (int c = 0; c < x.N; ++c) {
    const int i = c % ni, j = (c / ni) % nj, k = c / (ni * nj);
    cells[fill[i + j + k]++] = c;
  }
  std::vector<double> Rs(ns), cvs(ns);
  for (int s = 0; s < ns; ++s) {
    Rs[s] = kRu / M_host[s];
    cvs[s] = 0.5 * dof_host[s] * Rs[s];
  }
  double *dRs, *dcv, *dY;
  int *doff, *dcell;
  const size_t N = x.N;
  bool ok = balloc(b, &dRs, ns) && balloc(b, &dcv, ns) && balloc(b, &dY, ns) &&
            balloc(b, &doff, x.H + 1) && balloc(b, &dcell, N) && balloc(b, &b->Q, (ns + 4) * N) &&
            balloc(b, &b->aux, kAux * N) && balloc(b, &b->rf, 5 * N) && balloc(b, &b->xF, 5 * N) &&
            balloc(b, &b->xs, (size_t)ns * N) && balloc(b, &b->ci_x, (size_t)(ns + 4) * N) &&
            balloc(b, &b->err, 1);
  if (!ok) { cs_species_box_destroy(b); return CS_ERR_OOM; }
  ok = cudaMemcpyAsync(dRs, Rs.data(), ns * sizeof(double), cudaMemcpyHostToDevice, b->st) == cudaSuccess &&
       cudaMemcpyAsync(dcv, cvs.data(), ns * sizeof(double), cudaMemcpyHostToDevice, b->st) == cudaSuccess &&
       cudaMemcpyAsync(dY, Y_host, ns * sizeof(double), cudaMemcpyHostToDevice, b->st) == cudaSuccess &&
       cudaMemcpyAsync(doff, cnt.data(), (x.H + 1) * sizeof(int), cudaMemcpyHostToDevice, b->st) == cudaSuccess &&
       cudaMemcpyAsync(dcell, cells.data(), N * sizeof(int), cudaMemcpyHostToDevice, b->st) == cudaSuccess;
  x.Rs = dRs; x.cvs = dcv; x.hp_off = doff; x.hp_cell = dcell; x.Q = b->Q; x.aux = b->aux;
  if (ok) {
    k_state<<<(int)((N * 32 + 255) / 256), 256, 0, b->st>>>(x, dY, T, p, u_host[0], u_host[1], u_host[2], b->Q);
    ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(b->st) == cudaSuccess;
  }
  if (!ok) { cs_species_box_destroy(b); return CS_ERR_CUDA; }
  *out = b;
  return CS_OK;
}

extern "C" cs_status cs_species_box_destroy(cs_species_box b) {
  if (!b) return CS_ERR_ARG;
  if (b->st) cudaStreamSynchronize(b->st);
  for (void* p : b->allocs) cudaFree(p);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
  return CS_OK;
}

extern "C" cs_status cs_species_box_state(cs_species_box b, double* Q_dev) {
  if (!b || !Q_dev || !device_ptr(Q_dev)) return CS_ERR_ARG;
  const size_t n = (size_t)(b->b.ns + 4) * b->b.N;
  if (cudaMemcpyAsync(Q_dev, b->Q, n * sizeof(double), cudaMemcpyDeviceToDevice, b->st) != cudaSuccess ||
      cudaStreamSynchronize(b->st) != cudaSuccess)
    return bfail(b, CS_ERR_CUDA, "state copy");
  return CS_OK;
}

// enqueue one implicit step (no synchronisation)
static cs_status enqueue_step(cs_species_box b, int scheme, double cfl, const double* rhs, double* dQ) {
  Box& x = b->b;
  const size_t N = x.N;
  const int warps_grid = (int)((N * 32 + 255) / 256);
  k_aux<<<warps_grid, 256, 0, b->st>>>(x, cfl);
  if (scheme == CS_SCHEME_SPLIT) {
    k_rhs_flow<<<warps_grid, 256, 0, b->st>>>(x, rhs, b->rf);
    const int G = x.ns < kGroup ? x.ns : kGroup;
    const int groups = (x.ns + G - 1) / G;
    k_cs_sweeps<<<1 + groups, kSweepThreads, 0, b->st>>>(x, rhs, b->rf, b->xF, b->xs, dQ);
  } else {
    const int n = x.ns + 4;
    if ((double)N * n * n * sizeof(double) > kMaxFactorBytes)
      return bfail(b, CS_ERR_ARG, "coupled factors of %d cells x %d^2 exceed %.0f GB", (int)N, n,
                   kMaxFactorBytes / 1e9);
    if (!b->LU) {
      if (!balloc(b, &b->LU, (size_t)N * n * n) || !balloc(b, &b->piv, (size_t)N * n))
        return bfail(b, CS_ERR_OOM, "coupled factors: %zu bytes", (size_t)N * n * n * sizeof(double));
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)N < 4 * sms ? (int)N : 4 * sms;
    k_ci_factor<<<grid, kCiThreads, 0, b->st>>>(x, b->LU, b->piv, b->err);
    const size_t smem = 2 * (size_t)n * sizeof(double);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_ci_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return bfail(b, CS_ERR_ARG, "ns = %d too large for the coupled sweep's shared memory", x.ns);
    for (int pass = 0; pass < 2; ++pass)
      for (int hh = 0; hh < x.H; ++hh) {
        const int h = pass == 0 ? hh : x.H - 1 - hh;
        const int cnt = b->hp_off[h + 1] - b->hp_off[h];
        k_ci_sweep<<<cnt, kCiThreads, smem, b->st>>>(x, h, pass == 0, rhs, b->LU, b->piv, b->ci_x, dQ);
      }
  }
  if (cudaGetLastError() != cudaSuccess) return bfail(b, CS_ERR_CUDA, "launch");
  return CS_OK;
}

extern "C" cs_status cs_species_box_step(cs_species_box b, int scheme, double cfl, const double* rhs_dev,
                                         double* dQ_dev) {
  if (!b || !rhs_dev || !dQ_dev || !(cfl > 0.0)) return CS_ERR_ARG;
  if (scheme != CS_SCHEME_SPLIT && scheme != CS_SCHEME_COUPLED) return bfail(b, CS_ERR_ARG, "scheme %d", scheme);
  if (!device_ptr(rhs_dev) || !device_ptr(dQ_dev)) return bfail(b, CS_ERR_ARG, "device pointers required");
  if (cudaMemsetAsync(b->err, 0, sizeof(int), b->st) != cudaSuccess) return bfail(b, CS_ERR_CUDA, "memset");
  cs_status s = enqueue_step(b, scheme, cfl, rhs_dev, dQ_dev);
  if (s) return s;
  int e = 0;
  if (cudaMemcpyAsync(&e, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->st) != cudaSuccess ||
      cudaStreamSynchronize(b->st) != cudaSuccess)
    return bfail(b, CS_ERR_CUDA, "%s", cudaGetErrorString(cudaGetLastError()));
  if (e) return bfail(b, CS_ERR_NONPHYSICAL, "singular coupled block at cell %d", e - 1);
  return CS_OK;
}

extern "C" cs_status cs_species_box_time(cs_species_box b, int scheme, double cfl, const double* rhs_dev,
                                         double* dQ_dev, int reps, void* flush_dev, size_t flush_bytes,
                                         double* ms_out) {
  if (!b || !ms_out || reps < 1 || (flush_bytes && !flush_dev)) return CS_ERR_ARG;
  if (!rhs_dev || !dQ_dev || !(cfl > 0.0)) return CS_ERR_ARG;
  if (scheme != CS_SCHEME_SPLIT && scheme != CS_SCHEME_COUPLED) return bfail(b, CS_ERR_ARG, "scheme %d", scheme);
  if (!device_ptr(rhs_dev) || !device_ptr(dQ_dev) || (flush_bytes && !device_ptr(flush_dev)))
    return bfail(b, CS_ERR_ARG, "device pointers required");
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return bfail(b, CS_ERR_CUDA, "events");
  cs_status s = CS_OK;
  double total = 0.0;
  for (int r = 0; r < reps && !s; ++r) {
    // the flush (a write larger than L2) stays outside the timed events
    if (flush_bytes && cudaMemsetAsync(flush_dev, r & 0xff, flush_bytes, b->st) != cudaSuccess) {
      s = bfail(b, CS_ERR_CUDA, "flush");
      break;
    }
    cudaEventRecord(e0, b->st);
    s = enqueue_step(b, scheme, cfl, rhs_dev, dQ_dev);
    cudaEventRecord(e1, b->st);
    float ms = 0.f;
    if (!s && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      s = bfail(b, CS_ERR_CUDA, "timing");
    total += ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s) return s;
  *ms_out = total / reps;
  return CS_OK;
}

extern "C" const char* cs_species_box_last_error(cs_species_box b) { return b ? b->msg : "null box"; }
