// Device-side gas model for the GB300 path: species thermodynamics (rigid rotor / harmonic
// oscillator, two-temperature pools), Park air kinetics and transport.
//
// Paper: arXiv:2403.03440 Sec. 2.1 (e_t, e_v, ideal-gas law; thermodynamic, transport and
// kinetic data deferred to the paper's references) and Sec. 3.2 (Park's 11-species /
// 21-reaction air, rates as tabulated by Gnoffo et al.).
//
// Everything is templated on the gas model so that per-species arrays have compile-time
// size and live in registers.  All arithmetic is FP64.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace cs {

constexpr double kRu = 8314.462618;        // J/(kmol K)
constexpr double kKb = 1.380649e-23;       // J/K
constexpr double kH = 6.62607015e-34;      // J s
constexpr double kNa = 6.02214076e26;      // 1/kmol
constexpr double kPref = 101325.0;         // Pa, standard state
constexpr double kPi = 3.14159265358979323846;
constexpr double kTmin = 20.0, kTmax = 1.0e5;
constexpr double kSuthMu = 1.458e-6, kSuthT = 110.4, kPr = 0.72, kSc = 0.5;
// reciprocals of constants, so that the kernels multiply instead of dividing
constexpr double kInvPr = 1.0 / kPr, kInvSc = 1.0 / kSc, kInvRu = 1.0 / kRu, kInvPref = 1.0 / kPref;

enum Kind { ATOM = 0, DIATOMIC = 1, ELECTRON = 2 };
enum TempKind { TK_T = 0, TK_A = 1, TK_V = 2 };

struct SpeciesData {
  int kind;
  double M;       // kg/kmol
  double thv;     // vibrational temperature, K (0: none)
  double thr;     // rotational temperature, K
  double sigma;   // symmetry number
  double g0;      // ground-state degeneracy
  double h0;      // formation energy at 0 K, J/kmol
};

struct ReactionData {
  int nr, r[3], np, p[3];
  int third;
  double lnA;     // ln of A in m^3/(kmol s)
  double n, theta;
  int tf, tb;
  double eff[11];
};

// Molar masses from the element masses so that every reaction conserves mass exactly.
#define CS_MN 14.0067
#define CS_MO 15.9994
#define CS_ME 5.48579909e-4

#define CS_AIR_SPECIES                                             \
  {                                                                \
    {DIATOMIC, 2 * CS_MN, 3395.0, 2.88, 2, 1, 0.0},                \
    {DIATOMIC, 2 * CS_MO, 2239.0, 2.08, 2, 3, 0.0},                \
    {DIATOMIC, CS_MN + CS_MO, 2817.0, 2.45, 1, 4, 89.77e6},        \
    {ATOM, CS_MN, 0.0, 0.0, 1, 4, 470.82e6},                       \
    {ATOM, CS_MO, 0.0, 0.0, 1, 9, 246.79e6},                       \
    {DIATOMIC, CS_MN + CS_MO - CS_ME, 3419.0, 2.87, 1, 1, 983.6e6}, \
    {DIATOMIC, 2 * CS_MN - CS_ME, 3175.0, 2.78, 2, 2, 1503.3e6},   \
    {DIATOMIC, 2 * CS_MO - CS_ME, 2741.0, 2.43, 2, 4, 1164.5e6},   \
    {ATOM, CS_MN - CS_ME, 0.0, 0.0, 1, 9, 1873.1e6},               \
    {ATOM, CS_MO - CS_ME, 0.0, 0.0, 1, 4, 1560.7e6},               \
    {ELECTRON, CS_ME, 0.0, 0.0, 1, 2, 0.0},                        \
  }
__constant__ SpeciesData c_species_air[11] = CS_AIR_SPECIES;
static const SpeciesData kSpeciesHost[11] = CS_AIR_SPECIES;   // host copy (derived constants)
__constant__ SpeciesData c_species_perfect[1] = {
    {DIATOMIC, 28.9647, 0.0, 2.88, 2, 1, 0.0},
};

// Blottner's viscosity fits mu_s = 0.1 exp((A ln T + B) ln T + C) kg/(m s) (Blottner, Johnson
// & Ellis, Sandia report SC-RR-70-754, 1971), species order of the air table; the four other
// ions take the fit given for NO+.
#define CS_BLOTTNER                                                                          \
  {                                                                                          \
    {0.0268142, 0.3177838, -11.3155513}, {0.0449290, -0.0826158, -9.2019475},                \
        {0.0436378, -0.0335511, -9.5767430}, {0.0115572, 0.6031679, -12.4327495},            \
        {0.0203144, 0.4294404, -11.6031403}, {0.3020141, -3.5039791, -3.7355157},            \
        {0.3020141, -3.5039791, -3.7355157}, {0.3020141, -3.5039791, -3.7355157},            \
        {0.3020141, -3.5039791, -3.7355157}, {0.3020141, -3.5039791, -3.7355157},            \
        {0.0, 0.0, -12.5},                                                                   \
  }
static const double kBlottnerHost[11][3] = CS_BLOTTNER;

// Park's air reactions, forward rate A T^n exp(-theta/T).  Species order:
// N2 O2 NO N O NO+ N2+ O2+ N+ O+ e-.  ln A is filled on the host from A in cm^3/(mol s).
#define CS_EFF_N2 {1, 1, 1, 30.0 / 7.0, 30.0 / 7.0, 1, 1, 1, 30.0 / 7.0, 30.0 / 7.0, 3.0e24 / 7.0e21}
#define CS_EFF_O2 {1, 1, 1, 5, 5, 1, 1, 1, 5, 5, 0}
#define CS_EFF_NO {1, 1, 22, 22, 22, 1, 1, 1, 22, 22, 0}
__constant__ ReactionData c_reactions[21];

// Constants derived on the host from the species table (so that the kernels evaluate no
// logarithm or power of a constant):
//  gc0[s]  = -1.5 ln(2 pi m k / h^2) - ln(k / p0) - ln g0 [+ ln(sigma theta_r) for diatomics],
//            so that g_s/(R T) = h0/(R T) - (2.5 [+1]) ln T + gc0 [+ ln(1 - exp(-theta_v/T))]
//  mwA[s][q], mwAB[s][q]: Millikan-White tau_sq p = exp(A T^-1/3 - AB), AB = A B + 18.42
//  cbk[s]  = sqrt(8 R_u / (pi M_s)): mean molecular speed = cbk sqrt(T)
//  Rs[s] = R_u / M_s, hf[s] = h0_s / M_s, invM[s] = 1 / M_s (no division in the kernels)
struct GasConst {
  double gc0[11];
  double mwA[11][11];
  double mwAB[11][11];
  double cbk[11];
  double Rs[11], hf[11], invM[11];
  double icbk[11];  // 1 / cbk
  double lnPRu;     // ln(p0 / R_u)
  float Rsf[11], hff[11], thvf[11];   // FP32 copies for the temperature solves' predictor
  // species transport model (option transport = 1): Blottner fit coefficients A, B, C;
  // Wilke's (M_r/M_s)^(1/4) and 1/sqrt(8 (1 + M_s/M_r)); hard-sphere constants
  // hsd[s] = (5/16) sqrt(pi m_s k) / pi (sigma_s^2 = hsd sqrt(T) / mu_s), dsr[s][r] =
  // 3/8 sqrt(k / (2 pi m_sr)) (D_sr = dsr sqrt(T) / (n sigma_sr^2)), ipm[s] = N_A / M_s
  double blA[11], blB[11], blC[11];
  double wm[11][11], wd[11][11];
  double hsd[11], dsr[11][11], ipm[11];
};
__constant__ GasConst c_gas;

// 2^(j/64), j = 0..63, for exp_tab (filled on the host with exp2; read through the L1 cache)
__device__ double g_exp2_64[64];

// ln(1 + j/256) and 1/(1 + j/256), j = 0..255, for log_tab (filled on the host)
__device__ double g_lnF_256[256];
__device__ double g_invF_256[256];

// Natural logarithm by Tang's table-driven method (P. T. P. Tang, ACM Trans. Math. Softw.
// 16(4), 1990), with 256 table entries: x = 2^k y, y in [1, 2), F = 1 + j/256 the leading eight
// bits of y's mantissa, so that ln x = k ln2 + ln F + ln(1 + u) with u = (y - F)/F, 0 <= u <
// 1/256 (y - F is exact); ln(1 + u) from its Taylor series to degree 6 (truncation below 2e-18).
// Absolute error a few units of 1e-17 for the arguments of this library (temperatures, 1 -
// exp(-theta/T)); non-normal or non-finite arguments take CUDA's log.
__device__ __forceinline__ double log_tab(double x) {
  if (!(x >= 2.2250738585072014e-308 && x <= 1.7976931348623157e308)) return log(x);
  const long long b = __double_as_longlong(x);
  const int k = (int)((b >> 52) & 0x7ff) - 1023;
  const int j = (int)((b >> 44) & 0xff);
  const double y = __longlong_as_double((b & 0xFFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
  const double F = __longlong_as_double(0x3FF0000000000000LL | ((long long)j << 44));
  const double u = (y - F) * __ldg(&g_invF_256[j]);
  double p = fma(u, -1.0 / 6.0, 0.2);
  p = fma(u, p, -0.25);
  p = fma(u, p, 1.0 / 3.0);
  p = fma(u, p, -0.5);
  p = fma(u, p, 1.0);
  p *= u;
  return fma((double)k, 0.6931471805599453, __ldg(&g_lnF_256[j]) + p);
}

// Exponential by Tang's table-driven method (P. T. P. Tang, ACM Trans. Math. Softw. 15(2),
// 1989), with 64 table entries: x = (64 m + j) ln2/64 + r, |r| <= ln2/128, so that
// exp(x) = 2^m 2^(j/64) exp(r) with exp(r) - 1 from its Taylor series to degree 5 (truncation
// below 2e-17 relative).  The shifter 1.5 * 2^52 rounds x 64/ln2 to the integer N = 64 m + j in
// the low bits of a double; ln2/64 is split into a leading and a trailing part so that r is
// accurate to a few units of its last place.  2^m is applied by an integer add to the exponent
// field.  Measured against CUDA's exp on [-700, 700]: at most 1 ulp apart, ~1.5x the throughput
// on GB300 (fewer FP64 operations).  Arguments outside [-707, 709] (results below 1e-307 or
// near overflow) take CUDA's exp.
__device__ __forceinline__ double exp_tab(double x) {
  if (!(x > -707.0 && x < 709.0)) return exp(x);
  const double t = fma(x, 92.33248261689366, 6755399441055744.0);   // x 64/ln2 + 1.5 2^52
  const double N = t - 6755399441055744.0;
  double r = fma(-N, 0.010830424696249145, x);                         // ln2/64, leading part
  r = fma(-N, 3.623510646634843e-19, r);                               // ln2/64, trailing part
  double p = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  p = fma(r, p, 1.0 / 6.0);
  p = fma(r, p, 0.5);
  p = fma(r, p, 1.0);
  p *= r;
  // the low 52 bits of t hold 2^51 + N
  const long long n = (__double_as_longlong(t) & 0xFFFFFFFFFFFFFLL) - (1LL << 51);
  const int j = (int)(n & 63);
  const long long m = (n - j) >> 6;
  const double S = __ldg(&g_exp2_64[j]);
  const double y = fma(S, p, S);
  return __longlong_as_double(__double_as_longlong(y) + (m << 52));
}

struct ReactionInit {
  int nr, r0, r1, np, p0, p1, p2, third;
  double A_cgs, n, theta;
  int tf, tb, effset;
};
// host-side initialiser table (copied to c_reactions by the library at load time)
static constexpr ReactionInit kReactionInit[21] = {
    {1, 0, -1, 2, 3, 3, -1, 1, 7.0e21, -1.6, 113200.0, TK_A, TK_T, 1},
    {1, 1, -1, 2, 4, 4, -1, 1, 2.0e21, -1.5, 59500.0, TK_A, TK_T, 2},
    {1, 2, -1, 2, 3, 4, -1, 1, 5.0e15, 0.0, 75500.0, TK_A, TK_T, 3},
    {2, 0, 4, 2, 2, 3, -1, 0, 6.4e17, -1.0, 38400.0, TK_T, TK_T, 0},
    {2, 2, 4, 2, 1, 3, -1, 0, 8.4e12, 0.0, 19450.0, TK_T, TK_T, 0},
    {2, 3, 4, 2, 5, 10, -1, 0, 8.8e8, 1.0, 31900.0, TK_T, TK_T, 0},
    {2, 4, 4, 2, 7, 10, -1, 0, 7.1e2, 2.7, 80600.0, TK_T, TK_T, 0},
    {2, 3, 3, 2, 6, 10, -1, 0, 4.4e7, 1.5, 67500.0, TK_T, TK_T, 0},
    {2, 5, 4, 2, 8, 1, -1, 0, 1.0e12, 0.5, 77200.0, TK_T, TK_T, 0},
    {2, 8, 0, 2, 6, 3, -1, 0, 1.0e12, 0.5, 12200.0, TK_T, TK_T, 0},
    {2, 7, 3, 2, 8, 1, -1, 0, 8.7e13, 0.14, 28600.0, TK_T, TK_T, 0},
    {2, 9, 2, 2, 8, 1, -1, 0, 1.4e5, 1.9, 26600.0, TK_T, TK_T, 0},
    {2, 7, 0, 2, 6, 1, -1, 0, 9.9e12, 0.0, 40700.0, TK_T, TK_T, 0},
    {2, 7, 4, 2, 9, 1, -1, 0, 4.0e12, -0.09, 18000.0, TK_T, TK_T, 0},
    {2, 5, 3, 2, 9, 0, -1, 0, 3.4e13, -1.08, 12800.0, TK_T, TK_T, 0},
    {2, 5, 1, 2, 7, 2, -1, 0, 2.4e13, 0.41, 32600.0, TK_T, TK_T, 0},
    {2, 5, 4, 2, 7, 3, -1, 0, 7.2e12, 0.29, 48600.0, TK_T, TK_T, 0},
    {2, 9, 0, 2, 6, 4, -1, 0, 9.1e11, 0.36, 22800.0, TK_T, TK_T, 0},
    {2, 5, 3, 2, 6, 4, -1, 0, 7.2e13, 0.0, 35500.0, TK_T, TK_T, 0},
    {2, 4, 10, 3, 9, 10, 10, 0, 3.9e33, -3.78, 158500.0, TK_V, TK_V, 0},
    {2, 3, 10, 3, 8, 10, 10, 0, 2.5e34, -3.82, 168600.0, TK_V, TK_V, 0},
};

// Compile-time view of the same reaction table (structure only; the numbers lnA, n, theta and
// the efficiencies come from c_reactions): lets the kernels unroll the reaction loop so that
// every per-species index is a compile-time constant.
struct RxShape {
  int nr, r0, r1, np, p0, p1, p2, third, tf, tb;
};
__host__ __device__ constexpr RxShape rx_shape(int r) {
  return RxShape{kReactionInit[r].nr, kReactionInit[r].r0, kReactionInit[r].r1,
                 kReactionInit[r].np, kReactionInit[r].p0, kReactionInit[r].p1,
                 kReactionInit[r].p2, kReactionInit[r].third, kReactionInit[r].tf,
                 kReactionInit[r].tb};
}
// net stoichiometric coefficient of species s in reaction r
__host__ __device__ constexpr int rx_nu(int r, int s) {
  const RxShape x = rx_shape(r);
  return (x.p0 == s) + (x.np > 1 && x.p1 == s) + (x.np > 2 && x.p2 == s) - (x.r0 == s) -
         (x.nr > 1 && x.r1 == s);
}

// Compile-time description of one gas model.
template <int NS_, int NTEMP_, int NR_, bool PERFECT_ = false>
struct Gas {
  static constexpr int NS = NS_, NTEMP = NTEMP_, NR = NR_;
  static constexpr bool PERFECT = PERFECT_;
  __device__ static const SpeciesData& sp(int s) {
    return PERFECT ? c_species_perfect[0] : c_species_air[s];
  }
};
using GasPerfect = Gas<1, 1, 0, true>;
using GasAir5 = Gas<5, 1, 5>;
using GasAir11 = Gas<11, 2, 21>;

// ---- species thermodynamics -------------------------------------------------------------

template <class G>
__device__ __forceinline__ double Rs(int s) { return c_gas.Rs[s]; }

// trans(-rot) heat capacity per unit mass
template <class G>
__device__ __forceinline__ double cvtr(int s) {
  const int k = G::sp(s).kind;
  if (k == DIATOMIC) return 2.5 * Rs<G>(s);
  if (k == ATOM) return 1.5 * Rs<G>(s);
  return G::NTEMP == 1 ? 1.5 * Rs<G>(s) : 0.0;
}

// Harmonic-oscillator energy and heat capacity per unit mass at temperature 1/iT: one exp and
// one reciprocal (R theta em / (1 - em), R x^2 em / (1 - em)^2 with x = theta/T, em = e^-x);
// em is returned too (0 for a species without vibration).
template <class G>
__device__ __forceinline__ void vib_it(int s, double iT, double& e, double& cv, double& em) {
  const SpeciesData& d = G::sp(s);
  if (d.kind != DIATOMIC || d.thv <= 0.0) { e = 0.0; cv = 0.0; em = 0.0; return; }
  const double x = d.thv * iT;
  em = exp_tab(-x);
  const double r = 1.0 / (1.0 - em);
  const double Rem = c_gas.Rs[s] * em * r;
  e = Rem * d.thv;
  cv = Rem * x * x * r;
}
template <class G>
__device__ __forceinline__ void vib(int s, double T, double& e, double& cv) {
  double em;
  vib_it<G>(s, 1.0 / T, e, cv, em);
}

template <class G>
__device__ __forceinline__ double hf(int s) { return c_gas.hf[s]; }

}  // namespace cs
