/*
 * FP64 CPU oracle of one pseudo-time iteration of the component-splitting (CS) and coupled
 * (CI) implicit LU-SGS scheme for multicomponent reacting Navier-Stokes flow
 * (Zhang, Cai & Pan, arXiv:2403.03440, Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct restatement of
 * the method that the CUDA library is checked against.  It shares no code, header, table or
 * helper with the CUDA path; only tests, the smoke check and the CPU-baseline leg of the
 * benchmark may build, load or call it.
 *
 * Every function names the passage of the paper it follows.  Where the paper is silent or
 * garbled, the reading taken is stated at the function.
 *
 * Units: SI, dimensional finite volume (Ma/Re == 1); 2D grids have unit depth.
 * Layout: cell c = i + ni*(j + nj*k); conserved state Q is struct-of-arrays [var][cell] with
 * var = rho_1..rho_ns, m_1..m_d, rhoE, [rho*e_v] (two-temperature models only).
 *
 * Parity pins: see tests/test_oracle_*.py.  Functions with no independent pin say so.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define NSMAX 12
#define NRMAX 24
#define NQMAX 18            /* ns + 3 + 1 + 1 */
#define NGMAX (3 + 2 + NSMAX)

/* ---------------------------------------------------------------------------------------
 * Physical constants (CODATA exact SI values).
 * ------------------------------------------------------------------------------------- */
static const double RU = 8314.462618;        /* J/(kmol K)   universal gas constant */
static const double KB = 1.380649e-23;       /* J/K          Boltzmann */
static const double HPL = 6.62607015e-34;    /* J s          Planck */
static const double NAV = 6.02214076e26;     /* 1/kmol       Avogadro */
static const double PREF = 101325.0;         /* Pa           standard-state pressure */
static const double PI = 3.14159265358979323846;

/* Transport model constants (reading: paper Sec. 2.1 defers transport to its references). */
static const double SUTH_MU0 = 1.458e-6, SUTH_TS = 110.4;   /* Sutherland, air */
static const double PRANDTL = 0.72, SCHMIDT = 0.5;

/* Temperature solve bracket [K] */
static const double TMIN = 20.0, TMAX = 1.0e5;

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_FARFIELD = 2, BC_OUTFLOW = 3, BC_AXIS = 4 };
enum { KIND_ATOM = 0, KIND_DIATOMIC = 1, KIND_ELECTRON = 2 };
enum { TEMP_T = 0, TEMP_A = 1, TEMP_V = 2 };   /* T, sqrt(T*Tv), Tv */

/* ---------------------------------------------------------------------------------------
 * Gas model tables.  Values are standard spectroscopic/thermochemical constants (rounded)
 * and Park's air rates; they are inputs of the model, not part of the method.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    const char *name;
    int kind;              /* atom / diatomic / electron */
    int nN, nO, charge;    /* element composition -> molar mass */
    double thv;            /* characteristic vibrational temperature [K] (0: none) */
    double thr;            /* characteristic rotational temperature [K] */
    double sigma;          /* rotational symmetry number */
    double g0;             /* ground electronic degeneracy */
    double h0_molar;       /* formation energy at 0 K [J/kmol] */
} species_t;

typedef struct {
    int nreac, reac[3];    /* reactant species (repeated for stoichiometry 2) */
    int nprod, prod[3];
    int third;             /* 1: third-body reaction with efficiencies eff[] */
    double A_cgs;          /* cm^3/(mol s), bimolecular forward */
    double n, theta;       /* temperature exponent, activation temperature [K] */
    int tf, tb;            /* rate-controlling temperature, forward / backward */
    double eff[NSMAX];     /* third-body efficiency relative to A */
} reaction_t;

static const double M_N = 14.0067, M_O = 15.9994, M_E = 5.48579909e-4;

/* Perfect diatomic gas with air's molar mass and no vibration (tests). */
static const species_t SP_PERFECT[1] = {
    {"A2", KIND_DIATOMIC, 0, 0, 0, 0.0, 2.88, 2, 1, 0.0},
};
static const species_t SP_AIR11[11] = {
    {"N2", KIND_DIATOMIC, 2, 0, 0, 3395.0, 2.88, 2, 1, 0.0},
    {"O2", KIND_DIATOMIC, 0, 2, 0, 2239.0, 2.08, 2, 3, 0.0},
    {"NO", KIND_DIATOMIC, 1, 1, 0, 2817.0, 2.45, 1, 4, 89.77e6},
    {"N", KIND_ATOM, 1, 0, 0, 0.0, 0.0, 1, 4, 470.82e6},
    {"O", KIND_ATOM, 0, 1, 0, 0.0, 0.0, 1, 9, 246.79e6},
    {"NO+", KIND_DIATOMIC, 1, 1, 1, 3419.0, 2.87, 1, 1, 983.6e6},
    {"N2+", KIND_DIATOMIC, 2, 0, 1, 3175.0, 2.78, 2, 2, 1503.3e6},
    {"O2+", KIND_DIATOMIC, 0, 2, 1, 2741.0, 2.43, 2, 4, 1164.5e6},
    {"N+", KIND_ATOM, 1, 0, 1, 0.0, 0.0, 1, 9, 1873.1e6},
    {"O+", KIND_ATOM, 0, 1, 1, 0.0, 0.0, 1, 4, 1560.7e6},
    {"e-", KIND_ELECTRON, 0, 0, -1, 0.0, 0.0, 1, 2, 0.0},
};

/* species indices */
enum { S_N2 = 0, S_O2, S_NO, S_N, S_O, S_NOp, S_N2p, S_O2p, S_Np, S_Op, S_E };

/* Park's air reactions (forward rate A T^n exp(-theta/T), cm^3/mol/s).  Efficiencies are
 * A(partner)/A for the dissociation reactions. */
#define EFF_N2 {1, 1, 1, 30.0/7.0, 30.0/7.0, 1, 1, 1, 30.0/7.0, 30.0/7.0, 3.0e24/7.0e21}
#define EFF_O2 {1, 1, 1, 5, 5, 1, 1, 1, 5, 5, 0}
#define EFF_NO {1, 1, 22, 22, 22, 1, 1, 1, 22, 22, 0}
static const reaction_t RX_AIR[21] = {
    {1, {S_N2}, 2, {S_N, S_N}, 1, 7.0e21, -1.6, 113200.0, TEMP_A, TEMP_T, EFF_N2},
    {1, {S_O2}, 2, {S_O, S_O}, 1, 2.0e21, -1.5, 59500.0, TEMP_A, TEMP_T, EFF_O2},
    {1, {S_NO}, 2, {S_N, S_O}, 1, 5.0e15, 0.0, 75500.0, TEMP_A, TEMP_T, EFF_NO},
    {2, {S_N2, S_O}, 2, {S_NO, S_N}, 0, 6.4e17, -1.0, 38400.0, TEMP_T, TEMP_T, {0}},
    {2, {S_NO, S_O}, 2, {S_O2, S_N}, 0, 8.4e12, 0.0, 19450.0, TEMP_T, TEMP_T, {0}},
    {2, {S_N, S_O}, 2, {S_NOp, S_E}, 0, 8.8e8, 1.0, 31900.0, TEMP_T, TEMP_T, {0}},
    {2, {S_O, S_O}, 2, {S_O2p, S_E}, 0, 7.1e2, 2.7, 80600.0, TEMP_T, TEMP_T, {0}},
    {2, {S_N, S_N}, 2, {S_N2p, S_E}, 0, 4.4e7, 1.5, 67500.0, TEMP_T, TEMP_T, {0}},
    {2, {S_NOp, S_O}, 2, {S_Np, S_O2}, 0, 1.0e12, 0.5, 77200.0, TEMP_T, TEMP_T, {0}},
    {2, {S_Np, S_N2}, 2, {S_N2p, S_N}, 0, 1.0e12, 0.5, 12200.0, TEMP_T, TEMP_T, {0}},
    {2, {S_O2p, S_N}, 2, {S_Np, S_O2}, 0, 8.7e13, 0.14, 28600.0, TEMP_T, TEMP_T, {0}},
    {2, {S_Op, S_NO}, 2, {S_Np, S_O2}, 0, 1.4e5, 1.9, 26600.0, TEMP_T, TEMP_T, {0}},
    {2, {S_O2p, S_N2}, 2, {S_N2p, S_O2}, 0, 9.9e12, 0.0, 40700.0, TEMP_T, TEMP_T, {0}},
    {2, {S_O2p, S_O}, 2, {S_Op, S_O2}, 0, 4.0e12, -0.09, 18000.0, TEMP_T, TEMP_T, {0}},
    {2, {S_NOp, S_N}, 2, {S_Op, S_N2}, 0, 3.4e13, -1.08, 12800.0, TEMP_T, TEMP_T, {0}},
    {2, {S_NOp, S_O2}, 2, {S_O2p, S_NO}, 0, 2.4e13, 0.41, 32600.0, TEMP_T, TEMP_T, {0}},
    {2, {S_NOp, S_O}, 2, {S_O2p, S_N}, 0, 7.2e12, 0.29, 48600.0, TEMP_T, TEMP_T, {0}},
    {2, {S_Op, S_N2}, 2, {S_N2p, S_O}, 0, 9.1e11, 0.36, 22800.0, TEMP_T, TEMP_T, {0}},
    {2, {S_NOp, S_N}, 2, {S_N2p, S_O}, 0, 7.2e13, 0.0, 35500.0, TEMP_T, TEMP_T, {0}},
    {2, {S_O, S_E}, 3, {S_Op, S_E, S_E}, 0, 3.9e33, -3.78, 158500.0, TEMP_V, TEMP_V, {0}},
    {2, {S_N, S_E}, 3, {S_Np, S_E, S_E}, 0, 2.5e34, -3.82, 168600.0, TEMP_V, TEMP_V, {0}},
};

typedef struct {
    int mech, ns, nr, ntemp;        /* ntemp = 1 (one temperature) or 2 (T, Tv) */
    int transport;                  /* 0: Sutherland, constant Pr and Sc; 1: species model */
    species_t sp[NSMAX];
    double M[NSMAX], Rs[NSMAX], hf[NSMAX];   /* kg/kmol, J/(kg K), J/kg */
    reaction_t rx[NRMAX];
    double nu[NRMAX][NSMAX];        /* net stoichiometric coefficient nu'' - nu' */
    int nuf[NRMAX][NSMAX], nub[NRMAX][NSMAX];
} gas_t;

static int gas_init(gas_t *g, int mech)
{
    memset(g, 0, sizeof(*g));
    g->mech = mech;
    const species_t *sp;
    if (mech == 0) { sp = SP_PERFECT; g->ns = 1; g->nr = 0; g->ntemp = 1; }
    else if (mech == 1) { sp = SP_AIR11; g->ns = 5; g->nr = 5; g->ntemp = 1; }
    else if (mech == 2) { sp = SP_AIR11; g->ns = 11; g->nr = 21; g->ntemp = 2; }
    else return 1;
    for (int s = 0; s < g->ns; s++) {
        g->sp[s] = sp[s];
        if (mech == 0) g->M[s] = 28.9647;
        else g->M[s] = sp[s].nN * M_N + sp[s].nO * M_O - sp[s].charge * M_E;
        g->Rs[s] = RU / g->M[s];
        g->hf[s] = sp[s].h0_molar / g->M[s];
    }
    for (int r = 0; r < g->nr; r++) {
        g->rx[r] = RX_AIR[r];
        for (int a = 0; a < g->rx[r].nreac; a++) g->nuf[r][g->rx[r].reac[a]]++;
        for (int a = 0; a < g->rx[r].nprod; a++) g->nub[r][g->rx[r].prod[a]]++;
        for (int s = 0; s < g->ns; s++) g->nu[r][s] = g->nub[r][s] - g->nuf[r][s];
    }
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * Thermodynamics (Sec. 2.1: e_t, e_v, ideal-gas p).  Reading: rigid-rotor harmonic-oscillator
 * species, electronic excitation neglected; in the two-temperature model the trans-rotational
 * energy is at T and the vibrational energy and the electrons' translational energy form the
 * vibrational-electronic pool at Tv.
 * ------------------------------------------------------------------------------------- */
static int is_heavy(const gas_t *g, int s) { return g->sp[s].kind != KIND_ELECTRON; }

/* trans(-rot) specific heat at constant volume of species s [J/(kg K)] */
static double cv_tr(const gas_t *g, int s)
{
    if (g->sp[s].kind == KIND_DIATOMIC) return 2.5 * g->Rs[s];
    if (g->sp[s].kind == KIND_ATOM) return 1.5 * g->Rs[s];
    return g->ntemp == 1 ? 1.5 * g->Rs[s] : 0.0;   /* electron: in the pool for 2T */
}

/* vibrational energy of a harmonic oscillator, per unit mass: R theta / (exp(theta/T) - 1) */
static double e_vib(const gas_t *g, int s, double T)
{
    if (g->sp[s].kind != KIND_DIATOMIC || g->sp[s].thv <= 0.0) return 0.0;
    double x = g->sp[s].thv / T;
    return g->Rs[s] * g->sp[s].thv / expm1(x);
}

/* d e_vib / dT */
static double cv_vib(const gas_t *g, int s, double T)
{
    if (g->sp[s].kind != KIND_DIATOMIC || g->sp[s].thv <= 0.0) return 0.0;
    double x = g->sp[s].thv / T;
    double em = exp(-x), d = -expm1(-x);
    return g->Rs[s] * x * x * em / (d * d);
}

/* energy of species s in the vibrational-electronic pool at Tv (2T only) */
static double e_pool(const gas_t *g, int s, double Tv)
{
    if (g->sp[s].kind == KIND_ELECTRON) return 1.5 * g->Rs[s] * Tv;
    return e_vib(g, s, Tv);
}
static double cv_pool(const gas_t *g, int s, double Tv)
{
    if (g->sp[s].kind == KIND_ELECTRON) return 1.5 * g->Rs[s];
    return cv_vib(g, s, Tv);
}

/* species specific internal energy e_s(T, Tv), including formation energy */
static double e_species(const gas_t *g, int s, double T, double Tv)
{
    if (g->ntemp == 1) return cv_tr(g, s) * T + e_vib(g, s, T) + g->hf[s];
    return cv_tr(g, s) * T + e_pool(g, s, Tv) + g->hf[s];
}

/* species specific enthalpy h_s = e_s + p_s/rho_s */
static double h_species(const gas_t *g, int s, double T, double Tv)
{
    double pT = (g->ntemp == 2 && !is_heavy(g, s)) ? Tv : T;
    return e_species(g, s, T, Tv) + g->Rs[s] * pT;
}

/* Solve f(T) = target for monotone increasing f by safeguarded Newton in [TMIN, TMAX].
 * Returns 0 on convergence (|dT| <= 1e-12 T), 1 otherwise; result clamped to the bracket. */
typedef double (*energy_fn)(const gas_t *, const double *Y, double T, double *dfdT);

static double mix_e_1T(const gas_t *g, const double *Y, double T, double *cv)
{
    double e = 0.0, c = 0.0;
    for (int s = 0; s < g->ns; s++) {
        e += Y[s] * e_species(g, s, T, T);
        c += Y[s] * (cv_tr(g, s) + cv_vib(g, s, T));
    }
    *cv = c;
    return e;
}
static double mix_e_pool(const gas_t *g, const double *Y, double Tv, double *cv)
{
    double e = 0.0, c = 0.0;
    for (int s = 0; s < g->ns; s++) {
        e += Y[s] * e_pool(g, s, Tv);
        c += Y[s] * cv_pool(g, s, Tv);
    }
    *cv = c;
    return e;
}

static int solve_T(const gas_t *g, energy_fn f, const double *Y, double target, double guess,
                   double *Tout)
{
    double lo = TMIN, hi = TMAX, d;
    if (f(g, Y, lo, &d) >= target) { *Tout = lo; return 0; }
    if (f(g, Y, hi, &d) <= target) { *Tout = hi; return 1; }
    double T = (guess > lo && guess < hi) ? guess : 1000.0;
    for (int it = 0; it < 200; it++) {
        double dfdT, fv = f(g, Y, T, &dfdT) - target;
        if (fv > 0) hi = T; else lo = T;
        double Tn = (dfdT > 0) ? T - fv / dfdT : 0.5 * (lo + hi);
        if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
        if (fabs(Tn - T) <= 1e-12 * T) { *Tout = Tn; return 0; }
        T = Tn;
    }
    *Tout = T;
    return 1;
}

/* ---------------------------------------------------------------------------------------
 * Per-cell primitive / auxiliary state.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    double rhos[NSMAX], Y[NSMAX], rho, u[3], T, Tv, p, c, beta;
    double rhoE, rhoev, ev, H, Gam;            /* Gam = rho*e/p, rho*e = rhoE - rho|u|^2/2 */
    double prs[NSMAX], prev;                   /* dp/drho_s, dp/d(rho e_v) */
    double cvtr, cvve, cv;                     /* per unit mass */
    double mu, kt, kv, rhoD;                   /* rhoD: the largest species rho D_s */
    double rhoDs[NSMAX];                       /* effective diffusion rho D_s per species */
    double hs[NSMAX], eve[NSMAX];              /* species enthalpy and pool energy */
    double omega[NSMAX], omega_v, dom[NSMAX];  /* chemistry source and d omega_s/d rho_s */
    double relax;                              /* -d omega_v / d(rho e_v) */
    double tau[NSMAX];                         /* vibrational relaxation times */
} prim_t;

/* ---------------------------------------------------------------------------------------
 * Species transport model (Sec. 2.1 defers viscosity, conductivity and the effective
 * diffusion coefficient D_s of each species to its references).  Reading, in this order:
 *  1. species viscosity from Blottner's curve fits mu_s = 0.1 exp((A ln T + B) ln T + C)
 *     kg/(m s) (Blottner, Johnson & Ellis, Sandia report SC-RR-70-754, 1971); the four other
 *     ions take the fit given for NO+; heavy species at T, electrons at Tv;
 *  2. species conductivities from Eucken's relation: k_s = mu_s (5/2 c_v,t + c_v,r + c_v,v),
 *     split in the two-temperature model into k_tr,s = mu_s (5/2 c_v,t + c_v,r) and
 *     k_ve,s = mu_s c_v,v(Tv); electrons k_e = mu_e 5/2 c_v,t,e (all in the pool);
 *  3. mixture values by Wilke's rule: phi_s = sum_r X_r (1 + sqrt(mu_s/mu_r)(M_r/M_s)^(1/4))^2
 *     / sqrt(8 (1 + M_s/M_r)), mu = sum_s X_s mu_s / phi_s, likewise k_tr and k_ve;
 *  4. binary diffusion coefficients of hard spheres in the first Chapman-Enskog
 *     approximation, D_sr = 3/(8 n sigma_sr^2) sqrt(k T / (2 pi m_sr)), with each species'
 *     diameter from its Blottner viscosity, pi sigma_s^2 = (5/16) sqrt(pi m_s k T) / mu_s,
 *     sigma_sr = (sigma_s + sigma_r)/2, m_sr the reduced mass, n the number density, T the
 *     heavy-particle temperature;
 *  5. effective coefficient of each heavy species in the mixture by Blanc's law,
 *     D_s = (1 - X_s) / sum_{r != s, heavy} X_r / D_sr (the self-diffusion coefficient D_ss
 *     where the species is (nearly) alone); electrons carry no Fick flux of their own: their
 *     flux follows the ions' (no net charge flux, see the viscous flux).
 * ------------------------------------------------------------------------------------- */
static const double BLOTTNER[11][3] = {
    {0.0268142, 0.3177838, -11.3155513},   /* N2 */
    {0.0449290, -0.0826158, -9.2019475},   /* O2 */
    {0.0436378, -0.0335511, -9.5767430},   /* NO */
    {0.0115572, 0.6031679, -12.4327495},   /* N */
    {0.0203144, 0.4294404, -11.6031403},   /* O */
    {0.3020141, -3.5039791, -3.7355157},   /* NO+ */
    {0.3020141, -3.5039791, -3.7355157},   /* N2+ (fit of NO+) */
    {0.3020141, -3.5039791, -3.7355157},   /* O2+ (fit of NO+) */
    {0.3020141, -3.5039791, -3.7355157},   /* N+ (fit of NO+) */
    {0.3020141, -3.5039791, -3.7355157},   /* O+ (fit of NO+) */
    {0.0, 0.0, -12.5},                     /* e- */
};

static void species_transport(const gas_t *g, prim_t *w)
{
    int ns = g->ns;
    double T = w->T, Tv = w->Tv;
    double mus[NSMAX], ktr[NSMAX], kve[NSMAX], X[NSMAX], sig[NSMAX], m[NSMAX];
    double xs = 0.0, n = 0.0;
    for (int s = 0; s < ns; s++) {
        double Ts = is_heavy(g, s) ? T : Tv;
        double lnT = log(Ts);
        mus[s] = 0.1 * exp((BLOTTNER[s][0] * lnT + BLOTTNER[s][1]) * lnT + BLOTTNER[s][2]);
        double cvt = 1.5 * g->Rs[s], cvr = (g->sp[s].kind == KIND_DIATOMIC) ? g->Rs[s] : 0.0;
        if (!is_heavy(g, s)) {
            ktr[s] = 0.0;
            kve[s] = mus[s] * 2.5 * cvt;
        } else if (g->ntemp == 2) {
            ktr[s] = mus[s] * (2.5 * cvt + cvr);
            kve[s] = mus[s] * cv_vib(g, s, Tv);
        } else {
            ktr[s] = mus[s] * (2.5 * cvt + cvr + cv_vib(g, s, T));
            kve[s] = 0.0;
        }
        X[s] = w->Y[s] / g->M[s];
        xs += X[s];
        m[s] = g->M[s] / NAV;
        n += w->rhos[s] / m[s];
        sig[s] = sqrt((5.0 / 16.0) * sqrt(PI * m[s] * KB * Ts) / mus[s] / PI);
    }
    for (int s = 0; s < ns; s++) X[s] /= xs;
    double mu = 0.0, kt = 0.0, kv = 0.0;
    for (int s = 0; s < ns; s++) {
        double phi = 0.0;
        for (int r = 0; r < ns; r++) {
            double a = 1.0 + sqrt(mus[s] / mus[r]) * pow(g->M[r] / g->M[s], 0.25);
            phi += X[r] * a * a / sqrt(8.0 * (1.0 + g->M[s] / g->M[r]));
        }
        mu += X[s] * mus[s] / phi;
        kt += X[s] * ktr[s] / phi;
        kv += X[s] * kve[s] / phi;
    }
    w->mu = mu;
    w->kt = kt;
    w->kv = (g->ntemp == 2) ? kv : 0.0;
    w->rhoD = 0.0;
    for (int s = 0; s < ns; s++) {
        w->rhoDs[s] = 0.0;
        if (!is_heavy(g, s)) continue;
        double den = 0.0, Dss = 0.0;
        for (int r = 0; r < ns; r++) {
            if (!is_heavy(g, r)) continue;
            double sr = 0.5 * (sig[s] + sig[r]), mr = m[s] * m[r] / (m[s] + m[r]);
            double D = 3.0 / (8.0 * n * sr * sr) * sqrt(KB * T / (2.0 * PI * mr));
            if (r == s) Dss = D;
            else den += X[r] / D;
        }
        double D = (1.0 - X[s] > 1e-12 && den > 0.0) ? (1.0 - X[s]) / den : Dss;
        w->rhoDs[s] = w->rho * D;
        if (w->rhoDs[s] > w->rhoD) w->rhoD = w->rhoDs[s];
    }
}

/* Conserved -> primitive (Sec. 2.1, e_t / e_v definitions and ideal-gas law).  Tguess /
 * Tvguess <= 0 means "no previous value".  Returns 0, or 2 for a non-physical state, or 3 for
 * a temperature solve that did not converge. */
static int prim_from_cons(const gas_t *g, int nd, const double *q, double Tguess,
                          double Tvguess, prim_t *w)
{
    int ns = g->ns;
    memset(w, 0, sizeof(*w));
    double rho = 0.0;
    for (int s = 0; s < ns; s++) {
        w->rhos[s] = q[s];
        if (q[s] < 0.0) return 2;
        rho += q[s];
    }
    if (!(rho > 0.0)) return 2;
    w->rho = rho;
    for (int s = 0; s < ns; s++) w->Y[s] = w->rhos[s] / rho;
    double ke = 0.0;
    for (int d = 0; d < nd; d++) {
        w->u[d] = q[ns + d] / rho;
        ke += 0.5 * w->u[d] * w->u[d];
    }
    w->rhoE = q[ns + nd];
    double rhoe = w->rhoE - rho * ke;          /* internal energy incl. formation */
    int st = 0;
    if (g->ntemp == 1) {
        double T;
        st = solve_T(g, mix_e_1T, w->Y, rhoe / rho, Tguess, &T);
        w->T = w->Tv = T;
    } else {
        w->rhoev = q[ns + nd + 1];
        w->ev = w->rhoev / rho;
        double Tv;
        st = solve_T(g, mix_e_pool, w->Y, w->ev, Tvguess > 0 ? Tvguess : Tguess, &Tv);
        w->Tv = Tv;
        double etr = rhoe - w->rhoev, cvt = 0.0;
        for (int s = 0; s < ns; s++) {
            etr -= w->rhos[s] * g->hf[s];
            cvt += w->rhos[s] * cv_tr(g, s);
        }
        /* trans-rotational temperature is explicit; it is floored at TMIN like the
         * temperature solves (start-up transients can overshoot the energy) */
        w->T = etr / cvt;
        if (!(w->T > TMIN)) w->T = TMIN;
    }
    if (st) return 3;
    double T = w->T, Tv = w->Tv;
    /* pressure: heavy particles at T, electrons at Tv */
    double p = 0.0, Rh = 0.0;
    for (int s = 0; s < ns; s++) {
        if (g->ntemp == 2 && !is_heavy(g, s)) p += w->rhos[s] * g->Rs[s] * Tv;
        else { p += w->rhos[s] * g->Rs[s] * T; Rh += w->Y[s] * g->Rs[s]; }
    }
    w->p = p;
    /* specific heats */
    double cvtr = 0.0, cvve = 0.0, cv = 0.0;
    for (int s = 0; s < ns; s++) {
        cvtr += w->Y[s] * cv_tr(g, s);
        if (g->ntemp == 2) cvve += w->Y[s] * cv_pool(g, s, Tv);
        else cv += w->Y[s] * (cv_tr(g, s) + cv_vib(g, s, T));
    }
    w->cvtr = cvtr; w->cvve = cvve; w->cv = cv;
    /* beta = dp/d(rhoE) at fixed other conserved variables */
    double beta = (g->ntemp == 2) ? Rh / cvtr : Rh / cv;
    w->beta = beta;
    /* pressure derivatives (exact, from p(Q)) */
    double pe_fac = 0.0;   /* rho_e R_e / (rho cvve) */
    if (g->ntemp == 2) {
        for (int s = 0; s < ns; s++)
            if (!is_heavy(g, s)) pe_fac += w->rhos[s] * g->Rs[s];
        pe_fac = (cvve > 0.0) ? pe_fac / (rho * cvve) : 0.0;
        w->prev = -beta + pe_fac;
    }
    for (int s = 0; s < ns; s++) {
        if (g->ntemp == 1) {
            w->prs[s] = g->Rs[s] * T + beta * (ke - e_species(g, s, T, T));
        } else {
            double v = beta * (ke - g->hf[s] - cv_tr(g, s) * T) - pe_fac * e_pool(g, s, Tv);
            v += is_heavy(g, s) ? g->Rs[s] * T : g->Rs[s] * Tv;
            w->prs[s] = v;
        }
    }
    w->c = sqrt((1.0 + beta) * p / rho);
    w->H = (w->rhoE + p) / rho;
    w->Gam = rhoe / p;
    for (int s = 0; s < ns; s++) {
        w->hs[s] = h_species(g, s, T, Tv);
        w->eve[s] = (g->ntemp == 2) ? (is_heavy(g, s) ? e_pool(g, s, Tv)
                                                     : 2.5 * g->Rs[s] * Tv) : 0.0;
    }
    if (g->transport == 1) {
        species_transport(g, w);
        return 0;
    }
    /* transport (reading: Sutherland viscosity, constant Prandtl and Schmidt numbers) */
    w->mu = SUTH_MU0 * T * sqrt(T) / (T + SUTH_TS);
    if (g->ntemp == 2) {
        w->kt = w->mu * (cvtr + Rh) / PRANDTL;
        w->kv = w->mu * cvve / PRANDTL;
    } else {
        w->kt = w->mu * (cv + Rh) / PRANDTL;
        w->kv = 0.0;
    }
    w->rhoD = w->mu / SCHMIDT;
    for (int s = 0; s < ns; s++) w->rhoDs[s] = w->rhoD;
    return 0;
}

/* Primitive -> conserved (used to build initial states and ghost states). */
static void cons_from_prim(const gas_t *g, int nd, const double *rhos, const double *u,
                           double T, double Tv, double *q)
{
    int ns = g->ns;
    double rho = 0.0, rhoe = 0.0, rhoev = 0.0;
    for (int s = 0; s < ns; s++) {
        q[s] = rhos[s];
        rho += rhos[s];
        rhoe += rhos[s] * e_species(g, s, T, Tv);
        if (g->ntemp == 2) rhoev += rhos[s] * e_pool(g, s, Tv);
    }
    double ke = 0.0;
    for (int d = 0; d < nd; d++) {
        q[ns + d] = rho * u[d];
        ke += 0.5 * u[d] * u[d];
    }
    q[ns + nd] = rhoe + rho * ke;
    if (g->ntemp == 2) q[ns + nd + 1] = rhoev;
}

/* ---------------------------------------------------------------------------------------
 * Finite-rate chemistry (Sec. 2.1 source S; Park's air model, Sec. 3.2).
 * Reading: mass-action law; backward rate k_b = k_f / K_c with K_c from the species'
 * rigid-rotor harmonic-oscillator Gibbs energies (the paper does not state K_c).
 * ------------------------------------------------------------------------------------- */

/* dimensionless molar Gibbs energy g_s/(R_u T) at the standard pressure, written as
 * H/(R_u T) - S/R_u from the species' partition functions */
static double gibbs_RT(const gas_t *g, int s, double T)
{
    const species_t *sp = &g->sp[s];
    double m = g->M[s] / NAV;                       /* particle mass [kg] */
    double Htr = 2.5, Str;                          /* translational: H = 5/2 RT */
    double lam = 2.0 * PI * m * KB * T / (HPL * HPL);
    Str = 2.5 + log(pow(lam, 1.5) * KB * T / PREF);  /* Sackur-Tetrode */
    double Hrot = 0.0, Srot = 0.0, Hvib = 0.0, Svib = 0.0;
    if (sp->kind == KIND_DIATOMIC) {
        Hrot = 1.0;
        Srot = log(T / (sp->sigma * sp->thr)) + 1.0;
        if (sp->thv > 0.0) {
            double x = sp->thv / T;
            Hvib = x / expm1(x);
            Svib = x / expm1(x) - log(-expm1(-x));
        }
    }
    double Sel = log(sp->g0);
    double H = Htr + Hrot + Hvib + sp->h0_molar / (RU * T);
    double S = Str + Srot + Svib + Sel;
    return H - S;
}

/* dimensionless molar enthalpy H_s/(R_u T), including the formation energy */
static double enthalpy_RT(const gas_t *g, int s, double T)
{
    const species_t *sp = &g->sp[s];
    double H = 2.5 + sp->h0_molar / (RU * T);
    if (sp->kind == KIND_DIATOMIC) {
        H += 1.0;
        if (sp->thv > 0.0) { double x = sp->thv / T; H += x / expm1(x); }
    }
    return H;
}

/* d ln K_c / dT = Delta H / (R_u T^2) - Delta nu / T (Gibbs-Helmholtz) */
static double dlnKc_dT(const gas_t *g, int r, double T)
{
    double sh = 0.0, dn = 0.0;
    for (int s = 0; s < g->ns; s++)
        if (g->nu[r][s] != 0.0) { sh += g->nu[r][s] * enthalpy_RT(g, s, T); dn += g->nu[r][s]; }
    return sh / T - dn / T;
}

/* ln K_c of reaction r at temperature T (concentrations in kmol/m^3) */
static double lnKc(const gas_t *g, int r, double T)
{
    double sg = 0.0, dn = 0.0;
    for (int s = 0; s < g->ns; s++) {
        if (g->nu[r][s] != 0.0) {
            sg += g->nu[r][s] * gibbs_RT(g, s, T);
            dn += g->nu[r][s];
        }
    }
    return -sg + dn * log(PREF / (RU * T));
}

static double temp_of(int type, double T, double Tv)
{
    if (type == TEMP_A) return sqrt(T * Tv);
    if (type == TEMP_V) return Tv;
    return T;
}

/* forward and backward rate constants, SI (m^3/kmol/s for bimolecular) */
static void rate_constants(const gas_t *g, int r, double T, double Tv, double *kf, double *kb)
{
    const reaction_t *x = &g->rx[r];
    double lnA = log(x->A_cgs * 1e-3);
    double Tf = temp_of(x->tf, T, Tv), Tb = temp_of(x->tb, T, Tv);
    *kf = exp(lnA + x->n * log(Tf) - x->theta / Tf);
    *kb = exp(lnA + x->n * log(Tb) - x->theta / Tb - lnKc(g, r, Tb));
}

/* omega_s [kg/m^3/s], the Jacobian J[s][r] = d omega_s / d rho_r at fixed T, Tv, and the
 * temperature derivatives wT[s] = d omega_s/dT, wTv[s] = d omega_s/dTv at fixed rho_r */
static void chemistry_T(const gas_t *g, const double *rhos, double T, double Tv, double *omega,
                        double *J, double *wT, double *wTv)
{
    int ns = g->ns;
    double X[NSMAX];
    for (int s = 0; s < ns; s++) { X[s] = rhos[s] / g->M[s]; omega[s] = 0.0; }
    if (J) memset(J, 0, sizeof(double) * ns * ns);
    if (wT) for (int s = 0; s < ns; s++) { wT[s] = 0.0; wTv[s] = 0.0; }
    for (int r = 0; r < g->nr; r++) {
        const reaction_t *x = &g->rx[r];
        double kf, kb;
        rate_constants(g, r, T, Tv, &kf, &kb);
        /* d ln k / d(T, Tv) through the rate-controlling temperatures */
        double Tf = temp_of(x->tf, T, Tv), Tb = temp_of(x->tb, T, Tv);
        double dlf = x->n / Tf + x->theta / (Tf * Tf);
        double dlb = x->n / Tb + x->theta / (Tb * Tb) - dlnKc_dT(g, r, Tb);
        double fT = (x->tf == TEMP_T) ? 1.0 : (x->tf == TEMP_A) ? 0.5 * Tf / T : 0.0;
        double fV = (x->tf == TEMP_V) ? 1.0 : (x->tf == TEMP_A) ? 0.5 * Tf / Tv : 0.0;
        double bT = (x->tb == TEMP_T) ? 1.0 : (x->tb == TEMP_A) ? 0.5 * Tb / T : 0.0;
        double bV = (x->tb == TEMP_V) ? 1.0 : (x->tb == TEMP_A) ? 0.5 * Tb / Tv : 0.0;
        double M = 1.0, dM[NSMAX];
        for (int s = 0; s < ns; s++) dM[s] = 0.0;
        if (x->third) {
            M = 0.0;
            for (int s = 0; s < ns; s++) { M += x->eff[s] * X[s]; dM[s] = x->eff[s]; }
        }
        /* products of concentrations and their derivatives d/dX_s */
        double Pf = 1.0, Pb = 1.0;
        for (int s = 0; s < ns; s++) {
            Pf *= pow(X[s], g->nuf[r][s]);
            Pb *= pow(X[s], g->nub[r][s]);
        }
        double Rf = kf * Pf * M, Rb = kb * Pb * M;
        for (int s = 0; s < ns; s++) omega[s] += g->M[s] * g->nu[r][s] * (Rf - Rb);
        if (wT) {
            double dT = Rf * dlf * fT - Rb * dlb * bT, dV = Rf * dlf * fV - Rb * dlb * bV;
            for (int s = 0; s < ns; s++) {
                wT[s] += g->M[s] * g->nu[r][s] * dT;
                wTv[s] += g->M[s] * g->nu[r][s] * dV;
            }
        }
        if (!J) continue;
        for (int q = 0; q < ns; q++) {
            /* d(Pf)/dX_q */
            double dPf = 0.0, dPb = 0.0;
            if (g->nuf[r][q] > 0) {
                dPf = g->nuf[r][q] * pow(X[q], g->nuf[r][q] - 1);
                for (int s = 0; s < ns; s++) if (s != q) dPf *= pow(X[s], g->nuf[r][s]);
            }
            if (g->nub[r][q] > 0) {
                dPb = g->nub[r][q] * pow(X[q], g->nub[r][q] - 1);
                for (int s = 0; s < ns; s++) if (s != q) dPb *= pow(X[s], g->nub[r][s]);
            }
            double dRf = kf * (dPf * M + Pf * dM[q]) / g->M[q];
            double dRb = kb * (dPb * M + Pb * dM[q]) / g->M[q];
            for (int s = 0; s < ns; s++) J[s * ns + q] += g->M[s] * g->nu[r][s] * (dRf - dRb);
        }
    }
}

static void chemistry(const gas_t *g, const double *rhos, double T, double Tv, double *omega,
                      double *J)
{
    chemistry_T(g, rhos, T, Tv, omega, J, NULL, NULL);
}

/* Derivatives of the temperatures with respect to the conserved variables of a cell, at fixed
 * other conserved variables (full layout rho_s, m, rhoE, [rho e_v]): dT[k], dTv[k]. */
static void temperature_derivatives(const gas_t *g, int nd, const prim_t *w, double *dT, double *dTv)
{
    int ns = g->ns, nq = ns + nd + 1 + (g->ntemp == 2);
    double ke = 0.0;
    for (int q = 0; q < nd; q++) ke += 0.5 * w->u[q] * w->u[q];
    for (int k = 0; k < nq; k++) { dT[k] = 0.0; dTv[k] = 0.0; }
    if (g->ntemp == 1) {
        double rc = w->rho * w->cv;
        for (int s = 0; s < ns; s++) dT[s] = (ke - e_species(g, s, w->T, w->T)) / rc;
        for (int q = 0; q < nd; q++) dT[ns + q] = -w->u[q] / rc;
        dT[ns + nd] = 1.0 / rc;
        for (int k = 0; k < nq; k++) dTv[k] = dT[k];
    } else {
        double rc = w->rho * w->cvtr, rv = w->rho * w->cvve;
        for (int s = 0; s < ns; s++) {
            dT[s] = (ke - g->hf[s] - cv_tr(g, s) * w->T) / rc;
            dTv[s] = (rv > 0.0) ? -e_pool(g, s, w->Tv) / rv : 0.0;
        }
        for (int q = 0; q < nd; q++) dT[ns + q] = -w->u[q] / rc;
        dT[ns + nd] = 1.0 / rc;
        dT[ns + nd + 1] = -1.0 / rc;
        dTv[ns + nd + 1] = (rv > 0.0) ? 1.0 / rv : 0.0;
    }
}

/* Source Jacobian in conserved variables (Sec. 2.2, A_S = dS/(J dQ)): Jq[s][k] =
 * d omega_s / d Q_k at fixed other conserved variables, k over the full layout. */
static void source_jacobian(const gas_t *g, int nd, const prim_t *w, double *omega, double *Jq)
{
    int ns = g->ns, nq = ns + nd + 1 + (g->ntemp == 2);
    double J[NSMAX * NSMAX], wT[NSMAX], wTv[NSMAX], dT[NQMAX], dTv[NQMAX];
    chemistry_T(g, w->rhos, w->T, w->Tv, omega, J, wT, wTv);
    temperature_derivatives(g, nd, w, dT, dTv);
    for (int s = 0; s < ns; s++)
        for (int k = 0; k < nq; k++) {
            double v = wT[s] * dT[k] + wTv[s] * dTv[k];   /* 1T: dTv == dT */
            if (k < ns) v += J[s * ns + k];
            Jq[s * nq + k] = v;
        }
}

/* Vibrational relaxation times (reading: Millikan-White with Park's high-temperature
 * correction; the paper names omega_v only). */
static void relaxation_times(const gas_t *g, const prim_t *w, double *tau)
{
    int ns = g->ns;
    double T = w->T, patm = 0.0, nden = 0.0, xsum = 0.0;
    double X[NSMAX];
    for (int s = 0; s < ns; s++) {
        X[s] = 0.0;
        if (!is_heavy(g, s)) continue;
        X[s] = w->rhos[s] / g->M[s];
        xsum += X[s];
        patm += w->rhos[s] * g->Rs[s] * T;
    }
    nden = xsum * NAV;                     /* heavy-particle number density [1/m^3] */
    patm /= PREF;
    for (int s = 0; s < ns; s++) {
        tau[s] = 0.0;
        if (g->sp[s].kind != KIND_DIATOMIC || g->sp[s].thv <= 0.0) continue;
        double num = 0.0, den = 0.0;
        for (int q = 0; q < ns; q++) {
            if (!is_heavy(g, q)) continue;
            double mu = g->M[s] * g->M[q] / (g->M[s] + g->M[q]);
            double A = 1.16e-3 * sqrt(mu) * pow(g->sp[s].thv, 4.0 / 3.0);
            double B = 0.015 * pow(mu, 0.25);
            double tsq = exp(A * (pow(T, -1.0 / 3.0) - B) - 18.42) / patm;
            num += X[q];
            den += X[q] / tsq;
        }
        double tmw = num / den;
        double cbar = sqrt(8.0 * RU * T / (PI * g->M[s]));
        double sigv = 1e-21 * (50000.0 / T) * (50000.0 / T);
        tau[s] = tmw + 1.0 / (nden * sigv * cbar);
    }
}

/* Chemistry + vibrational source of one cell, stored in the primitive record. */
static void cell_sources(const gas_t *g, int nd, prim_t *w)
{
    int ns = g->ns, nq = ns + nd + 1 + (g->ntemp == 2);
    double Jq[NSMAX * NQMAX];
    source_jacobian(g, nd, w, w->omega, Jq);
    for (int s = 0; s < ns; s++) w->dom[s] = Jq[s * nq + s];
    w->omega_v = 0.0;
    w->relax = 0.0;
    if (g->ntemp == 2) {
        /* Landau-Teller exchange + species created/destroyed at the pool energy.
         * relax = -d(Landau-Teller)/d(rho e_v) at fixed rho_s, momentum and rho E (the
         * conserved-variable derivative of the source Jacobian reading): raising rho e_v
         * raises Tv (d Tv = d(rho e_v)/(rho c_v,ve)) and, the total energy being fixed,
         * lowers T (d T = -d(rho e_v)/(rho c_v,tr)), so both the pool's and the equilibrium
         * energy's heat capacities enter; the temperature dependence of tau is left out. */
        relaxation_times(g, w, w->tau);
        double lt = 0.0, rc = 0.0, rcT = 0.0;
        for (int s = 0; s < ns; s++) {
            if (w->tau[s] > 0.0) {
                lt += w->rhos[s] * (e_vib(g, s, w->T) - e_vib(g, s, w->Tv)) / w->tau[s];
                rc += w->rhos[s] * cv_vib(g, s, w->Tv) / w->tau[s];
                rcT += w->rhos[s] * cv_vib(g, s, w->T) / w->tau[s];
            }
            double epool = is_heavy(g, s) ? e_vib(g, s, w->Tv) : 1.5 * g->Rs[s] * w->Tv;
            lt += w->omega[s] * epool;
        }
        w->omega_v = lt;
        w->relax = ((w->cvve > 0.0) ? rc / (w->rho * w->cvve) : 0.0) +
                   ((w->cvtr > 0.0) ? rcT / (w->rho * w->cvtr) : 0.0);
    }
}

/* ---------------------------------------------------------------------------------------
 * Grid and geometry (Sec. 2.2: curvilinear metrics and Jacobian J, in finite-volume form:
 * xi_x/J etc. are the face area vectors S, 1/J is the cell volume V).
 * ------------------------------------------------------------------------------------- */
typedef struct {
    gas_t gas;
    int nd, n[3], bc[6], limiter;
    double efix;
    int hcorr;                       /* H-correction of the entropy fix on/off */
    int viscous;                     /* viscous and diffusive fluxes (and radii) on/off */
    double update_limit;             /* largest relative density change per update (0: off) */
    int ncell, nf[3];                /* faces per direction */
    int nq, nF, nsplit, nci;
    double *node[3];
    double *S[3];                    /* face vectors [dir][face*3] */
    double *fc[3];                   /* face centroids */
    double *V, *xc;                  /* volumes, centroids [cell*3] */
    double *Q, *R, *dQs, *dQ, *dQci_s, *dQci;
    prim_t *w;
    prim_t fs;                       /* freestream primitive */
    double fsQ[NQMAX], Tw;
    double *grad;                    /* [cell][NGMAX][3] */
    double *Fface[3];                /* [dir][face][nq] */
    double *lamF, *lamC, *lamCI;     /* hat-lambda per cell and direction [cell*3] */
    double *lamCIv;                  /* 2 lambda_vis of the coupled operator [cell*3] */
    int ci_split;                    /* coupled operator: 0 spectral splitting, 1 eigenvalue */
    int dtau_src;                    /* 1: lambda_S in the local time step (Sec. 2.2 Delta tau) */
    double *DF, *DFev, *Ds;          /* diagonals */
    double *DLU; int *piv;           /* CI diagonal blocks, LU factors */
    double norms[2], qstag;
    int stag_cell, have_R, iter;
    int status_cell, nclip;
    int react;                       /* 0: sources off (non-reactive runs) */
    /* dual time stepping (Sec. 2.3, Eq. dualimplicit): physical step dt (0: steady), theta,
     * stored physical levels Q^n, Q^{n-1} and how many of them exist (0, 1, 2) */
    double dual_dt, dual_theta;
    double *Qn, *Qnm1;
    int dual_levels;
    char err[256];
} orc_grid;

/* Physical-time coefficients of the dual time-stepping residual (Sec. 2.3): the unsteady term
 * V [(1+theta)(Q^m - Q^n) - theta (Q^n - Q^{n-1})] / dt is added to R, and (1+theta) V / dt to
 * every diagonal.  Reading: theta multiplies a level difference that exists only from the
 * second physical step on, so the first step after the start takes theta = 0 (implicit
 * Euler).  Returns 0 when dual time stepping is off or no physical step has begun. */
static int dual_coeffs(const orc_grid *G, double *a, double *b)
{
    *a = *b = 0.0;
    if (!(G->dual_dt > 0.0) || G->dual_levels < 1) return 0;
    double th = G->dual_levels >= 2 ? G->dual_theta : 0.0;
    *a = (1.0 + th) / G->dual_dt;
    *b = th / G->dual_dt;
    return 1;
}

static int fidx(const orc_grid *G, int d, int i, int j, int k)
{
    int fi = G->n[0] + (d == 0), fj = G->n[1] + (d == 1);
    return i + fi * (j + fj * k);
}
static int cidx(const orc_grid *G, int i, int j, int k) { return i + G->n[0] * (j + G->n[1] * k); }
static int nidx(const orc_grid *G, int i, int j, int k)
{
    return i + (G->n[0] + 1) * (j + (G->n[1] + 1) * k);
}
static void node_xyz(const orc_grid *G, int i, int j, int k, double *x)
{
    int n = nidx(G, i, j, k);
    for (int d = 0; d < 3; d++) x[d] = (d < G->nd) ? G->node[d][n] : 0.0;
}
static void cross(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static void compute_geometry(orc_grid *G)
{
    int nd = G->nd, ni = G->n[0], nj = G->n[1], nk = G->n[2];
    for (int d = 0; d < nd; d++) {
        int li = ni + (d == 0), lj = nj + (d == 1), lk = (nd == 3) ? nk + (d == 2) : 1;
        for (int k = 0; k < lk; k++)
            for (int j = 0; j < lj; j++)
                for (int i = 0; i < li; i++) {
                    int f = fidx(G, d, i, j, k);
                    double *S = &G->S[d][3 * f], *c = &G->fc[d][3 * f];
                    if (nd == 2) {
                        double a[3], b[3];
                        node_xyz(G, i, j, 0, a);
                        if (d == 0) node_xyz(G, i, j + 1, 0, b);
                        else node_xyz(G, i + 1, j, 0, b);
                        double ex = b[0] - a[0], ey = b[1] - a[1];
                        if (d == 0) { S[0] = ey; S[1] = -ex; }
                        else { S[0] = -ey; S[1] = ex; }
                        S[2] = 0.0;
                        for (int q = 0; q < 3; q++) c[q] = 0.5 * (a[q] + b[q]);
                    } else {
                        /* quad face spanned by the two other (cyclic) axes a, b:
                         * S = 1/2 (P_ab - P_00) x (P_b - P_a) */
                        int ea = (d + 1) % 3, eb = (d + 2) % 3;
                        int o[3] = {i, j, k}, pa[3], pb[3], pab[3];
                        for (int q = 0; q < 3; q++) { pa[q] = o[q]; pb[q] = o[q]; pab[q] = o[q]; }
                        pa[ea]++; pb[eb]++; pab[ea]++; pab[eb]++;
                        double x0[3], xa[3], xb[3], xab[3], d1[3], d2[3];
                        node_xyz(G, o[0], o[1], o[2], x0);
                        node_xyz(G, pa[0], pa[1], pa[2], xa);
                        node_xyz(G, pb[0], pb[1], pb[2], xb);
                        node_xyz(G, pab[0], pab[1], pab[2], xab);
                        for (int q = 0; q < 3; q++) { d1[q] = xab[q] - x0[q]; d2[q] = xb[q] - xa[q]; }
                        cross(d1, d2, S);
                        for (int q = 0; q < 3; q++) {
                            S[q] *= 0.5;
                            c[q] = 0.25 * (x0[q] + xa[q] + xb[q] + xab[q]);
                        }
                    }
                }
    }
    int lk = (nd == 3) ? nk : 1;
    for (int k = 0; k < lk; k++)
        for (int j = 0; j < nj; j++)
            for (int i = 0; i < ni; i++) {
                int c = cidx(G, i, j, k);
                double *xc = &G->xc[3 * c];
                if (nd == 2) {
                    /* quad split into triangles (0,1,2), (0,2,3) */
                    double p0[3], p1[3], p2[3], p3[3];
                    node_xyz(G, i, j, 0, p0); node_xyz(G, i + 1, j, 0, p1);
                    node_xyz(G, i + 1, j + 1, 0, p2); node_xyz(G, i, j + 1, 0, p3);
                    double a1 = 0.5 * ((p1[0] - p0[0]) * (p2[1] - p0[1]) - (p2[0] - p0[0]) * (p1[1] - p0[1]));
                    double a2 = 0.5 * ((p2[0] - p0[0]) * (p3[1] - p0[1]) - (p3[0] - p0[0]) * (p2[1] - p0[1]));
                    G->V[c] = a1 + a2;
                    for (int q = 0; q < 2; q++)
                        xc[q] = (a1 * (p0[q] + p1[q] + p2[q]) + a2 * (p0[q] + p2[q] + p3[q])) / (3.0 * (a1 + a2));
                    xc[2] = 0.0;
                } else {
                    /* divergence theorem: V = 1/3 sum_f x_f . S_f,out */
                    double v = 0.0;
                    int o[3] = {i, j, k};
                    for (int d = 0; d < 3; d++) {
                        int lo[3] = {o[0], o[1], o[2]}, hi[3] = {o[0], o[1], o[2]};
                        hi[d]++;
                        int fl = fidx(G, d, lo[0], lo[1], lo[2]), fh = fidx(G, d, hi[0], hi[1], hi[2]);
                        for (int q = 0; q < 3; q++)
                            v += G->fc[d][3 * fh + q] * G->S[d][3 * fh + q]
                               - G->fc[d][3 * fl + q] * G->S[d][3 * fl + q];
                    }
                    G->V[c] = v / 3.0;
                    for (int q = 0; q < 3; q++) xc[q] = 0.0;
                    for (int a = 0; a < 2; a++)
                        for (int b = 0; b < 2; b++)
                            for (int e = 0; e < 2; e++) {
                                double x[3];
                                node_xyz(G, i + e, j + b, k + a, x);
                                for (int q = 0; q < 3; q++) xc[q] += 0.125 * x[q];
                            }
                }
            }
}

/* neighbour of cell (o) across side s (-1/+1) of direction d: returns cell index, or -1 for a
 * boundary.  *hlower = 1 if the neighbour precedes the cell in the sweep order h = i+j+k. */
static int neighbour(const orc_grid *G, const int *o, int d, int s, int *hlower)
{
    int p[3] = {o[0], o[1], o[2]};
    p[d] += s;
    int n = G->n[d];
    if (p[d] < 0 || p[d] >= n) {
        int b = G->bc[2 * d + (s > 0)];
        if (b != BC_PERIODIC) return -1;
        p[d] = (p[d] + n) % n;
    }
    if (hlower) *hlower = (p[d] - o[d]) < 0;
    return cidx(G, p[0], p[1], G->nd == 3 ? p[2] : 0);
}

/* face between cell o and its neighbour on side s of direction d (face index along d) */
static int face_of(const orc_grid *G, const int *o, int d, int s)
{
    int p[3] = {o[0], o[1], o[2]};
    if (s > 0) p[d]++;
    return fidx(G, d, p[0], p[1], G->nd == 3 ? p[2] : 0);
}

static void cell_coords(const orc_grid *G, int c, int *o)
{
    o[0] = c % G->n[0];
    o[1] = (c / G->n[0]) % G->n[1];
    o[2] = c / (G->n[0] * G->n[1]);
}

/* ---------------------------------------------------------------------------------------
 * Inviscid flux (Sec. 3.2: MUSCL reconstruction with the minmod limiter + Roe's scheme).
 * Reading: reconstructed variables per cell are w = (rho_s, u, p, Gam = rho*e/p, beta,
 * [e_v]); the face state needs no temperature solve.  Roe average with sqrt(rho) weights;
 * Harten's entropy fix on all three wave speeds, with the width
 *   delta = max(eps (|u_n| + c), 2 eta_H),
 * so that a wave speed of zero is raised to eta_H, where eta_H is the multidimensional H-correction of Sanders, Morano and Druguet (J. Comput.
 * Phys. 145, 1998): the largest eta over this face and the faces of the other directions that
 * bound its two cells, eta = (|jump of u.n| + |jump of c|) / 2 between the two cell-centre
 * states of a face (the largest jump of u_n - c, u_n, u_n + c).  Faces on a non-periodic
 * boundary have eta = 0.  The paper does not state its entropy fix; without the H term Roe's
 * scheme develops the carbuncle instability on the stagnation line of a blunt body.
 * ------------------------------------------------------------------------------------- */
typedef struct { double rhos[NSMAX], u[3], p, Gam, beta, ev; } recon_t;

static int nrecon(const orc_grid *G) { return G->gas.ns + G->nd + 3 + (G->gas.ntemp == 2); }

static void recon_pack(const orc_grid *G, const prim_t *w, double *v)
{
    int ns = G->gas.ns, nd = G->nd, k = 0;
    for (int s = 0; s < ns; s++) v[k++] = w->rhos[s];
    for (int d = 0; d < nd; d++) v[k++] = w->u[d];
    v[k++] = w->p;
    v[k++] = w->Gam;
    v[k++] = w->beta;
    if (G->gas.ntemp == 2) v[k++] = w->ev;
}
static void recon_unpack(const orc_grid *G, const double *v, recon_t *r)
{
    int ns = G->gas.ns, nd = G->nd, k = 0;
    memset(r, 0, sizeof(*r));
    for (int s = 0; s < ns; s++) r->rhos[s] = v[k++];
    for (int d = 0; d < nd; d++) r->u[d] = v[k++];
    r->p = v[k++];
    r->Gam = v[k++];
    r->beta = v[k++];
    if (G->gas.ntemp == 2) r->ev = v[k++];
}

static double limiter(int type, double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    if (type == 1) return (fabs(a) < fabs(b)) ? a : b;            /* minmod */
    return (a * b * (a + b)) / (a * a + b * b);                    /* van Albada (eps = 0) */
}

/* physical flux F(w).S and conserved vector of a face state */
static void state_flux(const orc_grid *G, const recon_t *r, const double *S, double *Q, double *F)
{
    int ns = G->gas.ns, nd = G->nd;
    double rho = 0.0, ke = 0.0, U = 0.0;
    for (int s = 0; s < ns; s++) rho += r->rhos[s];
    for (int d = 0; d < nd; d++) { ke += 0.5 * r->u[d] * r->u[d]; U += r->u[d] * S[d]; }
    double rhoE = r->Gam * r->p + rho * ke;
    for (int s = 0; s < ns; s++) { Q[s] = r->rhos[s]; F[s] = r->rhos[s] * U; }
    for (int d = 0; d < nd; d++) { Q[ns + d] = rho * r->u[d]; F[ns + d] = rho * r->u[d] * U + r->p * S[d]; }
    Q[ns + nd] = rhoE;
    F[ns + nd] = (rhoE + r->p) * U;
    if (G->gas.ntemp == 2) { Q[ns + nd + 1] = rho * r->ev; F[ns + nd + 1] = rho * r->ev * U; }
}

static double harten(double lam, double delta)
{
    double a = fabs(lam);
    return (a < delta) ? (lam * lam + delta * delta) / (2.0 * delta) : a;
}

/* Roe numerical flux through face vector S (oriented from L to R), F = flux * |S|; etaH is the
 * face's H-correction width (0 for none) */
static void roe_flux(const orc_grid *G, const recon_t *L, const recon_t *R, const double *S,
                     double etaH, double *F)
{
    int ns = G->gas.ns, nd = G->nd, nq = G->nq;
    double QL[NQMAX], QR[NQMAX], FL[NQMAX], FR[NQMAX];
    state_flux(G, L, S, QL, FL);
    state_flux(G, R, S, QR, FR);
    double rhoL = 0.0, rhoR = 0.0;
    for (int s = 0; s < ns; s++) { rhoL += L->rhos[s]; rhoR += R->rhos[s]; }
    double area = 0.0;
    for (int d = 0; d < nd; d++) area += S[d] * S[d];
    area = sqrt(area);
    double nh[3] = {0, 0, 0};
    for (int d = 0; d < nd; d++) nh[d] = S[d] / area;
    double sl = sqrt(rhoL), sr = sqrt(rhoR), wl = sl / (sl + sr), wr = 1.0 - wl;
    double rt = sl * sr;
    double ut[3] = {0, 0, 0}, un = 0.0, du2 = 0.0, dun = 0.0;
    for (int d = 0; d < nd; d++) {
        ut[d] = wl * L->u[d] + wr * R->u[d];
        un += ut[d] * nh[d];
        du2 += (R->u[d] - L->u[d]) * (R->u[d] - L->u[d]);
        dun += (R->u[d] - L->u[d]) * nh[d];
    }
    double HL = (QL[ns + nd] + L->p) / rhoL, HR = (QR[ns + nd] + R->p) / rhoR;
    double Ht = wl * HL + wr * HR;
    double bt = wl * L->beta + wr * R->beta;
    double prt = wl * L->p / rhoL + wr * R->p / rhoR;
    double evt = wl * L->ev + wr * R->ev;
    double Yt[NSMAX];
    for (int s = 0; s < ns; s++) Yt[s] = wl * L->rhos[s] / rhoL + wr * R->rhos[s] / rhoR;
    double c2 = (1.0 + bt) * prt + 0.5 * bt * wl * wr * du2;
    double ct = sqrt(c2);
    double delta = G->efix * (fabs(un) + ct);
    if (2.0 * etaH > delta) delta = 2.0 * etaH;
    double l1 = harten(un - ct, delta), l2 = harten(un, delta), l3 = harten(un + ct, delta);
    double dp = R->p - L->p;
    double ap = (dp + rt * ct * dun) / (2.0 * c2), am = (dp - rt * ct * dun) / (2.0 * c2);
    double rp[NQMAX], rm[NQMAX];
    for (int s = 0; s < ns; s++) { rp[s] = Yt[s]; rm[s] = Yt[s]; }
    for (int d = 0; d < nd; d++) { rp[ns + d] = ut[d] + ct * nh[d]; rm[ns + d] = ut[d] - ct * nh[d]; }
    rp[ns + nd] = Ht + un * ct;
    rm[ns + nd] = Ht - un * ct;
    if (G->gas.ntemp == 2) { rp[ns + nd + 1] = evt; rm[ns + nd + 1] = evt; }
    for (int v = 0; v < nq; v++) {
        double D = l2 * (QR[v] - QL[v]) + (l3 - l2) * ap * rp[v] + (l1 - l2) * am * rm[v];
        F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * area * D;
    }
}

/* ---------------------------------------------------------------------------------------
 * Boundary ghost states (Sec. 3.2 boundary conditions; reading for the treatment).
 * ------------------------------------------------------------------------------------- */

/* ghost primitive beyond boundary side (d, s) next to interior cell c; returns the bc code.
 * FARFIELD: freestream if the freestream enters through the face, else the interior state.
 * WALL: no-slip mirror (only used for the limiter's slope at the first interior face). */
static int ghost_prim(const orc_grid *G, int c, int d, int s, prim_t *gw)
{
    int o[3];
    cell_coords(G, c, o);
    int b = G->bc[2 * d + (s > 0)];
    *gw = G->w[c];
    if (b == BC_FARFIELD) {
        const double *Sf = &G->S[d][3 * face_of(G, o, d, s)];
        double un = 0.0;
        for (int q = 0; q < G->nd; q++) un += G->fs.u[q] * Sf[q] * (double)s;
        if (un < 0.0) *gw = G->fs;
    } else if (b == BC_WALL) {
        for (int q = 0; q < G->nd; q++) gw->u[q] = -G->w[c].u[q];
    }
    return b;
}

/* reconstructed variables of the cell across from cell c on side s of d (interior or ghost) */
static void recon_neighbour(const orc_grid *G, int c, int d, int s, double *v)
{
    int o[3], hl;
    cell_coords(G, c, o);
    int nb = neighbour(G, o, d, s, &hl);
    if (nb >= 0) { recon_pack(G, &G->w[nb], v); return; }
    prim_t gw;
    ghost_prim(G, c, d, s, &gw);
    recon_pack(G, &gw, v);
}

static int recon_ok(const orc_grid *G, const recon_t *r)
{
    for (int s = 0; s < G->gas.ns; s++) if (r->rhos[s] < 0.0) return 0;
    if (!(r->p > 0.0) || !(r->Gam > 0.0) || !(r->beta > 0.0)) return 0;
    if (G->gas.ntemp == 2 && r->ev < 0.0) return 0;
    double rho = 0.0;
    for (int s = 0; s < G->gas.ns; s++) rho += r->rhos[s];
    return rho > 0.0;
}

/* eta of the face with vector S between cells a and b: half the largest jump of the three
 * wave speeds u.n - c, u.n, u.n + c, which is (|jump of u.n| + |jump of c|) / 2 */
static double eta_cells(const orc_grid *G, int a, int b, const double *S)
{
    double area = 0.0, dun = 0.0;
    for (int d = 0; d < G->nd; d++) area += S[d] * S[d];
    area = sqrt(area);
    for (int d = 0; d < G->nd; d++) dun += (G->w[b].u[d] - G->w[a].u[d]) * (S[d] / area);
    return 0.5 * (fabs(dun) + fabs(G->w[b].c - G->w[a].c));
}

/* H-correction width of the direction-d face with face coordinates o (o[d] = 0..n[d]) */
static double eta_h(const orc_grid *G, int d, const int *o)
{
    int cells[2], nc = 0, n = G->n[d];
    int oa[3] = {o[0], o[1], o[2]}, ob[3] = {o[0], o[1], o[2]};
    if (o[d] > 0 && o[d] < n) {
        oa[d] = o[d] - 1;
    } else if (G->bc[2 * d] == BC_PERIODIC) {
        oa[d] = n - 1;
        ob[d] = 0;
    } else {
        oa[d] = (o[d] == 0) ? -1 : n - 1;
        ob[d] = (o[d] == 0) ? 0 : -1;
    }
    if (oa[d] >= 0) cells[nc++] = cidx(G, oa[0], oa[1], G->nd == 3 ? oa[2] : 0);
    if (ob[d] >= 0) cells[nc++] = cidx(G, ob[0], ob[1], G->nd == 3 ? ob[2] : 0);
    double eta = 0.0;
    if (nc == 2) eta = eta_cells(G, cells[0], cells[1], &G->S[d][3 * fidx(G, d, o[0], o[1], G->nd == 3 ? o[2] : 0)]);
    for (int m = 0; m < nc; m++) {
        int oc[3];
        cell_coords(G, cells[m], oc);
        for (int e = 0; e < G->nd; e++) {
            if (e == d) continue;
            for (int s = -1; s <= 1; s += 2) {
                int nb = neighbour(G, oc, e, s, NULL);
                if (nb < 0) continue;
                double x = eta_cells(G, cells[m], nb, &G->S[e][3 * face_of(G, oc, e, s)]);
                if (x > eta) eta = x;
            }
        }
    }
    return eta;
}

/* inviscid flux at the interior face between cells a (minus side) and b (plus side) */
static void inviscid_interior(const orc_grid *G, int a, int b, int d, const double *S,
                              double etaH, double *F)
{
    int nr = nrecon(G);
    double wa[NQMAX + 4], wb[NQMAX + 4], wam[NQMAX + 4], wbp[NQMAX + 4], vl[NQMAX + 4], vr[NQMAX + 4];
    recon_pack(G, &G->w[a], wa);
    recon_pack(G, &G->w[b], wb);
    recon_neighbour(G, a, d, -1, wam);
    recon_neighbour(G, b, d, +1, wbp);
    for (int k = 0; k < nr; k++) {
        double dm = wa[k] - wam[k], dc = wb[k] - wa[k], dp = wbp[k] - wb[k];
        vl[k] = wa[k];
        vr[k] = wb[k];
        if (G->limiter) {
            vl[k] += 0.5 * limiter(G->limiter, dm, dc);
            vr[k] -= 0.5 * limiter(G->limiter, dc, dp);
        }
    }
    recon_t L, R;
    recon_unpack(G, vl, &L);
    recon_unpack(G, vr, &R);
    if (!recon_ok(G, &L) || !recon_ok(G, &R)) {
        recon_unpack(G, wa, &L);
        recon_unpack(G, wb, &R);
    }
    roe_flux(G, &L, &R, S, etaH, F);
}

/* inviscid flux at a boundary face of cell c (side s of d) */
static void inviscid_boundary(const orc_grid *G, int c, int d, int s, const double *S,
                              double etaH, double *F)
{
    int nq = G->nq, ns = G->gas.ns, nd = G->nd;
    prim_t gw;
    int b = ghost_prim(G, c, d, s, &gw);
    for (int v = 0; v < nq; v++) F[v] = 0.0;
    if (b == BC_AXIS) return;
    if (b == BC_WALL) {
        for (int q = 0; q < nd; q++) F[ns + q] = G->w[c].p * S[q];
        return;
    }
    double vi[NQMAX + 4], vg[NQMAX + 4];
    recon_pack(G, &G->w[c], vi);
    recon_pack(G, &gw, vg);
    recon_t I, Gh;
    recon_unpack(G, vi, &I);
    recon_unpack(G, vg, &Gh);
    if (s > 0) roe_flux(G, &I, &Gh, S, etaH, F);
    else roe_flux(G, &Gh, &I, S, etaH, F);
}

/* ---------------------------------------------------------------------------------------
 * Viscous and diffusive flux (Sec. 2.1: tau, q, q_v, Fick diffusion; Sec. 3.2: second-order
 * central).  Reading: Green-Gauss cell gradients; face gradient = mean of the two cell
 * gradients with its component along the centroid line replaced by the difference quotient.
 * ------------------------------------------------------------------------------------- */
static int ngrad(const orc_grid *G) { return G->nd + 1 + (G->gas.ntemp == 2) + G->gas.ns; }

static void grad_pack(const orc_grid *G, const prim_t *w, double *v)
{
    int k = 0;
    for (int d = 0; d < G->nd; d++) v[k++] = w->u[d];
    v[k++] = w->T;
    if (G->gas.ntemp == 2) v[k++] = w->Tv;
    for (int s = 0; s < G->gas.ns; s++) v[k++] = w->Y[s];
}

/* face value of the gradient variables on boundary side (d, s) of cell c */
static void grad_boundary_value(const orc_grid *G, int c, int d, int s, double *v)
{
    int ng = ngrad(G);
    double vc[NGMAX];
    grad_pack(G, &G->w[c], vc);
    prim_t gw;
    int b = ghost_prim(G, c, d, s, &gw);
    if (b == BC_WALL) {
        int k = 0;
        for (int q = 0; q < G->nd; q++) v[k++] = 0.0;
        v[k++] = G->Tw;
        if (G->gas.ntemp == 2) v[k++] = G->Tw;
        for (int q = 0; q < G->gas.ns; q++) { v[k] = vc[k]; k++; }
    } else if (b == BC_FARFIELD) {
        double vg[NGMAX];
        grad_pack(G, &gw, vg);
        for (int k = 0; k < ng; k++) v[k] = 0.5 * (vc[k] + vg[k]);
    } else {
        for (int k = 0; k < ng; k++) v[k] = vc[k];
    }
}

static void compute_gradients(orc_grid *G)
{
    int ng = ngrad(G), nd = G->nd;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < G->ncell; c++) {
        int o[3];
        cell_coords(G, c, o);
        double *gr = &G->grad[(size_t)c * NGMAX * 3];
        for (int k = 0; k < NGMAX * 3; k++) gr[k] = 0.0;
        double vc[NGMAX];
        grad_pack(G, &G->w[c], vc);
        for (int d = 0; d < nd; d++)
            for (int s = -1; s <= 1; s += 2) {
                const double *Sf = &G->S[d][3 * face_of(G, o, d, s)];
                double vf[NGMAX];
                int hl, nb = neighbour(G, o, d, s, &hl);
                if (nb >= 0) {
                    double vn[NGMAX];
                    grad_pack(G, &G->w[nb], vn);
                    for (int k = 0; k < ng; k++) vf[k] = 0.5 * (vc[k] + vn[k]);
                } else {
                    grad_boundary_value(G, c, d, s, vf);
                }
                for (int k = 0; k < ng; k++)
                    for (int q = 0; q < nd; q++) gr[3 * k + q] += (double)s * vf[k] * Sf[q];
            }
        for (int k = 0; k < ng * 3; k++) gr[k] /= G->V[c];
    }
}

/* viscous flux through S given face gradients g[k][q], face velocity uf, transport
 * coefficients and face species enthalpies; wall = 1 suppresses species diffusion */
/* Diffusive mass fluxes through S (Sec. 2.1 Fick's law with an effective coefficient per
 * species): J_s = -rho D_s grad(Y_s).S.  With the species transport model the electrons' flux
 * follows from no net charge flux, J_e = M_e sum_ions J_i / M_i, and a correction velocity makes
 * the fluxes sum to zero, J_s -= Y_s sum_r J_r (Yf: face mass fractions; the mixture being
 * neutral, the correction keeps the charge flux zero).  With the single-coefficient model the
 * fluxes sum to zero by themselves. */
static void diffusive_fluxes(const orc_grid *G, const double *g, const double *rhoDs,
                             const double *Yf, const double *S, double *J)
{
    int ns = G->gas.ns, nd = G->nd, two = (G->gas.ntemp == 2);
    int iY = nd + 1 + two;
    for (int s = 0; s < ns; s++) {
        J[s] = 0.0;
        for (int q = 0; q < nd; q++) J[s] -= rhoDs[s] * g[3 * (iY + s) + q] * S[q];
    }
    if (G->gas.transport != 1) return;
    double sum = 0.0, je = 0.0;
    int e = -1;
    for (int s = 0; s < ns; s++) {
        if (!is_heavy(&G->gas, s)) { e = s; continue; }
        if (G->gas.sp[s].charge != 0) je += J[s] / G->gas.M[s];
    }
    if (e >= 0) J[e] = je * G->gas.M[e];
    for (int s = 0; s < ns; s++) sum += J[s];
    for (int s = 0; s < ns; s++) J[s] -= Yf[s] * sum;
}

static void viscous_flux(const orc_grid *G, const double *g, const double *uf, double mu,
                         double kt, double kv, const double *rhoDs, const double *Yf,
                         const double *hs, const double *eve, const double *S, int wall,
                         double *F)
{
    int ns = G->gas.ns, nd = G->nd, two = (G->gas.ntemp == 2);
    int iT = nd, iTv = nd + 1;
    double tau[3][3], div = 0.0;
    for (int i = 0; i < nd; i++) div += g[3 * i + i];
    for (int i = 0; i < nd; i++)
        for (int l = 0; l < nd; l++)
            tau[i][l] = mu * (g[3 * i + l] + g[3 * l + i]) - (i == l ? 2.0 / 3.0 * mu * div : 0.0);
    for (int v = 0; v < G->nq; v++) F[v] = 0.0;
    double qdiff = 0.0, qvdiff = 0.0, Js[NSMAX];
    if (wall) for (int s = 0; s < ns; s++) Js[s] = 0.0;
    else diffusive_fluxes(G, g, rhoDs, Yf, S, Js);
    for (int s = 0; s < ns; s++) {
        double J = Js[s];
        F[s] = J;
        qdiff += J * hs[s];
        if (two) qvdiff += J * eve[s];
    }
    double work = 0.0;
    for (int i = 0; i < nd; i++) {
        double ts = 0.0;
        for (int l = 0; l < nd; l++) ts += tau[i][l] * S[l];
        F[ns + i] = -ts;
        work += uf[i] * ts;
    }
    double gT = 0.0, gTv = 0.0;
    for (int q = 0; q < nd; q++) {
        gT += g[3 * iT + q] * S[q];
        if (two) gTv += g[3 * iTv + q] * S[q];
    }
    F[ns + nd] = -work - kt * gT - kv * gTv + qdiff;
    if (two) F[ns + nd + 1] = -kv * gTv + qvdiff;
}

static void viscous_interior(const orc_grid *G, int a, int b, const double *S, double *F)
{
    int ng = ngrad(G), nd = G->nd, ns = G->gas.ns;
    const double *ga = &G->grad[(size_t)a * NGMAX * 3], *gb = &G->grad[(size_t)b * NGMAX * 3];
    double t[3], tl = 0.0;
    for (int q = 0; q < 3; q++) { t[q] = G->xc[3 * b + q] - G->xc[3 * a + q]; tl += t[q] * t[q]; }
    tl = sqrt(tl);
    for (int q = 0; q < 3; q++) t[q] /= tl;
    double va[NGMAX], vb[NGMAX], g[NGMAX * 3];
    grad_pack(G, &G->w[a], va);
    grad_pack(G, &G->w[b], vb);
    for (int k = 0; k < ng; k++) {
        double gt = 0.0;
        for (int q = 0; q < nd; q++) {
            g[3 * k + q] = 0.5 * (ga[3 * k + q] + gb[3 * k + q]);
            gt += g[3 * k + q] * t[q];
        }
        double corr = (vb[k] - va[k]) / tl - gt;
        for (int q = 0; q < nd; q++) g[3 * k + q] += corr * t[q];
    }
    const prim_t *A = &G->w[a], *B = &G->w[b];
    double uf[3] = {0, 0, 0}, hs[NSMAX], eve[NSMAX], rD[NSMAX], Yf[NSMAX];
    for (int q = 0; q < nd; q++) uf[q] = 0.5 * (A->u[q] + B->u[q]);
    for (int s = 0; s < ns; s++) {
        hs[s] = 0.5 * (A->hs[s] + B->hs[s]);
        eve[s] = 0.5 * (A->eve[s] + B->eve[s]);
        rD[s] = 0.5 * (A->rhoDs[s] + B->rhoDs[s]);
        Yf[s] = 0.5 * (A->Y[s] + B->Y[s]);
    }
    viscous_flux(G, g, uf, 0.5 * (A->mu + B->mu), 0.5 * (A->kt + B->kt), 0.5 * (A->kv + B->kv),
                 rD, Yf, hs, eve, S, 0, F);
}

/* viscous flux at a wall face of cell c (isothermal, no-slip, non-catalytic); other boundary
 * kinds carry no viscous flux */
static void viscous_boundary(const orc_grid *G, int c, int d, int s, int f, const double *S, double *F)
{
    int ng = ngrad(G), nd = G->nd;
    for (int v = 0; v < G->nq; v++) F[v] = 0.0;
    if (G->bc[2 * d + (s > 0)] != BC_WALL) return;
    const double *gc = &G->grad[(size_t)c * NGMAX * 3];
    const double *xf = &G->fc[d][3 * f];
    double t[3], tl = 0.0;     /* from the face (minus side) towards the cell, along +d */
    for (int q = 0; q < 3; q++) {
        t[q] = (s < 0) ? G->xc[3 * c + q] - xf[q] : xf[q] - G->xc[3 * c + q];
        tl += t[q] * t[q];
    }
    tl = sqrt(tl);
    for (int q = 0; q < 3; q++) t[q] /= tl;
    double vc[NGMAX], vw[NGMAX], g[NGMAX * 3];
    grad_pack(G, &G->w[c], vc);
    grad_boundary_value(G, c, d, s, vw);
    for (int k = 0; k < ng; k++) {
        double gt = 0.0;
        for (int q = 0; q < nd; q++) { g[3 * k + q] = gc[3 * k + q]; gt += g[3 * k + q] * t[q]; }
        double corr = ((s < 0) ? (vc[k] - vw[k]) : (vw[k] - vc[k])) / tl - gt;
        for (int q = 0; q < nd; q++) g[3 * k + q] += corr * t[q];
    }
    const prim_t *w = &G->w[c];
    double uf[3] = {0, 0, 0};
    viscous_flux(G, g, uf, w->mu, w->kt, w->kv, w->rhoDs, w->Y, w->hs, w->eve, S, 1, F);
}

/* ---------------------------------------------------------------------------------------
 * Residual R(Q) (Sec. 2.2, Eq. (iterate)): R = sum over faces of (F_inv + F_vis).S_out
 * minus V * S.  dQ/dt V = -R.
 * ------------------------------------------------------------------------------------- */
/* Every cell is independent; the first failing cell (lowest index) is reported.  (The
 * OpenMP build of the oracle, used only to time it on all host cores, runs this loop, the
 * gradients, the face fluxes and the spectral radii in parallel; results do not change.) */
static int compute_primitives(orc_grid *G)
{
    int nst = G->nq, N = G->ncell, bad = N, badst = 0;
#pragma omp parallel for schedule(static) reduction(min : bad)
    for (int c = 0; c < N; c++) {
        double q[NQMAX];
        for (int v = 0; v < nst; v++) q[v] = G->Q[(size_t)v * N + c];
        double Tg = G->w[c].T, Tvg = G->w[c].Tv;
        int st = prim_from_cons(&G->gas, G->nd, q, Tg, Tvg, &G->w[c]);
        if (st) {
            if (c < bad) bad = c;
            continue;
        }
        if (G->react) cell_sources(&G->gas, G->nd, &G->w[c]);
    }
    if (bad < N) {
        double q[NQMAX];
        prim_t w;
        for (int v = 0; v < nst; v++) q[v] = G->Q[(size_t)v * N + bad];
        badst = prim_from_cons(&G->gas, G->nd, q, G->w[bad].T, G->w[bad].Tv, &w);
        G->status_cell = bad;
        snprintf(G->err, sizeof(G->err), "primitive recovery failed (code %d) at cell %d", badst, bad);
        return badst == 3 ? 5 : 4;
    }
    return 0;
}

static void stagnation_heat_flux(orc_grid *G)
{
    /* Monitor (Sec. 3.2): heat flux at the wall cell whose outward body normal is most nearly
     * opposite the freestream.  q_w = k (T_1 - T_w)/d_1 [+ k_v (Tv_1 - T_w)/d_1]. */
    G->qstag = 0.0;
    if (G->stag_cell < 0) return;
    int c = G->stag_cell, o[3];
    cell_coords(G, c, o);
    int d = 1, s = -1;                        /* wall on the j-min side */
    if (G->bc[2] != BC_WALL) return;
    int f = face_of(G, o, d, s);
    const double *Sf = &G->S[d][3 * f], *xf = &G->fc[d][3 * f];
    double area = 0.0, dist = 0.0;
    for (int q = 0; q < 3; q++) area += Sf[q] * Sf[q];
    area = sqrt(area);
    for (int q = 0; q < 3; q++) dist += (G->xc[3 * c + q] - xf[q]) * Sf[q] / area;
    dist = fabs(dist);
    const prim_t *w = &G->w[c];
    G->qstag = w->kt * (w->T - G->Tw) / dist;
    if (G->gas.ntemp == 2) G->qstag += w->kv * (w->Tv - G->Tw) / dist;
}

static int residual(orc_grid *G)
{
    int nq = G->nq, nd = G->nd, ns = G->gas.ns;
    int st = compute_primitives(G);
    if (st) return st;
    compute_gradients(G);
    /* face fluxes, each face once */
    for (int d = 0; d < nd; d++) {
        int li = G->n[0] + (d == 0), lj = G->n[1] + (d == 1), lk = (nd == 3) ? G->n[2] + (d == 2) : 1;
#pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < lk; k++)
            for (int j = 0; j < lj; j++)
                for (int i = 0; i < li; i++) {
                    int f = fidx(G, d, i, j, k);
                    const double *S = &G->S[d][3 * f];
                    double *F = &G->Fface[d][(size_t)f * nq];
                    int o[3] = {i, j, k}, lo = o[d] - 1, hi = o[d], n = G->n[d];
                    int per = (G->bc[2 * d] == BC_PERIODIC);
                    double Fi[NQMAX], Fv[NQMAX];
                    double etaH = G->hcorr ? eta_h(G, d, o) : 0.0;
                    if (lo >= 0 && hi < n) {
                        int oa[3] = {o[0], o[1], o[2]};
                        oa[d] = lo;
                        int a = cidx(G, oa[0], oa[1], nd == 3 ? oa[2] : 0);
                        int b = cidx(G, o[0], o[1], nd == 3 ? o[2] : 0);
                        inviscid_interior(G, a, b, d, S, etaH, Fi);
                        if (G->viscous) viscous_interior(G, a, b, S, Fv);
                        else for (int v = 0; v < nq; v++) Fv[v] = 0.0;
                    } else if (per) {
                        int oa[3] = {o[0], o[1], o[2]}, ob[3] = {o[0], o[1], o[2]};
                        oa[d] = n - 1;
                        ob[d] = 0;
                        int a = cidx(G, oa[0], oa[1], nd == 3 ? oa[2] : 0);
                        int b = cidx(G, ob[0], ob[1], nd == 3 ? ob[2] : 0);
                        inviscid_interior(G, a, b, d, S, etaH, Fi);
                        if (G->viscous) viscous_interior(G, a, b, S, Fv);
                        else for (int v = 0; v < nq; v++) Fv[v] = 0.0;
                    } else {
                        int oc[3] = {o[0], o[1], o[2]}, s;
                        if (lo < 0) { oc[d] = 0; s = -1; } else { oc[d] = n - 1; s = +1; }
                        int c = cidx(G, oc[0], oc[1], nd == 3 ? oc[2] : 0);
                        inviscid_boundary(G, c, d, s, S, etaH, Fi);
                        if (G->viscous) viscous_boundary(G, c, d, s, f, S, Fv);
                        else for (int v = 0; v < nq; v++) Fv[v] = 0.0;
                    }
                    for (int v = 0; v < nq; v++) F[v] = Fi[v] + Fv[v];
                }
    }
    double rs = 0.0, re = 0.0;
    for (int c = 0; c < G->ncell; c++) {
        int o[3];
        cell_coords(G, c, o);
        double r[NQMAX];
        for (int v = 0; v < nq; v++) r[v] = 0.0;
        for (int d = 0; d < nd; d++) {
            const double *Fm = &G->Fface[d][(size_t)face_of(G, o, d, -1) * nq];
            const double *Fp = &G->Fface[d][(size_t)face_of(G, o, d, +1) * nq];
            for (int v = 0; v < nq; v++) r[v] += Fp[v] - Fm[v];
        }
        const prim_t *w = &G->w[c];
        for (int s = 0; s < ns; s++) r[s] -= G->V[c] * w->omega[s];
        if (G->gas.ntemp == 2) r[ns + nd + 1] -= G->V[c] * w->omega_v;
        double da, db;
        if (dual_coeffs(G, &da, &db))
            for (int v = 0; v < nq; v++) {
                size_t x = (size_t)v * G->ncell + c;
                r[v] += G->V[c] * (da * (G->Q[x] - G->Qn[x]) - db * (G->Qn[x] - G->Qnm1[x]));
            }
        for (int v = 0; v < nq; v++) G->R[(size_t)v * G->ncell + c] = r[v];
        /* residual monitors (Sec. 3.2; reading: L2 over cells of R/V) */
        for (int s = 0; s < ns; s++) rs += (r[s] / G->V[c]) * (r[s] / G->V[c]);
        re += (r[ns + nd] / G->V[c]) * (r[ns + nd] / G->V[c]);
    }
    G->norms[0] = sqrt(rs);
    G->norms[1] = sqrt(re);
    stagnation_heat_flux(G);
    G->have_R = 1;
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * Spectral radii, local time step and diagonals (Sec. 2.2 Delta tau and Eq. (vislambda);
 * Sec. 2.3.1 flow radius; Sec. 2.3.2 component radius).  Reading (the viscous radius is
 * garbled in the paper): lambda_vis,d = nu_eff |S_d|^2 / V with
 *   flow:       nu_eff = max(4 mu/3, k/c_v[, k_v/c_v,ve]) / rho
 *   components: nu_eff = rho D / rho
 *   coupled:    nu_eff = max of all of the above.
 * S_d = mean of the two face vectors of the cell in direction d; hat-lambda = lambda_inv +
 * 2 lambda_vis; V/dtau = sum_d (lambda_inv,d + lambda_vis,d) / CFL (flow radius, both
 * schemes); by default the source's radius lambda_S enters through the diagonals only.  With
 * dtau_src the local time step is the one Sec. 2.2 prints, its denominator carrying lambda_S
 * too: V/dtau = (sum_d (lambda_inv,d + lambda_vis,d) + V lambda_S) / CFL, lambda_S read as the
 * largest magnitude on the diagonal of the source Jacobian A_S = dS/dQ (|d omega_s/d rho_s| of
 * every species and, 2T, the vibrational relaxation rate).
 * ------------------------------------------------------------------------------------- */
static void absjac_ci(const orc_grid *G, const prim_t *w, const double *S, const double *dc, double *out);

static void spectral(orc_grid *G, double cfl)
{
    int nd = G->nd, ns = G->gas.ns;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < G->ncell; c++) {
        int o[3];
        cell_coords(G, c, o);
        const prim_t *w = &G->w[c];
        double nuF, nuC = w->rhoD / w->rho, nuCI;
        if (G->gas.ntemp == 2) {
            nuF = fmax(4.0 * w->mu / 3.0, w->kt / w->cvtr);
            if (w->cvve > 0.0) nuF = fmax(nuF, w->kv / w->cvve);
        } else {
            nuF = fmax(4.0 * w->mu / 3.0, w->kt / w->cv);
        }
        nuF /= w->rho;
        if (!G->viscous) nuF = nuC = 0.0;
        nuCI = fmax(nuF, nuC);
        double sumdt = 0.0, sF = 0.0, sC = 0.0, sCI = 0.0, sCIv = 0.0;
        double Sbar[3][3] = {{0}};
        for (int d = 0; d < nd; d++) {
            const double *Sm = &G->S[d][3 * face_of(G, o, d, -1)];
            const double *Sp = &G->S[d][3 * face_of(G, o, d, +1)];
            double *Sb = Sbar[d], a2 = 0.0, U = 0.0;
            for (int q = 0; q < nd; q++) {
                Sb[q] = 0.5 * (Sm[q] + Sp[q]);
                a2 += Sb[q] * Sb[q];
                U += w->u[q] * Sb[q];
            }
            double a = sqrt(a2);
            double liF = fabs(U) + w->c * a, liC = fabs(U);
            double lvF = nuF * a2 / G->V[c], lvC = nuC * a2 / G->V[c], lvCI = nuCI * a2 / G->V[c];
            G->lamF[3 * c + d] = liF + 2.0 * lvF;
            G->lamC[3 * c + d] = liC + 2.0 * lvC;
            G->lamCI[3 * c + d] = liF + 2.0 * lvCI;
            G->lamCIv[3 * c + d] = 2.0 * lvCI;
            sCIv += 2.0 * lvCI;
            sumdt += liF + lvF;
            sF += G->lamF[3 * c + d];
            sC += G->lamC[3 * c + d];
            sCI += G->lamCI[3 * c + d];
        }
        if (G->dtau_src && G->react) {
            double lS = G->gas.ntemp == 2 ? w->relax : 0.0;
            for (int s = 0; s < ns; s++) lS = fmax(lS, fabs(w->dom[s]));
            sumdt += G->V[c] * lS;
        }
        double Vdt = sumdt / cfl;                  /* V / dtau */
        double da, db;
        if (dual_coeffs(G, &da, &db)) Vdt += da * G->V[c];   /* + (1+theta) V / dt */
        G->DF[c] = Vdt + sF;
        G->DFev[c] = Vdt + sF + G->V[c] * w->relax;
        for (int s = 0; s < ns; s++)
            G->Ds[(size_t)s * G->ncell + c] = Vdt + sC + G->V[c] * fmax(0.0, -w->dom[s]);
        /* coupled diagonal block: (V/dtau + sum lambda) I - V dS/dQ (CI variables) */
        if (G->DLU) {
            int n = G->nci, nF = G->nF;
            double *A = &G->DLU[(size_t)c * n * n];
            for (int k = 0; k < n * n; k++) A[k] = 0.0;
            if (!G->ci_split) {
                for (int k = 0; k < n; k++) A[k * n + k] = Vdt + sCI;
            } else {
                /* eigenvalue splitting: (V/dtau + sum 2 lambda_vis) I + sum_d |A_c(S_d)| */
                for (int k = 0; k < n; k++) A[k * n + k] = Vdt + sCIv;
                for (int d = 0; d < nd; d++)
                    for (int col = 0; col < n; col++) {
                        double e[NQMAX] = {0}, a[NQMAX];
                        e[col] = 1.0;
                        absjac_ci(G, w, Sbar[d], e, a);
                        for (int r = 0; r < n; r++) A[r * n + col] += a[r];
                    }
            }
            if (G->gas.ntemp == 2) A[(nF - 1) * n + (nF - 1)] += G->V[c] * w->relax;
            int nq = G->nq;
            double Jq[NSMAX * NQMAX], om[NSMAX];
            if (G->react) source_jacobian(&G->gas, nd, w, om, Jq);
            else memset(Jq, 0, sizeof Jq);
            /* rows: species s = 1..ns-1 (row nF + s - 1).  Columns in coupled variables: rho
             * (0) is d/d rho_1st, rho_r (nF + r - 1) is d/d rho_r - d/d rho_1st since the first
             * species is rho - sum_{r>0} rho_r (Sec. 2.3.3, see jvp_ci); m, rhoE, [rho e_v]
             * columns (1..nF-1) map to full columns ns.. */
            for (int s = 1; s < ns; s++) {
                const double *row = &Jq[s * nq];
                A[(nF + s - 1) * n + 0] -= G->V[c] * row[0];
                for (int k = 1; k < nF; k++) A[(nF + s - 1) * n + k] -= G->V[c] * row[ns + k - 1];
                for (int r = 1; r < ns; r++)
                    A[(nF + s - 1) * n + nF + r - 1] -= G->V[c] * (row[r] - row[0]);
            }
        }
    }
}

/* LU factorisation with partial pivoting (ties: lowest row index), in place */
static int lu_factor(double *A, int *piv, int n)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = fabs(A[k * n + k]);
        for (int i = k + 1; i < n; i++)
            if (fabs(A[i * n + k]) > best) { best = fabs(A[i * n + k]); p = i; }
        piv[k] = p;
        if (best == 0.0) return 1;
        if (p != k)
            for (int j = 0; j < n; j++) { double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t; }
        for (int i = k + 1; i < n; i++) {
            double l = A[i * n + k] / A[k * n + k];
            A[i * n + k] = l;
            for (int j = k + 1; j < n; j++) A[i * n + j] -= l * A[k * n + j];
        }
    }
    return 0;
}
static void lu_solve(const double *A, const int *piv, int n, double *b)
{
    for (int k = 0; k < n; k++)
        if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
    for (int i = 1; i < n; i++)
        for (int j = 0; j < i; j++) b[i] -= A[i * n + j] * b[j];
    for (int i = n - 1; i >= 0; i--) {
        for (int j = i + 1; j < n; j++) b[i] -= A[i * n + j] * b[j];
        b[i] /= A[i * n + i];
    }
}

/* ---------------------------------------------------------------------------------------
 * Convective flux Jacobian times a vector (Sec. 2.3, Eq. (convectiveJacobian)), evaluated at
 * a cell state w with face vector S.  Exact Jacobian of the Euler flux of the thermally
 * perfect mixture, matrix-free.  Full conserved layout: (rho_s, m, rhoE, [rho e_v]).
 * ------------------------------------------------------------------------------------- */
static void jvp_full(const orc_grid *G, const prim_t *w, const double *S, const double *dq, double *out)
{
    int ns = G->gas.ns, nd = G->nd, two = G->gas.ntemp == 2;
    double drho = 0.0, dp = 0.0, U = 0.0, Sdm = 0.0;
    for (int s = 0; s < ns; s++) { drho += dq[s]; dp += w->prs[s] * dq[s]; }
    for (int q = 0; q < nd; q++) {
        U += w->u[q] * S[q];
        Sdm += S[q] * dq[ns + q];
        dp -= w->beta * w->u[q] * dq[ns + q];
    }
    dp += w->beta * dq[ns + nd];
    if (two) dp += w->prev * dq[ns + nd + 1];
    double dU = (Sdm - U * drho) / w->rho;
    for (int s = 0; s < ns; s++) out[s] = dq[s] * U + w->rhos[s] * dU;
    for (int q = 0; q < nd; q++) out[ns + q] = dq[ns + q] * U + w->rho * w->u[q] * dU + dp * S[q];
    out[ns + nd] = (dq[ns + nd] + dp) * U + (w->rhoE + w->p) * dU;
    if (two) out[ns + nd + 1] = dq[ns + nd + 1] * U + w->rhoev * dU;
}

/* Flow block (Sec. 2.3.1): Q_F = (rho, m, rhoE, [rho e_v]) with frozen mass fractions,
 * i.e. the species increments are Y_s * d rho.  Only the flow rows are kept. */
static void jvp_flow(const orc_grid *G, const prim_t *w, const double *S, const double *dF, double *out)
{
    int ns = G->gas.ns, nF = G->nF;
    double dq[NQMAX], o[NQMAX];
    for (int s = 0; s < ns; s++) dq[s] = w->Y[s] * dF[0];
    for (int k = 1; k < nF; k++) dq[ns + k - 1] = dF[k];
    jvp_full(G, w, S, dq, o);
    double orho = 0.0;
    for (int s = 0; s < ns; s++) orho += o[s];
    out[0] = orho;
    for (int k = 1; k < nF; k++) out[k] = o[ns + k - 1];
}

/* Coupled (CI) variables (Sec. 2.3.3): (rho, m, rhoE, [rho e_v], rho_s for s = 2..ns); one
 * species density is eliminated through rho_1 = rho - sum_{s>1} rho_s.  Reading: the paper
 * eliminates its ns-th species, which in its 11-species list is the electron (about 1e-8 of
 * the density): taking it as a difference of the total and the others loses all its digits
 * and leaves the coupled blocks singular to working precision.  The eliminated species is
 * therefore the first of the list, N2, the most abundant in air. */
static void jvp_ci(const orc_grid *G, const prim_t *w, const double *S, const double *dc, double *out)
{
    int ns = G->gas.ns, nF = G->nF;
    double dq[NQMAX], o[NQMAX];
    double first = dc[0];
    for (int s = 1; s < ns; s++) { dq[s] = dc[nF + s - 1]; first -= dc[nF + s - 1]; }
    dq[0] = first;
    for (int k = 1; k < nF; k++) dq[ns + k - 1] = dc[k];
    jvp_full(G, w, S, dq, o);
    double orho = 0.0;
    for (int s = 0; s < ns; s++) orho += o[s];
    out[0] = orho;
    for (int k = 1; k < nF; k++) out[k] = o[ns + k - 1];
    for (int s = 1; s < ns; s++) out[nF + s - 1] = o[s];
}

/* |A(S)| dq at the state w (full layout) for the eigenvalue splitting A+- = (A +- |A|)/2 of
 * Sec. 2.3, |A| = R |Lambda| R^-1.  A has the eigenvalue U_n (all waves but the two acoustic
 * ones) and U_n +- c, with right eigenvectors (Y_s, u +- c n, H +- U_n c, e_v) per unit
 * normal n and projections alpha+- = (dp +- rho c dU_n) / (2 c^2) (dp the linearised
 * pressure of jvp_full, dU_n = (n.dm - U_n d rho)/rho), so that
 *   |A| dq = |S| (|U_n| dq + (|U_n+c| - |U_n|) alpha+ r+ + (|U_n-c| - |U_n|) alpha- r-),
 * the same wave decomposition as the Roe dissipation, at one state. */
static void absjac_full(const orc_grid *G, const prim_t *w, const double *S, const double *dq, double *out)
{
    int ns = G->gas.ns, nd = G->nd, two = G->gas.ntemp == 2;
    double area = 0.0;
    for (int q = 0; q < nd; q++) area += S[q] * S[q];
    area = sqrt(area);
    double n[3] = {0, 0, 0};
    for (int q = 0; q < nd; q++) n[q] = S[q] / area;
    double drho = 0.0, dp = 0.0, Un = 0.0, ndm = 0.0;
    for (int s = 0; s < ns; s++) { drho += dq[s]; dp += w->prs[s] * dq[s]; }
    for (int q = 0; q < nd; q++) {
        Un += w->u[q] * n[q];
        ndm += n[q] * dq[ns + q];
        dp -= w->beta * w->u[q] * dq[ns + q];
    }
    dp += w->beta * dq[ns + nd];
    if (two) dp += w->prev * dq[ns + nd + 1];
    double dUn = (ndm - Un * drho) / w->rho;
    double c = w->c, c2 = c * c;
    double ap = (dp + w->rho * c * dUn) / (2.0 * c2), am = (dp - w->rho * c * dUn) / (2.0 * c2);
    double l0 = fabs(Un), lp = fabs(Un + c) - l0, lm = fabs(Un - c) - l0;
    double H = (w->rhoE + w->p) / w->rho;
    for (int s = 0; s < ns; s++) out[s] = area * (l0 * dq[s] + (lp * ap + lm * am) * w->Y[s]);
    for (int q = 0; q < nd; q++)
        out[ns + q] = area * (l0 * dq[ns + q] + lp * ap * (w->u[q] + c * n[q]) + lm * am * (w->u[q] - c * n[q]));
    out[ns + nd] = area * (l0 * dq[ns + nd] + lp * ap * (H + Un * c) + lm * am * (H - Un * c));
    if (two) out[ns + nd + 1] = area * (l0 * dq[ns + nd + 1] + (lp * ap + lm * am) * w->rhoev / w->rho);
}

/* |A(S)| in the coupled variables (the similarity transform of jvp_ci) */
static void absjac_ci(const orc_grid *G, const prim_t *w, const double *S, const double *dc, double *out)
{
    int ns = G->gas.ns, nF = G->nF;
    double dq[NQMAX], o[NQMAX];
    double first = dc[0];
    for (int s = 1; s < ns; s++) { dq[s] = dc[nF + s - 1]; first -= dc[nF + s - 1]; }
    dq[0] = first;
    for (int k = 1; k < nF; k++) dq[ns + k - 1] = dc[k];
    absjac_full(G, w, S, dq, o);
    double orho = 0.0;
    for (int s = 0; s < ns; s++) orho += o[s];
    out[0] = orho;
    for (int k = 1; k < nF; k++) out[k] = o[ns + k - 1];
    for (int s = 1; s < ns; s++) out[nF + s - 1] = o[s];
}

/* ---------------------------------------------------------------------------------------
 * LU-SGS sweeps (Sec. 2.2: (D+L) dQ* = RHS forward, (D+U) dQ = D dQ* backward, with the
 * spectral splitting A^+- = (A +- lambda I)/2 and the point equation Eq. (ijkiterate)).
 * Reading: RHS = -R; the neighbour nb on the minus side of direction d couples with
 * -(A_nb(S_f) + lambda_nb)/2, on the plus side with +(A_nb(S_f) - lambda_nb)/2, S_f the face
 * between the two cells; L holds the couplings to neighbours earlier in h = i+j+k order.
 * Cells are swept in lexicographic order (i fastest), which agrees with h order on every
 * neighbour pair; boundary neighbours contribute nothing (explicit boundary conditions).
 * ------------------------------------------------------------------------------------- */

/* accumulate -sum coef * x_nb over neighbours in L (lower = 1) or U (lower = 0) */
typedef void (*jvp_fn)(const orc_grid *, const prim_t *, const double *, const double *, double *);

static void gather(const orc_grid *G, int c, int lower, int nv, const double *x, size_t stride,
                   jvp_fn A, const double *lam, double *acc)
{
    int o[3];
    cell_coords(G, c, o);
    for (int d = 0; d < G->nd; d++)
        for (int s = -1; s <= 1; s += 2) {
            int hl, nb = neighbour(G, o, d, s, &hl);
            if (nb < 0 || hl != lower) continue;
            const double *Sf = &G->S[d][3 * face_of(G, o, d, s)];
            double xn[NQMAX], ax[NQMAX];
            for (int v = 0; v < nv; v++) xn[v] = x[(size_t)v * stride + nb];
            A(G, &G->w[nb], Sf, xn, ax);
            double l = lam[3 * nb + d];
            for (int v = 0; v < nv; v++) {
                if (s < 0) acc[v] += 0.5 * (ax[v] + l * xn[v]);
                else acc[v] -= 0.5 * (ax[v] - l * xn[v]);
            }
        }
}

/* coupled operator with the eigenvalue splitting: the neighbour couples with
 * -(A_nb(S_f) + |A_nb(S_f)| + 2 lambda_vis)/2 (minus side) or +(A_nb - |A_nb| - 2 lambda_vis)/2 */
static void gather_ci_eigen(const orc_grid *G, int c, int lower, const double *x, double *acc)
{
    int o[3], n = G->nci, N = G->ncell;
    cell_coords(G, c, o);
    for (int d = 0; d < G->nd; d++)
        for (int s = -1; s <= 1; s += 2) {
            int hl, nb = neighbour(G, o, d, s, &hl);
            if (nb < 0 || hl != lower) continue;
            const double *Sf = &G->S[d][3 * face_of(G, o, d, s)];
            double xn[NQMAX], ax[NQMAX], bx[NQMAX];
            for (int v = 0; v < n; v++) xn[v] = x[(size_t)v * N + nb];
            jvp_ci(G, &G->w[nb], Sf, xn, ax);
            absjac_ci(G, &G->w[nb], Sf, xn, bx);
            double l = G->lamCIv[3 * nb + d];
            for (int v = 0; v < n; v++) {
                if (s < 0) acc[v] += 0.5 * (ax[v] + bx[v] + l * xn[v]);
                else acc[v] -= 0.5 * (ax[v] - bx[v] - l * xn[v]);
            }
        }
}

/* component operator (Sec. 2.3.2): Jacobian U I for every species */
static double face_U(const orc_grid *G, const prim_t *w, const double *S)
{
    double U = 0.0;
    for (int q = 0; q < G->nd; q++) U += w->u[q] * S[q];
    return U;
}
static void gather_species(const orc_grid *G, int c, int lower, const double *x, double *acc)
{
    int o[3], ns = G->gas.ns;
    cell_coords(G, c, o);
    for (int d = 0; d < G->nd; d++)
        for (int s = -1; s <= 1; s += 2) {
            int hl, nb = neighbour(G, o, d, s, &hl);
            if (nb < 0 || hl != lower) continue;
            const double *Sf = &G->S[d][3 * face_of(G, o, d, s)];
            double U = face_U(G, &G->w[nb], Sf), l = G->lamC[3 * nb + d];
            for (int k = 0; k < ns; k++) {
                double xn = x[(size_t)k * G->ncell + nb];
                if (s < 0) acc[k] += 0.5 * (U * xn + l * xn);
                else acc[k] -= 0.5 * (U * xn - l * xn);
            }
        }
}

/* split operator: dQ layout (rho, m, rhoE, [rho e_v], rho_1..rho_ns) */
static int lusgs_split(orc_grid *G, double cfl)
{
    if (!G->have_R) { snprintf(G->err, sizeof(G->err), "residual not evaluated"); return 7; }
    int N = G->ncell, nF = G->nF, ns = G->gas.ns, nd = G->nd;
    spectral(G, cfl);
    double *x = G->dQs, *y = G->dQ;
    /* forward sweep */
    for (int c = 0; c < N; c++) {
        double acc[NQMAX], accs[NSMAX];
        /* RHS = -R for the flow block: (sum_s R_s, R_m, R_E, [R_ev]) */
        double rr = 0.0;
        for (int s = 0; s < ns; s++) rr += G->R[(size_t)s * N + c];
        acc[0] = -rr;
        for (int k = 1; k < nF; k++) acc[k] = -G->R[(size_t)(ns + k - 1) * N + c];
        for (int s = 0; s < ns; s++) accs[s] = -G->R[(size_t)s * N + c];
        gather(G, c, 1, nF, x, N, jvp_flow, G->lamF, acc);
        gather_species(G, c, 1, x + (size_t)nF * N, accs);
        for (int k = 0; k < nF; k++) {
            double D = (G->gas.ntemp == 2 && k == nF - 1) ? G->DFev[c] : G->DF[c];
            x[(size_t)k * N + c] = acc[k] / D;
        }
        for (int s = 0; s < ns; s++) x[(size_t)(nF + s) * N + c] = accs[s] / G->Ds[(size_t)s * N + c];
    }
    /* backward sweep */
    for (int c = N - 1; c >= 0; c--) {
        double acc[NQMAX], accs[NSMAX];
        for (int k = 0; k < nF; k++) acc[k] = 0.0;
        for (int s = 0; s < ns; s++) accs[s] = 0.0;
        gather(G, c, 0, nF, y, N, jvp_flow, G->lamF, acc);
        gather_species(G, c, 0, y + (size_t)nF * N, accs);
        for (int k = 0; k < nF; k++) {
            double D = (G->gas.ntemp == 2 && k == nF - 1) ? G->DFev[c] : G->DF[c];
            y[(size_t)k * N + c] = x[(size_t)k * N + c] + acc[k] / D;
        }
        for (int s = 0; s < ns; s++)
            y[(size_t)(nF + s) * N + c] = x[(size_t)(nF + s) * N + c] + accs[s] / G->Ds[(size_t)s * N + c];
    }
    (void)nd;
    return 0;
}

/* coupled operator (Sec. 2.2 with the unified radius; Sec. 2.3.3 ns-1 species):
 * dQ layout (rho, m, rhoE, [rho e_v], rho_2..rho_ns) */
static int lusgs_coupled(orc_grid *G, double cfl)
{
    if (!G->have_R) { snprintf(G->err, sizeof(G->err), "residual not evaluated"); return 7; }
    int N = G->ncell, n = G->nci, nF = G->nF, ns = G->gas.ns;
    spectral(G, cfl);
    for (int c = 0; c < N; c++)
        if (lu_factor(&G->DLU[(size_t)c * n * n], &G->piv[(size_t)c * n], n)) {
            G->status_cell = c;
            snprintf(G->err, sizeof(G->err), "singular coupled diagonal block at cell %d", c);
            return 4;
        }
    double *x = G->dQci_s, *y = G->dQci;
    for (int c = 0; c < N; c++) {
        double acc[NQMAX];
        double rr = 0.0;
        for (int s = 0; s < ns; s++) rr += G->R[(size_t)s * N + c];
        acc[0] = -rr;
        for (int k = 1; k < nF; k++) acc[k] = -G->R[(size_t)(ns + k - 1) * N + c];
        for (int s = 1; s < ns; s++) acc[nF + s - 1] = -G->R[(size_t)s * N + c];
        if (G->ci_split) gather_ci_eigen(G, c, 1, x, acc);
        else gather(G, c, 1, n, x, N, jvp_ci, G->lamCI, acc);
        lu_solve(&G->DLU[(size_t)c * n * n], &G->piv[(size_t)c * n], n, acc);
        for (int k = 0; k < n; k++) x[(size_t)k * N + c] = acc[k];
    }
    for (int c = N - 1; c >= 0; c--) {
        double acc[NQMAX];
        for (int k = 0; k < n; k++) acc[k] = 0.0;
        if (G->ci_split) gather_ci_eigen(G, c, 0, y, acc);
        else gather(G, c, 0, n, y, N, jvp_ci, G->lamCI, acc);
        lu_solve(&G->DLU[(size_t)c * n * n], &G->piv[(size_t)c * n], n, acc);
        for (int k = 0; k < n; k++) y[(size_t)k * N + c] = x[(size_t)k * N + c] + acc[k];
    }
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * Consistency corrections and update (Sec. 2.3.3).
 * Reading: the weight of correction 1 is W_s = rho_s^m / sum_r rho_r^m (the printed weight
 * does not sum to one, contradicting the conservation statement that follows it).  With
 * clip = 1, negative densities are set to zero (commented-out remark at the end of Sec. 2.3.3)
 * and counted.  mode 1: CS-1, mode 2: CS-2, mode 0: coupled (CI) update with the
 * eliminated (first) species = rho - sum of the others.
 * Update limit (not in the paper; off unless set): with f = update_limit > 0, the cell's whole
 * increment is scaled by alpha = min(1, f rho / |d rho|) before the corrections, so that no
 * iteration changes a cell's density by more than the fraction f; alpha is then halved (at
 * most 30 times) while the corrected state is non-physical or its specific thermal energies
 * leave the band: e_tr = (rho E - |m|^2/(2 rho) [- rho e_v] - sum_s rho_s h0_s)/rho, which is
 * proportional to the translational(-rotational) temperature, within a factor 1 + f of the
 * old value, and (2T) the pool's e_v = rho e_v / rho gaining at most f (e_tr + e_v) of the
 * old values.  alpha = 1 once the increments are small, so the converged solution is
 * unchanged; it only carries an impulsively started hypersonic flow through its start-up
 * transient at large CFL (where a cell can otherwise, e.g., dissociate more than its thermal
 * energy can pay for, or take the energy of an arriving shock before its density).
 * ------------------------------------------------------------------------------------- */

/* New conserved state qn of cell c for the increment alpha * dq with the correction of
 * `mode`; returns 0, or 4 (message in G->err) for a non-physical result.  *ncl counts the
 * values that were clipped. */
static int cell_update(orc_grid *G, int mode, int clip, const double *dqall, int c,
                       double alpha, double *qn, int *ncl)
{
    int N = G->ncell, ns = G->gas.ns, nF = G->nF;
    int nv = (mode == 0) ? G->nci : G->nsplit;
    double rho = 0.0, rs[NSMAX], dloc[NQMAX + NSMAX];
    *ncl = 0;
    for (int s = 0; s < ns; s++) { rs[s] = G->Q[(size_t)s * N + c]; rho += rs[s]; }
    for (int k = 0; k < nv; k++) dloc[k] = alpha * dqall[(size_t)k * N + c];
    double drho = dloc[0];
    double rnew = rho + drho;
    if (!(rnew > 0.0)) {
        snprintf(G->err, sizeof(G->err), "non-positive density after update at cell %d", c);
        return 4;
    }
    double out[NSMAX];
    if (mode == 1) {
        double sd = 0.0;
        for (int s = 0; s < ns; s++) sd += dloc[nF + s];
        for (int s = 0; s < ns; s++)
            out[s] = rs[s] + dloc[nF + s] + (rs[s] / rho) * (drho - sd);
    } else if (mode == 2) {
        double t[NSMAX], sum = 0.0;
        for (int s = 0; s < ns; s++) {
            t[s] = rs[s] + dloc[nF + s];
            if (clip && t[s] < 0.0) { t[s] = 0.0; (*ncl)++; }
            sum += t[s];
        }
        if (!(sum > 0.0)) {
            snprintf(G->err, sizeof(G->err), "non-positive species sum at cell %d", c);
            return 4;
        }
        for (int s = 0; s < ns; s++) out[s] = rnew * t[s] / sum;
    } else {
        double sum = 0.0;
        for (int s = 1; s < ns; s++) { out[s] = rs[s] + dloc[nF + s - 1]; sum += out[s]; }
        out[0] = rnew - sum;
    }
    for (int s = 0; s < ns; s++) {
        if (clip && out[s] < 0.0 && mode != 2) { out[s] = 0.0; (*ncl)++; }
        qn[s] = out[s];
    }
    for (int k = 1; k < nF; k++) {
        double v = G->Q[(size_t)(ns + k - 1) * N + c] + dloc[k];
        if (clip && G->gas.ntemp == 2 && k == nF - 1 && v < 0.0) { v = 0.0; (*ncl)++; }
        qn[ns + k - 1] = v;
    }
    return 0;
}

/* specific energies of a conserved state: e[0] = translational(-rotational) thermal energy per
 * unit mass (formation energy, kinetic energy [and the pool] taken out), e[1] = pool energy per
 * unit mass (2T; 0 for 1T) */
static void specific_thermal(const orc_grid *G, const double *q, double *e)
{
    int ns = G->gas.ns, nd = G->nd;
    double rho = 0.0, m2 = 0.0, et = q[ns + nd];
    for (int s = 0; s < ns; s++) rho += q[s];
    for (int d = 0; d < nd; d++) m2 += q[ns + d] * q[ns + d];
    et -= 0.5 * m2 / rho;
    for (int s = 0; s < ns; s++) et -= q[s] * G->gas.hf[s];
    e[1] = 0.0;
    if (G->gas.ntemp == 2) {
        et -= q[ns + nd + 1];
        e[1] = q[ns + nd + 1] / rho;
    }
    e[0] = et / rho;
}

/* is the updated state qn inside the update limit's band around q0? */
static int within_limit(const orc_grid *G, const double *q0, const double *qn, double f)
{
    double e0[2], en[2];
    specific_thermal(G, q0, e0);
    if (!(e0[0] > 0.0)) return 1;               /* no band without a positive thermal energy */
    specific_thermal(G, qn, en);
    if (!(en[0] * (1.0 + f) >= e0[0] && en[0] <= (1.0 + f) * e0[0])) return 0;
    if (G->gas.ntemp == 2 && !(en[1] <= e0[1] + f * (e0[0] + e0[1]))) return 0;
    return 1;
}

static int correct_update(orc_grid *G, int mode, int clip, const double *dq)
{
    int N = G->ncell, ns = G->gas.ns, nq = G->nq;
    double f = G->update_limit;
    G->nclip = 0;
    for (int c = 0; c < N; c++) {
        double rho = 0.0, q0[NQMAX], qn[NQMAX];
        for (int v = 0; v < nq; v++) q0[v] = G->Q[(size_t)v * N + c];
        for (int s = 0; s < ns; s++) rho += q0[s];
        double alpha = 1.0;
        if (f > 0.0 && fabs(dq[c]) > f * rho) alpha = f * rho / fabs(dq[c]);
        int ncl = 0;
        int st = cell_update(G, mode, clip, dq, c, alpha, qn, &ncl);
        if (f > 0.0) {
            for (int it = 0; it < 30 && (st || !within_limit(G, q0, qn, f)); it++) {
                alpha *= 0.5;
                st = cell_update(G, mode, clip, dq, c, alpha, qn, &ncl);
            }
        }
        if (st) {
            G->status_cell = c;
            return st;
        }
        for (int v = 0; v < nq; v++) G->Q[(size_t)v * N + c] = qn[v];
        G->nclip += ncl;
    }
    G->have_R = 0;
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * Public oracle API (host pointers only).
 * ------------------------------------------------------------------------------------- */
int orc_create(int nd, int ni, int nj, int nk, const int *bc, int mech, int lim, double efix,
               const double *nodes, orc_grid **out)
{
    if (nd < 2 || nd > 3 || ni < 2 || nj < 1 || (nd == 3 && nk < 1)) return 1;
    orc_grid *G = calloc(1, sizeof(orc_grid));
    if (!G) return 2;
    if (gas_init(&G->gas, mech)) { free(G); return 1; }
    G->nd = nd; G->n[0] = ni; G->n[1] = nj; G->n[2] = (nd == 3) ? nk : 1;
    for (int k = 0; k < 6; k++) G->bc[k] = bc[k];
    G->limiter = lim; G->efix = efix; G->hcorr = 1; G->viscous = 1;
    G->ncell = ni * nj * G->n[2];
    int ns = G->gas.ns;
    G->nq = ns + nd + 1 + (G->gas.ntemp == 2);
    G->nF = 1 + nd + 1 + (G->gas.ntemp == 2);
    G->nsplit = G->nF + ns;
    G->nci = G->nF + ns - 1;
    size_t nn = (size_t)(ni + 1) * (nj + 1) * (nd == 3 ? nk + 1 : 1), N = G->ncell;
    for (int d = 0; d < nd; d++) {
        G->node[d] = malloc(sizeof(double) * nn);
        memcpy(G->node[d], nodes + d * nn, sizeof(double) * nn);
        G->nf[d] = (ni + (d == 0)) * (nj + (d == 1)) * (nd == 3 ? nk + (d == 2) : 1);
        G->S[d] = calloc((size_t)G->nf[d] * 3, sizeof(double));
        G->fc[d] = calloc((size_t)G->nf[d] * 3, sizeof(double));
        G->Fface[d] = calloc((size_t)G->nf[d] * G->nq, sizeof(double));
    }
    G->V = calloc(N, sizeof(double));
    G->xc = calloc(N * 3, sizeof(double));
    G->Q = calloc(N * G->nq, sizeof(double));
    G->R = calloc(N * G->nq, sizeof(double));
    G->dQs = calloc(N * G->nsplit, sizeof(double));
    G->dQ = calloc(N * G->nsplit, sizeof(double));
    G->dQci_s = calloc(N * G->nci, sizeof(double));
    G->dQci = calloc(N * G->nci, sizeof(double));
    G->w = calloc(N, sizeof(prim_t));
    G->grad = calloc(N * NGMAX * 3, sizeof(double));
    G->lamF = calloc(N * 3, sizeof(double));
    G->lamC = calloc(N * 3, sizeof(double));
    G->lamCI = calloc(N * 3, sizeof(double));
    G->lamCIv = calloc(N * 3, sizeof(double));
    G->DF = calloc(N, sizeof(double));
    G->DFev = calloc(N, sizeof(double));
    G->Ds = calloc(N * ns, sizeof(double));
    G->DLU = calloc(N * G->nci * G->nci, sizeof(double));
    G->piv = calloc(N * G->nci, sizeof(int));
    compute_geometry(G);
    G->stag_cell = -1;
    G->react = 1;
    *out = G;
    return 0;
}

/* reacting = 0 switches the chemical and vibrational sources off */
int orc_set_reacting(orc_grid *G, int reacting) { G->react = reacting != 0; return 0; }
/* H-correction of the entropy fix on (1, the default) or off (0) */
int orc_set_hcorr(orc_grid *G, int on) { G->hcorr = on != 0; return 0; }

/* Inviscid flow (a test switch): off drops the viscous and diffusive fluxes from the residual
 * and the viscous radii from the operator (mu = k = rho D = 0 in both). */
int orc_set_viscous(orc_grid *G, int on) { G->viscous = on != 0; return 0; }

/* Transport model: 0 Sutherland viscosity with constant Prandtl and Schmidt numbers (one
 * diffusion coefficient), 1 the species model (Blottner, Eucken, Wilke, Blanc; air only). */
int orc_set_transport(orc_grid *G, int model)
{
    if (model != 0 && model != 1) return 1;
    if (model == 1 && G->gas.mech == 0) return 1;
    G->gas.transport = model;
    return 0;
}
/* update limit f (see correct_update); 0 switches it off */
int orc_set_update_limit(orc_grid *G, double f) { if (!(f >= 0.0)) return 1; G->update_limit = f; return 0; }

/* flux-Jacobian splitting of the coupled operator: 0 spectral (the paper's choice), 1 the
 * eigenvalue splitting A+- = (A +- |A|)/2 */
int orc_set_ci_splitting(orc_grid *G, int mode)
{
    if (mode != 0 && mode != 1) return 1;
    G->ci_split = mode;
    return 0;
}

/* Local time step of Sec. 2.2 with (1) or without (0, default) the source term's radius
 * lambda_S in its denominator. */
int orc_set_dtau_source(orc_grid *G, int on)
{
    if (on != 0 && on != 1) return 1;
    G->dtau_src = on;
    return 0;
}

/* dual time stepping: physical step dt (0 switches it off) and theta >= 0; the stored levels
 * are discarded (the next orc_dual_advance starts from the current state) */
int orc_set_dual(orc_grid *G, double dt, double theta)
{
    if (!(dt >= 0.0) || !(theta >= 0.0)) return 1;
    size_t n = (size_t)G->nq * G->ncell;
    if (dt > 0.0 && !G->Qn) {
        G->Qn = calloc(n, sizeof(double));
        G->Qnm1 = calloc(n, sizeof(double));
        if (!G->Qn || !G->Qnm1) return 1;
    }
    G->dual_dt = dt;
    G->dual_theta = theta;
    G->dual_levels = 0;
    G->have_R = 0;
    return 0;
}

/* begin a physical time step from the current state: Q^{n-1} <- Q^n, Q^n <- Q */
int orc_dual_advance(orc_grid *G)
{
    if (!(G->dual_dt > 0.0) || !G->Qn) return 1;
    size_t n = (size_t)G->nq * G->ncell;
    memcpy(G->Qnm1, G->Qn, n * sizeof(double));
    memcpy(G->Qn, G->Q, n * sizeof(double));
    if (G->dual_levels < 2) G->dual_levels++;
    G->have_R = 0;
    return 0;
}

void orc_destroy(orc_grid *G)
{
    if (!G) return;
    for (int d = 0; d < G->nd; d++) { free(G->node[d]); free(G->S[d]); free(G->fc[d]); free(G->Fface[d]); }
    free(G->V); free(G->xc); free(G->Q); free(G->R); free(G->dQs); free(G->dQ); free(G->dQci_s);
    free(G->dQci); free(G->w); free(G->grad); free(G->lamF); free(G->lamC); free(G->lamCI); free(G->lamCIv);
    free(G->DF); free(G->DFev); free(G->Ds); free(G->DLU); free(G->piv);
    free(G->Qn); free(G->Qnm1);
    free(G);
}

/* Set freestream (T, Tv, p, Mach, Y[ns], direction) and wall temperature.  The freestream
 * velocity is Mach times the frozen sound speed of the freestream state. */
int orc_set_boundary(orc_grid *G, double T, double Tv, double p, double mach, const double *Y,
                     const double *dir, double Tw)
{
    gas_t *g = &G->gas;
    int ns = g->ns, nd = G->nd;
    double Rmix = 0.0;
    for (int s = 0; s < ns; s++) Rmix += Y[s] * g->Rs[s] * ((g->ntemp == 2 && !is_heavy(g, s)) ? Tv / T : 1.0);
    double rho = p / (Rmix * T), rhos[NSMAX], u0[3] = {0, 0, 0}, q[NQMAX];
    for (int s = 0; s < ns; s++) rhos[s] = rho * Y[s];
    cons_from_prim(g, nd, rhos, u0, T, Tv, q);
    prim_t w0;
    if (prim_from_cons(g, nd, q, T, Tv, &w0)) return 4;
    double dn = 0.0, u[3];
    for (int d = 0; d < nd; d++) dn += dir[d] * dir[d];
    dn = sqrt(dn);
    for (int d = 0; d < nd; d++) u[d] = mach * w0.c * dir[d] / dn;
    cons_from_prim(g, nd, rhos, u, T, Tv, G->fsQ);
    if (prim_from_cons(g, nd, G->fsQ, T, Tv, &G->fs)) return 4;
    cell_sources(g, nd, &G->fs);
    G->Tw = Tw;
    /* stagnation wall cell: j = 0, normal most nearly opposite the freestream */
    G->stag_cell = -1;
    if (G->bc[2] == BC_WALL) {
        double best = 1e300;
        int lk = (nd == 3) ? G->n[2] : 1;
        for (int k = 0; k < lk; k++)
            for (int i = 0; i < G->n[0]; i++) {
                int o[3] = {i, 0, k};
                const double *Sf = &G->S[1][3 * face_of(G, o, 1, -1)];
                double a = 0.0, dd = 0.0;
                for (int q2 = 0; q2 < nd; q2++) { a += Sf[q2] * Sf[q2]; dd += Sf[q2] * dir[q2]; }
                if (a <= 0.0) continue;
                dd /= sqrt(a) * dn;
                if (dd < best - 1e-12) { best = dd; G->stag_cell = cidx(G, i, 0, k); }
            }
    }
    return 0;
}

void orc_freestream_state(const orc_grid *G, double *Q)
{
    for (int v = 0; v < G->nq; v++)
        for (int c = 0; c < G->ncell; c++) Q[(size_t)v * G->ncell + c] = G->fsQ[v];
}

int orc_set_state(orc_grid *G, const double *Q)
{
    memcpy(G->Q, Q, sizeof(double) * G->ncell * G->nq);
    for (int c = 0; c < G->ncell; c++) { G->w[c].T = 0.0; G->w[c].Tv = 0.0; }
    G->have_R = 0;
    G->iter = 0;
    return 0;
}
void orc_get_state(const orc_grid *G, double *Q) { memcpy(Q, G->Q, sizeof(double) * G->ncell * G->nq); }

int orc_residual(orc_grid *G, double *R, double *norms)
{
    int st = residual(G);
    if (st) return st;
    if (R) memcpy(R, G->R, sizeof(double) * G->ncell * G->nq);
    if (norms) { norms[0] = G->norms[0]; norms[1] = G->norms[1]; norms[2] = G->qstag; }
    return 0;
}

int orc_lusgs_split(orc_grid *G, double cfl, double *dQ)
{
    int st = lusgs_split(G, cfl);
    if (!st && dQ) memcpy(dQ, G->dQ, sizeof(double) * G->ncell * G->nsplit);
    return st;
}

int orc_lusgs_coupled(orc_grid *G, double cfl, double *dQ)
{
    int st = lusgs_coupled(G, cfl);
    if (!st && dQ) memcpy(dQ, G->dQci, sizeof(double) * G->ncell * G->nci);
    return st;
}

int orc_correct(orc_grid *G, int mode, int clip, const double *dQ, int *nclip)
{
    const double *d = dQ ? dQ : (mode == 0 ? G->dQci : G->dQ);
    int st = correct_update(G, mode, clip, d);
    if (nclip) *nclip = G->nclip;
    return st;
}

/* One or more pseudo-time iterations (Sec. 2.2-2.3): residual, implicit operator (split or
 * coupled), correction + update.  CFL ramps geometrically from cfl_start to cfl over
 * ramp_iters iterations (reading; the paper gives fixed CFL numbers).
 * stats: [iters_done, r_species, r_energy, q_stag, nclip] of the last iteration. */
int orc_step(orc_grid *G, int scheme, int correction, int clip, double cfl, double cfl_start,
             int ramp_iters, int iters, double *stats)
{
    int st = 0, done = 0;
    for (int it = 0; it < iters; it++) {
        double c = cfl;
        if (ramp_iters > 0 && G->iter < ramp_iters && cfl_start > 0.0)
            c = cfl_start * pow(cfl / cfl_start, (double)G->iter / (double)ramp_iters);
        st = residual(G);
        if (st) break;
        if (scheme == 0) { st = lusgs_split(G, c); if (!st) st = correct_update(G, correction, clip, G->dQ); }
        else { st = lusgs_coupled(G, c); if (!st) st = correct_update(G, 0, clip, G->dQci); }
        if (st) break;
        G->iter++;
        done++;
    }
    if (stats) {
        stats[0] = done; stats[1] = G->norms[0]; stats[2] = G->norms[1]; stats[3] = G->qstag;
        stats[4] = G->nclip;
    }
    return st;
}

const char *orc_last_error(const orc_grid *G) { return G->err; }
int orc_dims(const orc_grid *G, int *out)
{
    out[0] = G->ncell; out[1] = G->nq; out[2] = G->nsplit; out[3] = G->nci; out[4] = G->gas.ns;
    out[5] = G->gas.ntemp; out[6] = G->nF; out[7] = G->stag_cell;
    return 0;
}

/* Copy internal per-cell or per-face arrays (test access).  Returns the number of doubles
 * written, or -1 for an unknown name. */
int orc_field(const orc_grid *G, const char *name, double *out)
{
    int N = G->ncell, ns = G->gas.ns;
    if (!strcmp(name, "V")) { memcpy(out, G->V, sizeof(double) * N); return N; }
    if (!strcmp(name, "xc")) { memcpy(out, G->xc, sizeof(double) * N * 3); return N * 3; }
    for (int d = 0; d < G->nd; d++) {
        char nm[16];
        snprintf(nm, sizeof nm, "S%d", d);
        if (!strcmp(name, nm)) { memcpy(out, G->S[d], sizeof(double) * G->nf[d] * 3); return G->nf[d] * 3; }
        snprintf(nm, sizeof nm, "F%d", d);
        if (!strcmp(name, nm)) { memcpy(out, G->Fface[d], sizeof(double) * G->nf[d] * G->nq); return G->nf[d] * G->nq; }
    }
    if (!strcmp(name, "lamF")) { memcpy(out, G->lamF, sizeof(double) * N * 3); return N * 3; }
    if (!strcmp(name, "lamC")) { memcpy(out, G->lamC, sizeof(double) * N * 3); return N * 3; }
    if (!strcmp(name, "lamCI")) { memcpy(out, G->lamCI, sizeof(double) * N * 3); return N * 3; }
    if (!strcmp(name, "lamCIv")) { memcpy(out, G->lamCIv, sizeof(double) * N * 3); return N * 3; }
    if (!strcmp(name, "DF")) { memcpy(out, G->DF, sizeof(double) * N); return N; }
    if (!strcmp(name, "DFev")) { memcpy(out, G->DFev, sizeof(double) * N); return N; }
    if (!strcmp(name, "Ds")) { memcpy(out, G->Ds, sizeof(double) * N * ns); return N * ns; }
    if (!strcmp(name, "Dci")) {
        /* unfactored coupled diagonal blocks (valid after orc_build_diagonals) */
        memcpy(out, G->DLU, sizeof(double) * N * G->nci * G->nci);
        return N * G->nci * G->nci;
    }
    if (!strcmp(name, "grad")) { memcpy(out, G->grad, sizeof(double) * N * NGMAX * 3); return N * NGMAX * 3; }
    if (!strcmp(name, "dQstar")) { memcpy(out, G->dQs, sizeof(double) * N * G->nsplit); return N * G->nsplit; }
    if (!strcmp(name, "dQci_star")) { memcpy(out, G->dQci_s, sizeof(double) * N * G->nci); return N * G->nci; }
#define CELLF(nm, expr) if (!strcmp(name, nm)) { for (int c = 0; c < N; c++) out[c] = G->w[c].expr; return N; }
    CELLF("T", T) CELLF("Tv", Tv) CELLF("p", p) CELLF("c", c) CELLF("beta", beta) CELLF("rho", rho)
    CELLF("mu", mu) CELLF("kt", kt) CELLF("kv", kv) CELLF("rhoD", rhoD) CELLF("omega_v", omega_v)
    CELLF("relax", relax) CELLF("Gam", Gam) CELLF("H", H) CELLF("cv", cv) CELLF("cvtr", cvtr) CELLF("cvve", cvve)
#undef CELLF
    if (!strcmp(name, "omega")) { for (int s = 0; s < ns; s++) for (int c = 0; c < N; c++) out[(size_t)s * N + c] = G->w[c].omega[s]; return N * ns; }
    if (!strcmp(name, "rhoDs")) { for (int s = 0; s < ns; s++) for (int c = 0; c < N; c++) out[(size_t)s * N + c] = G->w[c].rhoDs[s]; return N * ns; }
    if (!strcmp(name, "dom")) { for (int s = 0; s < ns; s++) for (int c = 0; c < N; c++) out[(size_t)s * N + c] = G->w[c].dom[s]; return N * ns; }
    if (!strcmp(name, "prs")) { for (int s = 0; s < ns; s++) for (int c = 0; c < N; c++) out[(size_t)s * N + c] = G->w[c].prs[s]; return N * ns; }
    return -1;
}

/* Build the spectral radii and diagonals for a given CFL without sweeping (test access). */
int orc_build_diagonals(orc_grid *G, double cfl)
{
    if (!G->have_R) return 7;
    spectral(G, cfl);
    return 0;
}

/* Apply the off-diagonal coupling of neighbour nb onto cell c (test access for the assembled
 * operator): out = coefficient block (nv x nv, row-major) of the point equation for the pair,
 * for scheme 0 = split flow block, 1 = split species (diagonal, nv = ns), 2 = coupled. */
int orc_coupling_block(orc_grid *G, int c, int d, int side, int scheme, double *out, int *nb_out)
{
    int o[3], hl;
    cell_coords(G, c, o);
    int nb = neighbour(G, o, d, side, &hl);
    *nb_out = nb;
    if (nb < 0) return 1;
    const double *Sf = &G->S[d][3 * face_of(G, o, d, side)];
    int nv = scheme == 0 ? G->nF : scheme == 1 ? G->gas.ns : G->nci;
    const double *lam = scheme == 0 ? G->lamF : scheme == 1 ? G->lamC : scheme == 2 ? G->lamCI : G->lamCIv;
    double l = lam[3 * nb + d];
    for (int col = 0; col < nv; col++) {
        double e[NQMAX] = {0}, a[NQMAX], b[NQMAX] = {0};
        e[col] = 1.0;
        if (scheme == 0) jvp_flow(G, &G->w[nb], Sf, e, a);
        else if (scheme >= 2) jvp_ci(G, &G->w[nb], Sf, e, a);
        else { double U = face_U(G, &G->w[nb], Sf); for (int r = 0; r < nv; r++) a[r] = (r == col) ? U : 0.0; }
        if (scheme == 3) absjac_ci(G, &G->w[nb], Sf, e, b);     /* eigenvalue splitting */
        for (int r = 0; r < nv; r++) {
            double dis = b[r] + (r == col ? l : 0.0);
            out[r * nv + col] = (side < 0) ? -0.5 * (a[r] + dis) : 0.5 * (a[r] - dis);
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * Single-state entry points for the pins (no grid).
 * ------------------------------------------------------------------------------------- */
int orc_gas_info(int mech, double *M, double *hf, int *dims)
{
    gas_t g;
    if (gas_init(&g, mech)) return 1;
    for (int s = 0; s < g.ns; s++) { M[s] = g.M[s]; hf[s] = g.hf[s]; }
    dims[0] = g.ns; dims[1] = g.nr; dims[2] = g.ntemp;
    return 0;
}

/* prim record summary: out = [T, Tv, p, c, beta, rho, Gam, H, mu, kt, kv, rhoD, cvtr, cvve, cv,
 * prev, prs[0..ns-1]] */
int orc_state_prim(int mech, int nd, const double *q, double *out)
{
    gas_t g;
    if (gas_init(&g, mech)) return 1;
    prim_t w;
    int st = prim_from_cons(&g, nd, q, 0.0, 0.0, &w);
    if (st) return st;
    double v[16] = {w.T, w.Tv, w.p, w.c, w.beta, w.rho, w.Gam, w.H, w.mu, w.kt, w.kv, w.rhoD,
                    w.cvtr, w.cvve, w.cv, w.prev};
    memcpy(out, v, sizeof v);
    for (int s = 0; s < g.ns; s++) out[16 + s] = w.prs[s];
    return 0;
}

int orc_state_cons(int mech, int nd, const double *rhos, const double *u, double T, double Tv, double *q)
{
    gas_t g;
    if (gas_init(&g, mech)) return 1;
    cons_from_prim(&g, nd, rhos, u, T, Tv, q);
    return 0;
}

/* physical Euler flux F(Q).S */
int orc_state_flux(int mech, int nd, const double *q, const double *S, double *F)
{
    orc_grid G;
    memset(&G, 0, sizeof G);
    if (gas_init(&G.gas, mech)) return 1;
    G.nd = nd; G.nq = G.gas.ns + nd + 1 + (G.gas.ntemp == 2);
    prim_t w;
    int st = prim_from_cons(&G.gas, nd, q, 0.0, 0.0, &w);
    if (st) return st;
    double v[NQMAX + 4], Qd[NQMAX];
    recon_pack(&G, &w, v);
    recon_t r;
    recon_unpack(&G, v, &r);
    state_flux(&G, &r, S, Qd, F);
    return 0;
}

int orc_state_roe(int mech, int nd, const double *qL, const double *qR, const double *S, double efix, double *F)
{
    orc_grid G;
    memset(&G, 0, sizeof G);
    if (gas_init(&G.gas, mech)) return 1;
    G.nd = nd; G.nq = G.gas.ns + nd + 1 + (G.gas.ntemp == 2); G.efix = efix;
    prim_t wl, wr;
    if (prim_from_cons(&G.gas, nd, qL, 0.0, 0.0, &wl) || prim_from_cons(&G.gas, nd, qR, 0.0, 0.0, &wr)) return 4;
    double vl[NQMAX + 4], vr[NQMAX + 4];
    recon_pack(&G, &wl, vl);
    recon_pack(&G, &wr, vr);
    recon_t L, R;
    recon_unpack(&G, vl, &L);
    recon_unpack(&G, vr, &R);
    roe_flux(&G, &L, &R, S, 0.0, F);
    return 0;
}

/* Jacobian-vector product: which = 0 full conserved, 1 flow block, 2 coupled variables */
int orc_state_jvp(int mech, int nd, const double *q, const double *S, int which, const double *dq, double *out)
{
    orc_grid G;
    memset(&G, 0, sizeof G);
    if (gas_init(&G.gas, mech)) return 1;
    G.nd = nd; G.nq = G.gas.ns + nd + 1 + (G.gas.ntemp == 2);
    G.nF = 1 + nd + 1 + (G.gas.ntemp == 2); G.nci = G.nF + G.gas.ns - 1;
    prim_t w;
    int st = prim_from_cons(&G.gas, nd, q, 0.0, 0.0, &w);
    if (st) return st;
    if (which == 0) jvp_full(&G, &w, S, dq, out);
    else if (which == 1) jvp_flow(&G, &w, S, dq, out);
    else if (which == 2) jvp_ci(&G, &w, S, dq, out);
    else if (which == 3) absjac_full(&G, &w, S, dq, out);
    else absjac_ci(&G, &w, S, dq, out);
    return 0;
}

/* chemistry of a state at given temperatures: omega[ns], J[ns*ns] */
int orc_state_chem(int mech, const double *rhos, double T, double Tv, double *omega, double *J)
{
    gas_t g;
    if (gas_init(&g, mech)) return 1;
    chemistry(&g, rhos, T, Tv, omega, J);
    return 0;
}

int orc_lnKc(int mech, int r, double T, double *out)
{
    gas_t g;
    if (gas_init(&g, mech) || r < 0 || r >= g.nr) return 1;
    *out = lnKc(&g, r, T);
    return 0;
}

int orc_gibbs(int mech, int s, double T, double *out)
{
    gas_t g;
    if (gas_init(&g, mech) || s < 0 || s >= g.ns) return 1;
    *out = gibbs_RT(&g, s, T);
    return 0;
}

/* vibrational source pieces of a conserved state: out = [omega_v, relax, tau[0..ns-1]] */
int orc_state_vib(int mech, int nd, const double *q, double *out)
{
    gas_t g;
    if (gas_init(&g, mech)) return 1;
    prim_t w;
    int st = prim_from_cons(&g, nd, q, 0.0, 0.0, &w);
    if (st) return st;
    cell_sources(&g, nd, &w);
    out[0] = w.omega_v;
    out[1] = w.relax;
    for (int s = 0; s < g.ns; s++) out[2 + s] = w.tau[s];
    return 0;
}

/* species energies at given temperatures: out[s] = e_s(T, Tv) */
int orc_species_energy(int mech, double T, double Tv, double *out)
{
    gas_t g;
    if (gas_init(&g, mech)) return 1;
    for (int s = 0; s < g.ns; s++) out[s] = e_species(&g, s, T, Tv);
    return 0;
}

/* conserved-variable source Jacobian of a state: omega[ns], Jq[ns][nq] (full layout) */
int orc_state_source_jac(int mech, int nd, const double *q, double *omega, double *Jq)
{
    gas_t g;
    if (gas_init(&g, mech)) return 1;
    prim_t w;
    int st = prim_from_cons(&g, nd, q, 0.0, 0.0, &w);
    if (st) return st;
    source_jacobian(&g, nd, &w, omega, Jq);
    return 0;
}
