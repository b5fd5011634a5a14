"""Pins of the oracle's finite-rate chemistry (Sec. 2.1 source S; Park's air model, Sec. 3.2):
conservation laws the mass-action law must satisfy, equilibrium constants against a separate
statistical-mechanics derivation and against each other, detailed balance at equilibrium,
and Jacobians against finite differences."""
import math

import numpy as np
import pytest

import inputs
import oracle

KB, HPL, NAV, RU, PREF = 1.380649e-23, 6.62607015e-34, 6.02214076e26, 8314.462618, 101325.0
# element composition (N, O, charge) per species, in table order
COMP = {"N2": (2, 0, 0), "O2": (0, 2, 0), "NO": (1, 1, 0), "N": (1, 0, 0), "O": (0, 1, 0),
        "NO+": (1, 1, 1), "N2+": (2, 0, 1), "O2+": (0, 2, 1), "N+": (1, 0, 1), "O+": (0, 1, 1),
        "e-": (0, 0, -1)}


def air_state(mech, seed, rho=0.02):
    rng = np.random.default_rng(seed)
    ns = oracle.gas_info(mech)["ns"]
    Y = rng.uniform(0.05, 1.0, ns)
    if ns == 11:
        # electrons: charge neutral with the ions
        M = oracle.gas_info(mech)["M"]
        Y[10] = 0.0
        ions = sum(Y[s] / M[s] for s in range(5, 10))
        Y[10] = ions * M[10]
    Y /= Y.sum()
    return rho * Y


@pytest.mark.parametrize("mech", [inputs.MECH_AIR5, inputs.MECH_AIR11])
@pytest.mark.parametrize("T,Tv", [(3000.0, 3000.0), (8000.0, 5000.0), (15000.0, 9000.0)])
def test_mass_element_charge_conservation(mech, T, Tv):
    info = oracle.gas_info(mech)
    names = inputs.SPECIES[mech]
    rhos = air_state(mech, 4)
    om, _ = oracle.state_chem(mech, rhos, T, Tv)
    scale = np.max(np.abs(om))
    assert scale > 0
    assert abs(om.sum()) / scale < 1e-13
    for e in range(3):
        flux = sum(om[s] / info["M"][s] * COMP[names[s]][e] for s in range(info["ns"]))
        ref = sum(abs(om[s] / info["M"][s]) for s in range(info["ns"]))
        assert abs(flux) / ref < 1e-13


def stat_mech_lnKc_dissociation(M2, M1, thr, sigma, thv, g2, g1, dE0, T):
    """K_c of A2 <=> 2 A from partition functions per unit volume (kmol/m^3)."""
    def qtr(M):
        m = M / NAV
        return (2 * math.pi * m * KB * T / HPL ** 2) ** 1.5
    q_atom = qtr(M1) * g1
    q_mol = qtr(M2) * g2 * (T / (sigma * thr)) / (1 - math.exp(-thv / T))
    # K_c (molecules/m^3) = q_atom^2 / q_mol * exp(-D0/kT); divide by N_A for kmol/m^3
    return 2 * math.log(q_atom) - math.log(q_mol) - dE0 / (RU * T) - math.log(NAV)


@pytest.mark.parametrize("T", [2500.0, 5000.0, 10000.0])
def test_Kc_against_partition_functions(T):
    mech = inputs.MECH_AIR5
    M = oracle.gas_info(mech)["M"]
    # O2 <=> 2 O (reaction index 1): theta_r 2.08, sigma 2, theta_v 2239, g(O2)=3, g(O)=9
    ref = stat_mech_lnKc_dissociation(M[1], M[4], 2.08, 2, 2239.0, 3, 9, 2 * 246.79e6, T)
    assert abs(oracle.lnKc(mech, 1, T) - ref) < 1e-10
    # N2 <=> 2 N (reaction index 0)
    ref = stat_mech_lnKc_dissociation(M[0], M[3], 2.88, 2, 3395.0, 1, 4, 2 * 470.82e6, T)
    assert abs(oracle.lnKc(mech, 0, T) - ref) < 1e-10


@pytest.mark.parametrize("T", [1500.0, 6000.0, 20000.0])
def test_Kc_additivity(T):
    """Reactions that are sums of others have K_c products (thermodynamic consistency)."""
    m = inputs.MECH_AIR11
    k = [oracle.lnKc(m, r, T) for r in range(21)]
    assert abs(k[3] - (k[0] - k[2])) < 1e-9          # N2+O->NO+N = (N2->2N) - (NO->N+O)
    assert abs(k[4] - (k[2] - k[1])) < 1e-9          # NO+O->O2+N = (NO->N+O) - (O2->2O)
    assert abs(k[8] - (-k[5] + k[20] - k[1])) < 1e-9  # NO+ + O -> N+ + O2


def test_isothermal_reactor_detailed_balance():
    """A constant-volume isothermal reactor relaxes to the state where every reaction is in
    detailed balance (forward = backward), with elements conserved along the way."""
    mech = inputs.MECH_AIR5
    info = oracle.gas_info(mech)
    M = info["M"]
    names = inputs.SPECIES[mech]
    T = 4500.0
    rhos = np.array([0.767, 0.233, 0, 0, 0]) * 0.01
    elem0 = [sum(rhos[s] / M[s] * COMP[names[s]][e] for s in range(5)) for e in range(2)]
    dt = 1e-7
    for _ in range(4000):
        om, J = oracle.state_chem(mech, rhos, T)
        rhos = rhos + np.linalg.solve(np.eye(5) - dt * J, dt * om)
        dt = min(dt * 1.01, 1e-3)
    elem = [sum(rhos[s] / M[s] * COMP[names[s]][e] for s in range(5)) for e in range(2)]
    assert max(abs(elem[e] / elem0[e] - 1) for e in range(2)) < 1e-12
    om, _ = oracle.state_chem(mech, rhos, T)
    X = rhos / M
    for r, (reac, prod) in enumerate([([0], [3, 3]), ([1], [4, 4]), ([2], [3, 4]),
                                      ([0, 4], [2, 3]), ([2, 4], [1, 3])]):
        lnQ = sum(math.log(X[s]) for s in prod) - sum(math.log(X[s]) for s in reac)
        assert abs(lnQ - oracle.lnKc(mech, r, T)) < 1e-8


@pytest.mark.parametrize("mech", [inputs.MECH_AIR5, inputs.MECH_AIR11])
def test_fixed_temperature_jacobian_fd(mech):
    rhos = air_state(mech, 9)
    T, Tv = 7000.0, 6000.0
    om, J = oracle.state_chem(mech, rhos, T, Tv)
    ns = len(rhos)
    for r in range(ns):
        h = 1e-5 * max(rhos[r], 1e-2 * rhos.sum())
        p, m = rhos.copy(), rhos.copy()
        p[r] += h
        m[r] -= h
        fd = (oracle.state_chem(mech, p, T, Tv)[0] - oracle.state_chem(mech, m, T, Tv)[0]) / (2 * h)
        assert np.max(np.abs(J[:, r] - fd) / np.max(np.abs(fd))) < 1e-6


@pytest.mark.parametrize("mech", [inputs.MECH_AIR5, inputs.MECH_AIR11])
def test_conserved_source_jacobian_fd(mech):
    """A_S = dS/dQ at fixed other conserved variables (Sec. 2.2), through T(Q), Tv(Q)."""
    nd = 2
    rhos = air_state(mech, 12, rho=0.01)
    q = oracle.state_cons(mech, nd, rhos, [800.0, -300.0], 6500.0, 5500.0)
    om, Jq = oracle.state_source_jac(mech, nd, q)
    ns = len(rhos)
    for k in range(len(q)):
        h = 1e-6 * (abs(q[k]) if abs(q[k]) > 0 else 1e-3 * rhos.sum())
        if k < ns:
            h = 1e-6 * max(rhos[k], 1e-2 * rhos.sum())
        p, m = q.copy(), q.copy()
        p[k] += h
        m[k] -= h
        fd = (oracle.state_source_jac(mech, nd, p)[0] - oracle.state_source_jac(mech, nd, m)[0]) / (2 * h)
        ref = np.max(np.abs(Jq[:, k])) + 1e-300
        assert np.max(np.abs(Jq[:, k] - fd)) / ref < 2e-5, k


def test_landau_teller_sign_and_zero():
    """Vibrational source (2T): the relaxation part drives Tv towards T and vanishes at
    Tv = T; checked at a low temperature where chemistry is frozen."""
    mech = inputs.MECH_AIR11
    rhos = np.zeros(11)
    rhos[0], rhos[1] = 0.767e-2, 0.233e-2
    for Tv, sign in ((900.0, 1), (1200.0, -1)):
        q = oracle.state_cons(mech, 2, rhos, [0.0, 0.0], 1000.0, Tv)
        v = oracle.state_vib(mech, 2, q)
        assert np.sign(v["omega_v"]) == sign
        assert v["relax"] > 0
    q = oracle.state_cons(mech, 2, rhos, [0.0, 0.0], 1000.0, 1000.0)
    v = oracle.state_vib(mech, 2, q)
    ref = oracle.state_vib(mech, 2, oracle.state_cons(mech, 2, rhos, [0.0, 0.0], 1000.0, 900.0))
    assert abs(v["omega_v"]) < 1e-10 * abs(ref["omega_v"])


def test_relaxation_diagonal_is_conserved_variable_derivative():
    """At T = Tv the Landau-Teller source vanishes, and so do the terms from the temperature
    dependence of tau; there the vibrational diagonal relax equals -d omega_v / d(rho e_v) at
    fixed species densities, momentum and total energy (both Tv and T move), which a central
    difference of the source gives independently.  Pure N2 at 3000 K: chemistry is frozen
    to ~1e-17 relative, so the pool-energy term of omega_v does not enter."""
    mech = inputs.MECH_AIR11
    nd = 2
    rhos = np.zeros(11)
    rhos[0] = 0.02
    q = oracle.state_cons(mech, nd, rhos, [300.0, 0.0], 3000.0, 3000.0)
    v = oracle.state_vib(mech, nd, q)
    iev = 11 + nd + 1                        # rho e_v slot of the conserved vector
    h = 1e-6 * q[iev]
    qp, qm = q.copy(), q.copy()
    qp[iev] += h
    qm[iev] -= h
    d = (oracle.state_vib(mech, nd, qp)["omega_v"] - oracle.state_vib(mech, nd, qm)["omega_v"]) / (2 * h)
    # (the Tv part alone is relax / (1 + c_v,ve / c_v,tr), ~26 % smaller for N2 at 3000 K)
    assert abs(-d - v["relax"]) < 1e-6 * v["relax"], (-d, v["relax"])
