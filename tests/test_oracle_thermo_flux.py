"""Pins of the oracle's thermodynamics and inviscid fluxes against closed forms, finite
differences of the oracle's own physical flux, and a textbook Roe solver (perfect gas).

Paper passages: Sec. 2.1 (e_t, e_v, ideal-gas law), Sec. 2.3 Eq. (convectiveJacobian) and the
eigenvalues / spectral radius stated after it, Sec. 3.2 (Roe scheme)."""
import math

import numpy as np
import pytest

import inputs
import oracle

MECHS = [inputs.MECH_AIR5, inputs.MECH_AIR11]


def random_state(mech, nd, seed, T=4000.0, Tv=None, p=2e4, speed=2000.0):
    rng = np.random.default_rng(seed)
    ns = oracle.gas_info(mech)["ns"]
    Y = rng.uniform(0.05, 1.0, ns)
    if mech == inputs.MECH_AIR11:
        Y[10] = 1e-4  # electrons
    Y /= Y.sum()
    rho = p / (287.0 * T)
    u = rng.uniform(-1, 1, nd) * speed
    return oracle.state_cons(mech, nd, rho * Y, u, T, T if Tv is None else Tv)


@pytest.mark.parametrize("mech", MECHS)
@pytest.mark.parametrize("T,Tv", [(300.0, 300.0), (3000.0, 8000.0), (12000.0, 5000.0)])
def test_temperature_round_trip(mech, T, Tv):
    ns = oracle.gas_info(mech)["ns"]
    rng = np.random.default_rng(1)
    Y = rng.uniform(0.1, 1, ns)
    Y /= Y.sum()
    ntemp = oracle.gas_info(mech)["ntemp"]
    Tv_ = Tv if ntemp == 2 else T
    q = oracle.state_cons(mech, 2, 0.01 * Y, [300.0, -50.0], T, Tv_)
    w = oracle.state_prim(mech, 2, q)
    assert abs(w["T"] / T - 1) < 1e-11
    assert abs(w["Tv"] / Tv_ - 1) < 1e-11


def test_perfect_gas_limit():
    # single diatomic species with frozen vibration: gamma = 7/5 exactly
    q = oracle.state_cons(inputs.MECH_PERFECT, 2, [1.2], [100.0, 30.0], 300.0)
    w = oracle.state_prim(inputs.MECH_PERFECT, 2, q)
    assert abs(w["c"] ** 2 * w["rho"] / w["p"] - 1.4) < 1e-14
    assert abs(w["beta"] - 0.4) < 1e-14


def test_cold_air_gamma():
    # 300 K air: vibration barely excited, gamma within 0.5% of 1.4
    for mech in MECHS:
        ns = oracle.gas_info(mech)["ns"]
        rhos = np.zeros(ns)
        rhos[0], rhos[1] = 0.767, 0.233
        q = oracle.state_cons(mech, 2, rhos, [0.0, 0.0], 300.0, 300.0)
        w = oracle.state_prim(mech, 2, q)
        g = w["c"] ** 2 * w["rho"] / w["p"]
        assert abs(g - 1.4) < 0.007, g


def test_vibrational_energy_limits():
    # harmonic oscillator: e_v -> R T (1 - theta/(2T)) at high T, -> 0 at low T
    mech = inputs.MECH_AIR5
    M = oracle.gas_info(mech)["M"]
    R_N2 = 8314.462618 / M[0]
    for T in (5e4, 9e4):
        e = oracle.species_energy(mech, T)[0]   # N2: 2.5 R T + e_v
        ev = e - 2.5 * R_N2 * T
        assert abs(ev / (R_N2 * T) - (1 - 3395.0 / (2 * T))) < 2e-3
    e = oracle.species_energy(mech, 100.0)[0]
    assert abs(e / (2.5 * R_N2 * 100.0) - 1.0) < 1e-12


@pytest.mark.parametrize("mech", MECHS)
def test_pressure_derivatives_fd(mech):
    nd = 2
    q = random_state(mech, nd, 7, T=5000.0, Tv=7000.0)
    w = oracle.state_prim(mech, nd, q)
    ns = oracle.gas_info(mech)["ns"]
    nq = len(q)
    grad = np.zeros(nq)
    for k in range(nq):
        h = 1e-6 * max(abs(q[k]), 1e-3 * np.max(np.abs(q[:ns])))
        qp, qm = q.copy(), q.copy()
        qp[k] += h
        qm[k] -= h
        grad[k] = (oracle.state_prim(mech, nd, qp)["p"] - oracle.state_prim(mech, nd, qm)["p"]) / (2 * h)
    an = np.zeros(nq)
    an[:ns] = w["prs"]
    u = q[ns:ns + nd] / w["rho"]
    an[ns:ns + nd] = -w["beta"] * u
    an[ns + nd] = w["beta"]
    if nq > ns + nd + 1:
        an[ns + nd + 1] = w["prev"]
    scale = np.abs(an * np.where(np.abs(q) > 0, q, 1)).max()
    assert np.max(np.abs((grad - an) * np.where(np.abs(q) > 0, q, 1))) / scale < 1e-6
    # Euler homogeneity: sum_k Q_k dp/dQ_k = p
    assert abs(np.dot(an, q) / w["p"] - 1.0) < 1e-12


def fd_jacobian(mech, nd, q, S, which):
    """Finite-difference Jacobian of the physical flux F(Q).S in the chosen variables."""
    ns = oracle.gas_info(mech)["ns"]
    nq = len(q)
    rho = q[:ns].sum()
    Y = q[:ns] / rho
    nF = nq - ns + 1

    def to_full(x):
        if which == 0:
            return x
        full = np.zeros(nq)
        if which == 1:      # flow block (rho, m, E, [ev]) with frozen mass fractions
            full[:ns] = Y * x[0]
            full[ns:] = x[1:nF]
        else:               # coupled variables (rho, m, E, [ev], rho_2..rho_ns)
            full[1:ns] = x[nF:]
            full[0] = x[0] - x[nF:].sum()
            full[ns:] = x[1:nF]
        return full

    def from_full(F):
        if which == 0:
            return F
        out = np.concatenate([[F[:ns].sum()], F[ns:]])
        if which == 2:
            out = np.concatenate([out, F[1:ns]])
        return out

    n = nq if which == 0 else (nF if which == 1 else nq)
    cols = []
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        dq = to_full(e)
        # step: a relative perturbation of 1e-6 of every component it touches
        floor = np.where(np.arange(nq) < ns, 1e-2 * rho, np.abs(q) + 1e-3 * np.max(np.abs(q)))
        mag = np.maximum(np.abs(q), floor)
        touched = np.abs(dq) > 0
        h = 1e-6 * np.min(mag[touched] / np.abs(dq[touched]))
        Fp = oracle.state_flux(mech, nd, q + h * dq, S)
        Fm = oracle.state_flux(mech, nd, q - h * dq, S)
        cols.append(from_full((Fp - Fm) / (2 * h)))
    return np.array(cols).T


@pytest.mark.parametrize("mech", MECHS)
@pytest.mark.parametrize("which", [0, 1, 2])
def test_flux_jacobian_vector_product(mech, which):
    """Matrix-free Jacobian of Eq. (convectiveJacobian) vs central differences."""
    nd = 2
    q = random_state(mech, nd, 11, T=6000.0, Tv=4000.0)
    S = np.array([0.3, -0.7, 0.0])
    A = fd_jacobian(mech, nd, q, S, which)
    n = A.shape[1]
    # column by column, each row scaled by its own magnitude: a dropped term, a wrong sign
    # or a transposed index in any entry shows up as an O(1) error
    An = np.array([oracle.state_jvp(mech, nd, q, S, which, e) for e in np.eye(n)]).T
    rowscale = np.maximum(np.max(np.abs(A), axis=1, keepdims=True), 1e-300)
    assert np.max(np.abs(An - A) / rowscale) < 1e-5


@pytest.mark.parametrize("mech", MECHS + [inputs.MECH_PERFECT])
def test_spectral_radius_is_max_eigenvalue(mech):
    """Eigenvalues of the Euler Jacobian are U +- c|S| and U: the spectral radius
    |U| + c|S| (Sec. 2.3) follows from the frozen sound speed the oracle uses."""
    nd = 2
    q = random_state(mech, nd, 3, T=7000.0, Tv=6000.0) if mech else \
        oracle.state_cons(mech, 2, [0.3], [250.0, -80.0], 500.0)
    S = np.array([0.6, 0.8, 0.0])
    A = fd_jacobian(mech, nd, q, S, 0)
    ev = np.sort(np.linalg.eigvals(A).real)
    w = oracle.state_prim(mech, nd, q)
    ns = oracle.gas_info(mech)["ns"]
    U = (q[ns:ns + 2] / w["rho"]) @ S[:2]
    assert abs(ev[-1] - (U + w["c"])) / w["c"] < 1e-5
    assert abs(ev[0] - (U - w["c"])) / w["c"] < 1e-5
    assert np.all(np.abs(ev[1:-1] - U) < 1e-5 * w["c"])


def textbook_roe_2d(qL, qR, S, gamma, efix):
    """Roe's flux for a perfect gas in 2D written out wave by wave (Toro, ch. 11)."""
    def prim(q):
        rho = q[0]
        u = q[1:3] / rho
        p = (gamma - 1) * (q[3] - 0.5 * rho * u @ u)
        return rho, u, p, (q[3] + p) / rho

    area = np.linalg.norm(S[:2])
    n = S[:2] / area
    t = np.array([-n[1], n[0]])
    rL, uL, pL, HL = prim(qL)
    rR, uR, pR, HR = prim(qR)
    sL, sR = math.sqrt(rL), math.sqrt(rR)
    u = (sL * uL + sR * uR) / (sL + sR)
    H = (sL * HL + sR * HR) / (sL + sR)
    c = math.sqrt((gamma - 1) * (H - 0.5 * u @ u))
    rt = sL * sR
    un, ut = u @ n, u @ t
    dp, drho = pR - pL, rR - rL
    dun, dut = (uR - uL) @ n, (uR - uL) @ t
    a1 = (dp - rt * c * dun) / (2 * c * c)
    a2 = drho - dp / (c * c)
    a3 = rt * dut
    a4 = (dp + rt * c * dun) / (2 * c * c)
    r1 = np.array([1, *(u - c * n), H - un * c])
    r2 = np.array([1, *u, 0.5 * u @ u])
    r3 = np.array([0, *t, ut])
    r4 = np.array([1, *(u + c * n), H + un * c])
    delta = efix * (abs(un) + c)

    def fix(l):
        return (l * l + delta * delta) / (2 * delta) if abs(l) < delta else abs(l)

    def flux(r, uu, p, H_):
        U = uu @ S[:2]
        return np.array([r * U, r * uu[0] * U + p * S[0], r * uu[1] * U + p * S[1], r * H_ * U])

    D = fix(un - c) * a1 * r1 + fix(un) * (a2 * r2 + a3 * r3) + fix(un + c) * a4 * r4
    return 0.5 * (flux(rL, uL, pL, HL) + flux(rR, uR, pR, HR)) - 0.5 * area * D


def test_roe_matches_textbook_perfect_gas():
    mech = inputs.MECH_PERFECT
    rng = np.random.default_rng(2)
    for trial in range(20):
        qL = oracle.state_cons(mech, 2, [rng.uniform(0.1, 2)], rng.normal(size=2) * 300,
                               rng.uniform(200, 2000))
        qR = oracle.state_cons(mech, 2, [rng.uniform(0.1, 2)], rng.normal(size=2) * 300,
                               rng.uniform(200, 2000))
        S = np.array([*rng.normal(size=2), 0.0])
        F = oracle.state_roe(mech, 2, qL, qR, S, efix=0.1)
        Ft = textbook_roe_2d(qL, qR, S, 1.4, 0.1)
        assert np.max(np.abs(F - Ft)) / np.max(np.abs(Ft)) < 1e-10


@pytest.mark.parametrize("mech", MECHS)
def test_roe_consistency_and_conservation(mech):
    nd = 2
    qL = random_state(mech, nd, 21, T=3000.0, Tv=2500.0)
    qR = random_state(mech, nd, 22, T=5000.0, Tv=6000.0)
    S = np.array([0.4, 0.2, 0.0])
    # consistency: F(Q, Q) = F(Q)
    F = oracle.state_roe(mech, nd, qL, qL, S)
    Fp = oracle.state_flux(mech, nd, qL, S)
    assert np.max(np.abs(F - Fp)) / np.max(np.abs(Fp)) < 1e-14
    # conservation / orientation: F(L, R, S) = -F(R, L, -S)
    F1 = oracle.state_roe(mech, nd, qL, qR, S)
    F2 = oracle.state_roe(mech, nd, qR, qL, -S)
    assert np.max(np.abs(F1 + F2)) / np.max(np.abs(F1)) < 1e-13


def test_roe_supersonic_upwinding():
    """With both states supersonic along S (and the entropy fix inactive) the flux is F(L)."""
    mech = inputs.MECH_AIR5
    nd = 2
    rhos = np.array([0.767, 0.233, 0, 0, 0]) * 0.01
    qL = oracle.state_cons(mech, nd, rhos, [3000.0, 100.0], 400.0)
    qR = oracle.state_cons(mech, nd, rhos * 1.1, [2900.0, 50.0], 420.0)
    S = np.array([1.0, 0.0, 0.0])
    F = oracle.state_roe(mech, nd, qL, qR, S, efix=0.05)
    FL = oracle.state_flux(mech, nd, qL, S)
    assert np.max(np.abs(F - FL)) / np.max(np.abs(FL)) < 1e-13
