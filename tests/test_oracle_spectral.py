"""Pins of the oracle's spectral radii, local time step, diagonals and wall heat flux (Sec. 2.2
Eq. (vislambda) and the local time step; Sec. 2.3.1-2.3.2 radii; Sec. 3.2 heat-flux monitor)
against what the mathematics fixes, not against the oracle's own formulas:

* the inviscid radius of every cell and direction equals the spectral radius of the
  finite-difference Jacobian of the physical flux through the cell's mean face vector, and it
  makes the spectral splitting's two halves semi-definite at every face (the property the
  splitting needs);
* the viscous radius is the weight of the discrete viscous and diffusive stencil: on a uniform
  state at rest, the finite-difference Jacobian of the oracle's own residual (viscous minus
  inviscid run) couples a cell to its neighbour with spectral radius lambda_vis and to itself
  with 2 lambda_vis per direction, for the flow block (frozen composition) and the species;
* on a uniform Cartesian box in uniform inviscid flow of a perfect gas the diagonals are the
  closed forms D_F = (1 + 1/CFL) sum_d (|u_d| + c) h and
  D_s = sum_d (|u_d| + c) h / CFL + sum_d |u_d| h, with c^2 = 1.4 R T;
* the species diagonal adds V max(0, -d omega_s / d rho_s) with the derivative taken by finite
  differences of the source at fixed other conserved variables;
* the stagnation heat flux is the conduction through the wall face that the residual itself
  carries, k (T_1 - T_w) / d_1 (+ k_v (T_v1 - T_w) / d_1) with d_1 half the cell height."""
import numpy as np
import pytest

import inputs
import oracle
from test_oracle_thermo_flux import fd_jacobian

RU = 8314.462618


def _sbar(g, c):
    """Mean face vector of cell c per direction ([nd][3])."""
    ni, nj = g.ni, g.nj
    i, j = c % ni, c // ni
    S0 = g.field("S0").reshape(-1, 3)
    S1 = g.field("S1").reshape(-1, 3)
    si = 0.5 * (S0[i + (ni + 1) * j] + S0[i + 1 + (ni + 1) * j])
    sj = 0.5 * (S1[i + ni * j] + S1[i + ni * (j + 1)])
    return [si, sj]


def _state(mech, nd, shape, seed, **kw):
    pr = inputs.perturbed_primitive(mech, shape, seed=seed, ndim=nd, **kw)
    return oracle.prim_to_cons_field(mech, nd, pr)


@pytest.mark.parametrize("mech,kw", [(inputs.MECH_AIR5, dict(T=3000.0, p=3000.0)),
                                     (inputs.MECH_AIR11, dict(T=6000.0, Tv=4500.0, p=8000.0))])
def test_inviscid_radius_is_the_flux_jacobian_spectral_radius(mech, kw):
    nodes = inputs.cylinder_ogrid(8, 6)
    g = oracle.OracleGrid(nodes, inputs.cylinder_bc(), mech, limiter=0)
    g.set_boundary(inputs.freestream(mech, mach=8.0), Tw=500.0)
    g.set_viscous(False)
    g.set_reacting(False)
    Q = _state(mech, 2, (g.nj, g.ni), seed=3, **kw)
    g.set_state(Q)
    g.residual()
    g.build_diagonals(5.0)
    lamF = g.field("lamF").reshape(-1, 3)
    for c in range(g.ncell):
        for d, S in enumerate(_sbar(g, c)):
            A = fd_jacobian(mech, 2, Q[:, c], S, 0)
            rho_A = np.max(np.abs(np.linalg.eigvals(A)))
            assert abs(lamF[c, d] - rho_A) <= 1e-6 * rho_A, (c, d, lamF[c, d], rho_A)


def test_spectral_splitting_halves_are_semidefinite():
    """With the viscous radius on, (A(S_f) + lambda I)/2 >= 0 and (A(S_f) - lambda I)/2 <= 0 in
    their eigenvalues at every interior face, lambda the radius of either cell.  Exact where
    the face vector equals the cell's mean face vector (here: a uniform Cartesian box with a
    non-uniform state); on a stretched curvilinear grid |S_f| differs from the mean and the
    halves are definite only up to that ratio (the radius is defined with the cell's metrics,
    as in the paper)."""
    mech = inputs.MECH_AIR5
    nodes = inputs.box_grid(6, 5, lx=0.06, ly=0.05)
    bc = [inputs.BC_PERIODIC] * 4 + [inputs.BC_FARFIELD] * 2
    g = oracle.OracleGrid(nodes, bc, mech, limiter=0)
    g.set_boundary(inputs.freestream(mech, mach=8.0), Tw=500.0)
    Q = _state(mech, 2, (g.nj, g.ni), seed=4, T=3000.0, p=3000.0)
    g.set_state(Q)
    g.residual()
    g.build_diagonals(5.0)
    lamF = g.field("lamF").reshape(-1, 3)
    S0 = g.field("S0").reshape(-1, 3)
    S1 = g.field("S1").reshape(-1, 3)
    ni, nj = g.ni, g.nj
    for j in range(nj):
        for i in range(ni):
            c = i + ni * j
            for d, nb, S in ((0, (i + 1) % ni + ni * j, S0[i + 1 + (ni + 1) * j]),
                             (1, i + ni * ((j + 1) % nj), S1[i + ni * (j + 1)])):
                for cell in (c, nb):
                    A = fd_jacobian(mech, 2, Q[:, cell], S, 0)
                    lam = lamF[cell, d]
                    scale = np.abs(np.linalg.eigvals(A)).max()
                    ep = np.linalg.eigvals(0.5 * (A + lam * np.eye(len(A)))).real
                    em = np.linalg.eigvals(0.5 * (A - lam * np.eye(len(A)))).real
                    assert ep.min() >= -1e-7 * scale and em.max() <= 1e-7 * scale, (c, d)


def _rest_box(mech, T, Tv, p, Y, h=2.5e-5, n=4):
    """Uniform state at rest on an n x n box of spacing h, periodic in both directions."""
    nodes = inputs.box_grid(n, n, lx=n * h, ly=n * h)
    bc = [inputs.BC_PERIODIC] * 4 + [inputs.BC_FARFIELD] * 2
    g = oracle.OracleGrid(nodes, bc, mech, limiter=0)
    g.set_boundary(inputs.freestream(mech, T=T, p=p, mach=2.0), Tw=T)
    g.set_reacting(False)
    ns = g.ns
    M = oracle.gas_info(mech)["M"]
    R = RU * np.sum(Y / M)                   # p = rho R T (heavy particles; no electrons here)
    rho = p / (R * T)
    q = oracle.state_cons(mech, 2, rho * np.asarray(Y), np.zeros(2), T, Tv)
    Q = np.repeat(q[:, None], g.ncell, axis=1)
    return g, Q


def _fd_residual_jacobian(g, Q, c, col_cell, scales, rel_step=1e-6):
    """d R_c / d Q_col_cell by central differences of the oracle's residual (forward
    differences for a species that is absent, whose density cannot go below zero)."""
    nq = g.nq
    J = np.zeros((nq, nq))
    g.set_state(Q)
    R0, _ = g.residual()
    for v in range(nq):
        dq = rel_step * scales[v]
        Qp, Qm = Q.copy(), Q.copy()
        Qp[v, col_cell] += dq
        g.set_state(Qp)
        Rp, _ = g.residual()
        if v < g.ns and Q[v, col_cell] < dq:
            J[:, v] = (Rp[:, c] - R0[:, c]) / dq
            continue
        Qm[v, col_cell] -= dq
        g.set_state(Qm)
        Rm, _ = g.residual()
        J[:, v] = (Rp[:, c] - Rm[:, c]) / (2 * dq)
    return J


def _flow_block(J, Y, ns):
    """Flow rows/columns (rho, m, rho E, [rho e_v]) at frozen mass fractions."""
    nq = J.shape[0]
    nF = nq - ns + 1
    T = np.zeros((nq, nF))              # flow increments -> full conserved increments
    T[:ns, 0] = Y
    T[ns:, 1:] = np.eye(nq - ns)
    P = np.zeros((nF, nq))              # full residual rows -> flow rows
    P[0, :ns] = 1.0
    P[1:, ns:] = np.eye(nq - ns)
    return P @ J @ T


@pytest.mark.parametrize("mech,T,Tv,Y", [
    (inputs.MECH_AIR5, 2000.0, 2000.0, [0.6, 0.15, 0.05, 0.1, 0.1]),
    (inputs.MECH_AIR11, 3000.0, 2200.0, [0.55, 0.12, 0.06, 0.12, 0.15, 0, 0, 0, 0, 0, 0]),
])
def test_viscous_radius_is_the_discrete_viscous_stencil_weight(mech, T, Tv, Y):
    Y = np.asarray(Y) / np.sum(Y)
    g, Q = _rest_box(mech, T, Tv, 200.0, Y)
    ns, nq = g.ns, g.nq
    rho = Q[:ns, 0].sum()
    c_snd = oracle.state_prim(mech, 2, Q[:, 0])["c"]
    scales = np.concatenate([np.full(ns, rho), np.full(2, rho * c_snd), np.abs(Q[ns:, 0]).max() * np.ones(nq - ns - 2)])
    c, nb = 5, 6                                  # cell (1, 1) and its +i neighbour
    jac = {}
    lam = {}
    for visc in (True, False):
        g.set_viscous(visc)
        jac[visc] = (_fd_residual_jacobian(g, Q, c, nb, scales), _fd_residual_jacobian(g, Q, c, c, scales))
        g.set_state(Q)
        g.residual()
        g.build_diagonals(5.0)
        lam[visc] = (g.field("lamF").reshape(-1, 3)[c], g.field("lamC").reshape(-1, 3)[c])
    Jnb = jac[True][0] - jac[False][0]
    Jself = jac[True][1] - jac[False][1]
    lvF = 0.5 * (lam[True][0] - lam[False][0])     # lambda-hat = lambda_inv + 2 lambda_vis
    lvC = 0.5 * (lam[True][1] - lam[False][1])
    assert lvF[0] > 0 and lvC[0] > 0

    def radius(M):
        return np.max(np.abs(np.linalg.eigvals(M)))
    # neighbour coupling: -lambda_vis (flow block at frozen composition; species)
    assert abs(radius(_flow_block(Jnb, Y, ns)) - lvF[0]) <= 1e-5 * lvF[0]
    assert abs(radius(Jnb[:ns, :ns]) - lvC[0]) <= 1e-5 * lvC[0]
    # self coupling: 2 lambda_vis per direction, both directions (square box: equal radii)
    assert abs(radius(_flow_block(Jself, Y, ns)) - 2.0 * (lvF[0] + lvF[1])) <= 1e-5 * lvF[0]
    assert abs(radius(Jself[:ns, :ns]) - 2.0 * (lvC[0] + lvC[1])) <= 1e-5 * lvC[0]


def test_diagonals_closed_form_uniform_inviscid_flow():
    mech = inputs.MECH_PERFECT
    n, h, T, cfl = 5, 0.01, 400.0, 7.0
    nodes = inputs.box_grid(n, n, lx=n * h, ly=n * h)
    bc = [inputs.BC_PERIODIC] * 4 + [inputs.BC_FARFIELD] * 2
    g = oracle.OracleGrid(nodes, bc, mech, limiter=0)
    g.set_boundary(inputs.freestream(mech, T=T, p=1e4, mach=2.0), Tw=T)
    g.set_viscous(False)
    M = oracle.gas_info(mech)["M"][0]
    c = np.sqrt(1.4 * RU / M * T)
    u = np.array([0.8 * c, -0.3 * c])
    rho = 0.05
    q = oracle.state_cons(mech, 2, [rho], u, T, T)
    g.set_state(np.repeat(q[:, None], g.ncell, axis=1))
    g.residual()
    g.build_diagonals(cfl)
    inv = np.sum((np.abs(u) + c) * h)
    DF = g.field("DF")
    Ds = g.field("Ds")
    np.testing.assert_allclose(DF, (1.0 + 1.0 / cfl) * inv, rtol=1e-12)
    np.testing.assert_allclose(Ds, inv / cfl + np.sum(np.abs(u) * h), rtol=1e-12)


def test_species_diagonal_adds_the_stabilising_source_derivative():
    mech = inputs.MECH_AIR5
    n, h = 2, 1e-3
    nodes = inputs.box_grid(n, n, lx=n * h, ly=n * h)
    bc = [inputs.BC_PERIODIC] * 4 + [inputs.BC_FARFIELD] * 2
    g = oracle.OracleGrid(nodes, bc, mech, limiter=0)
    g.set_boundary(inputs.freestream(mech, T=300.0, p=1e4, mach=2.0), Tw=300.0)
    Y = np.array([0.6, 0.15, 0.05, 0.1, 0.1])
    q = oracle.state_cons(mech, 2, 0.02 * Y, np.array([300.0, 100.0]), 6500.0)
    Q = np.repeat(q[:, None], g.ncell, axis=1)
    V = h * h
    Ds = {}
    for react in (True, False):
        g.set_reacting(react)
        g.set_state(Q)
        g.residual()
        g.build_diagonals(3.0)
        Ds[react] = g.field("Ds").reshape(g.ns, -1)[:, 0]
    g.set_reacting(True)
    for s in range(g.ns):
        dq = 1e-6 * q[:g.ns].sum()
        om = []
        for sgn in (1, -1):
            Qp = Q.copy()
            Qp[s] += sgn * dq
            g.set_state(Qp)
            g.residual()
            om.append(g.field("omega").reshape(g.ns, -1)[s, 0])
        dom = (om[0] - om[1]) / (2 * dq)
        expect = V * max(0.0, -dom)
        assert abs((Ds[True][s] - Ds[False][s]) - expect) <= 1e-6 * max(expect, 1e-12 * Ds[False][s]), (s, dom)
    assert np.any(Ds[True] > Ds[False])


@pytest.mark.parametrize("mech,T1,Tv1", [(inputs.MECH_AIR5, 1200.0, 1200.0),
                                          (inputs.MECH_AIR11, 1500.0, 900.0)])
def test_stagnation_heat_flux_is_the_residual_wall_conduction(mech, T1, Tv1):
    """A box at rest, periodic in i, wall below and far field above, uniform T_1 (and T_v1) with
    a wall at T_w: every face but the wall carries no energy flux, so the wall cell's energy
    residual is the conduction through the wall face, q_w |S_w|."""
    ni, nj, h, Tw = 6, 4, 2e-3, 500.0
    nodes = inputs.box_grid(ni, nj, lx=ni * h, ly=nj * h)
    bc = [inputs.BC_PERIODIC, inputs.BC_PERIODIC, inputs.BC_WALL, inputs.BC_FARFIELD,
          inputs.BC_FARFIELD, inputs.BC_FARFIELD]
    g = oracle.OracleGrid(nodes, bc, mech, limiter=0)
    g.set_reacting(False)
    Y = np.zeros(g.ns)
    Y[0], Y[1] = 0.767, 0.233
    fs = inputs.freestream(mech, T=T1, Tv=Tv1, p=2000.0, mach=0.0, direction=(0.0, -1.0, 0.0))
    g.set_boundary(fs, Tw=Tw)
    q = oracle.state_cons(mech, 2, 0.01 * Y, np.zeros(2), T1, Tv1)
    g.set_state(np.repeat(q[:, None], g.ncell, axis=1))
    R, norms = g.residual()
    c = g.stag_cell
    assert 0 <= c < ni                                     # a wall cell
    area = h                                               # unit depth
    ns = g.ns
    kt, kv = g.field("kt")[c], g.field("kv")[c]
    expect = kt * (T1 - Tw) / (0.5 * h)
    if g.ntemp == 2:
        expect += kv * (Tv1 - Tw) / (0.5 * h)
        # the pool-energy residual carries the vibrational part alone
        np.testing.assert_allclose(R[ns + 3, c], kv * (Tv1 - Tw) / (0.5 * h) * area, rtol=1e-12)
    np.testing.assert_allclose(norms[2], expect, rtol=1e-12)
    np.testing.assert_allclose(R[ns + 2, c], norms[2] * area, rtol=1e-12)
    # the cells above the wall row carry no energy residual
    assert np.max(np.abs(R[ns + 2, ni:])) <= 1e-9 * abs(R[ns + 2, c])


@pytest.mark.parametrize("mech,kw", [(inputs.MECH_AIR5, dict(T=9000.0, p=40000.0)),
                                     (inputs.MECH_AIR11, dict(T=9000.0, Tv=6000.0, p=8000.0))])
def test_source_radius_in_the_local_time_step(mech, kw):
    """Sec. 2.2's local time step with the source radius (option dtau_source): V/dtau grows by
    V lambda_S / CFL in every cell, on every diagonal alike, with lambda_S the largest magnitude
    on the diagonal of the conserved-variable source Jacobian -- taken here from the single-state
    Jacobian (itself pinned by central differences in test_oracle_chem) and, 2T, the
    relaxation rate (pinned as -d omega_v / d(rho e_v) there) -- and nothing changes without
    chemistry."""
    nd = 2
    nodes = inputs.cylinder_ogrid(6, 5)
    cfl = 7.0
    out = {}
    for react in (True, False):
        for on in (0, 1):
            g = oracle.OracleGrid(nodes, inputs.cylinder_bc(), mech, limiter=0)
            g.set_boundary(inputs.freestream(mech, mach=8.0), Tw=500.0)
            g.set_reacting(react)
            g.set_dtau_source(on)
            Q = _state(mech, nd, (g.nj, g.ni), seed=11, **kw)
            g.set_state(Q)
            g.residual()
            g.build_diagonals(cfl)
            out[react, on] = (g.field("DF"), g.field("DFev"), g.field("Ds").reshape(-1, g.ncell), g.field("V"), Q)
    for k in range(3):
        assert np.array_equal(out[False, 0][k], out[False, 1][k])
    DF0, DFev0, Ds0, V, Q = out[True, 0]
    DF1, DFev1, Ds1, _, _ = out[True, 1]
    ns = Ds0.shape[0]
    two_t = oracle.gas_info(mech)["ntemp"] == 2
    for c in range(len(V)):
        _, J = oracle.state_source_jac(mech, nd, Q[:, c])
        lam = np.max(np.abs(np.diag(J[:, :ns])))
        if two_t:
            lam = max(lam, oracle.state_vib(mech, nd, Q[:, c])["relax"])
        want = V[c] * lam / cfl
        assert want > 1e-4 * DF0[c]        # the states are chemically active
        for a, b in ((DF1[c], DF0[c]), (DFev1[c], DFev0[c])) + tuple((Ds1[s, c], Ds0[s, c]) for s in range(ns)):
            assert abs((a - b) - want) <= 1e-9 * a, (c, a - b, want)
