"""Pins of the oracle's implicit operator and corrections.

* LU-SGS (Sec. 2.2): the matrix-free forward/backward sweeps equal a dense solve of
  (D+L) D^-1 (D+U) dQ = -R assembled block by block from the point equation
  Eq. (ijkiterate), for the split flow block, the split species (Sec. 2.3.1-2.3.2) and the
  coupled (CI) operator, on small 2D/3D grids with periodic, wall and far-field sides.
* The coupling blocks equal -(A(S_f) + lambda)/2 and (A(S_f) - lambda)/2 with A from
  finite differences of the physical flux (spectral splitting, Sec. 2.2).
* Consistency corrections (Sec. 2.3.3): species-to-total density identities.
"""
import numpy as np
import pytest

import inputs
import oracle
from test_oracle_thermo_flux import fd_jacobian

CASES = {
    "box2d_air5": (lambda: inputs.box_grid(5, 4, seed=4, wiggle=0.3), [inputs.BC_FARFIELD] * 6,
                   inputs.MECH_AIR5),
    "ogrid_air11": (lambda: inputs.cylinder_ogrid(6, 4), inputs.cylinder_bc(), inputs.MECH_AIR11),
    "box3d_air5_kper": (lambda: inputs.box_grid(3, 3, 3, seed=2, wiggle=0.3),
                        [2, 2, 2, 2, inputs.BC_PERIODIC, inputs.BC_PERIODIC], inputs.MECH_AIR5),
}


def make_case(name, seed=1):
    nodes_fn, bc, mech = CASES[name]
    nodes = nodes_fn()
    nd = nodes.shape[0]
    g = oracle.OracleGrid(nodes, bc, mech, limiter=1)
    fs = inputs.freestream(mech, T=300.0, p=500.0, mach=8.0)
    g.set_boundary(fs, Tw=500.0)
    shape = (g.nj, g.ni) if nd == 2 else (g.nk, g.nj, g.ni)
    pr = inputs.perturbed_primitive(mech, shape, seed=seed, ndim=nd, T=3000.0, Tv=2500.0, p=3000.0)
    Q = oracle.prim_to_cons_field(mech, nd, pr)
    g.set_state(Q)
    return g, Q


def assemble(g, scheme):
    """Dense D, L, U (block size nv) from the diagonals and the coupling blocks."""
    N = g.ncell
    nv = g.nF if scheme == 0 else g.ns if scheme == 1 else g.nci
    D = np.zeros((N * nv, N * nv))
    L = np.zeros_like(D)
    U = np.zeros_like(D)
    if scheme == 0:
        DF, DFev = g.field("DF"), g.field("DFev")
        for c in range(N):
            for k in range(nv):
                D[c * nv + k, c * nv + k] = DFev[c] if (g.ntemp == 2 and k == nv - 1) else DF[c]
    elif scheme == 1:
        Ds = g.field("Ds").reshape(g.ns, N)
        for c in range(N):
            for s in range(nv):
                D[c * nv + s, c * nv + s] = Ds[s, c]
    else:
        Dci = g.field("Dci").reshape(N, nv, nv)
        for c in range(N):
            D[c * nv:(c + 1) * nv, c * nv:(c + 1) * nv] = Dci[c]
    for c in range(N):
        for d in range(g.nd):
            for side in (-1, 1):
                B, nb = g.coupling_block(c, d, side, scheme)
                if nb < 0:
                    continue
                target = L if nb < c else U      # lexicographic order (i fastest)
                target[c * nv:(c + 1) * nv, nb * nv:(nb + 1) * nv] += B
    return D, L, U


def scaled_factored_solve(g, Q, scheme, D, L, U, b):
    """Solve (D+L) D^-1 (D+U) x = b densely, with the unknowns scaled by the magnitude of
    the matching conserved variables so that the dense solve is well conditioned."""
    ns, N = g.ns, g.ncell
    rho = np.abs(Q[:ns].sum(axis=0)).max()
    flow = [rho] + [np.abs(Q[k]).max() for k in range(ns, g.nq)]
    if scheme == 0:
        sv = np.array(flow)
    elif scheme == 1:
        sv = np.full(ns, rho)
    else:
        sv = np.array(flow + [rho] * (ns - 1))
    S = np.tile(sv, N)
    Dh = D * S[None, :] / S[:, None]
    Lh = L * S[None, :] / S[:, None]
    Uh = U * S[None, :] / S[:, None]
    y = np.linalg.solve(Dh + Lh, b / S)
    x = np.linalg.solve(Dh + Uh, Dh @ y)
    return x * S


def rhs(g, R, scheme):
    N, ns = g.ncell, g.ns
    if scheme == 1:
        return (-R[:ns]).T.reshape(-1)
    flow = np.concatenate([[R[:ns].sum(axis=0)], R[ns:]])
    if scheme == 2:
        flow = np.concatenate([flow, R[1:ns]])
    return (-flow).T.reshape(-1)


@pytest.mark.parametrize("name", list(CASES))
def test_split_sweeps_equal_dense_factored_solve(name):
    g, Q = make_case(name)
    R, _ = g.residual()
    cfl = 7.0
    g.build_diagonals(cfl)
    out = {}
    for scheme in (0, 1):
        D, L, U = assemble(g, scheme)
        out[scheme] = scaled_factored_solve(g, Q, scheme, D, L, U, rhs(g, R, scheme))
    dQ = g.lusgs_split(cfl)
    N = g.ncell
    # per variable (the dense solve mixes variables of very different magnitude, so its own
    # rounding is ~cond * eps; a wrong index, sign or order gives O(1) differences)
    flow = out[0].reshape(N, g.nF).T
    spec = out[1].reshape(N, g.ns).T
    assert np.max(np.abs(dQ[:g.nF] - flow).max(axis=1) / np.abs(flow).max(axis=1)) < 1e-11
    assert np.max(np.abs(dQ[g.nF:] - spec).max(axis=1) / np.abs(spec).max(axis=1)) < 1e-11
    # and the factored operator is not the unfactored one (the approximation is real)
    D, L, U = assemble(g, 0)
    xe = np.linalg.solve(D + L + U, rhs(g, R, 0))
    assert np.max(np.abs(xe - out[0])) / np.max(np.abs(xe)) > 1e-6
    assert N == g.ncell


@pytest.mark.parametrize("name", list(CASES))
def test_coupled_sweeps_equal_dense_factored_solve(name):
    g, Q = make_case(name, seed=3)
    R, _ = g.residual()
    cfl = 4.0
    g.build_diagonals(cfl)
    D, L, U = assemble(g, 2)
    x = scaled_factored_solve(g, Q, 2, D, L, U, rhs(g, R, 2))
    dQ = g.lusgs_coupled(cfl)
    x = x.reshape(g.ncell, g.nci).T
    # the coupled blocks carry the source Jacobian; for the ionised mixture their
    # equilibrated condition number is ~4e7, so the dense reference keeps ~1e-7
    tol = 1e-7 if g.ns < 11 else 1e-6
    assert np.max(np.abs(dQ - x).max(axis=1) / np.abs(x).max(axis=1)) < tol


@pytest.mark.parametrize("scheme", [0, 2])
def test_coupling_blocks_are_spectral_splitting(scheme):
    """Off-diagonal block of the point equation = -(A_nb(S_f) + lambda_nb I)/2 on the minus
    side and (A_nb(S_f) - lambda_nb I)/2 on the plus side, A from finite differences."""
    g, Q = make_case("ogrid_air11", seed=5)
    g.residual()
    g.build_diagonals(5.0)
    lam = g.field("lamF" if scheme == 0 else "lamCI").reshape(-1, 3)
    S0 = g.field("S0").reshape(-1, 3)
    S1 = g.field("S1").reshape(-1, 3)
    ni = g.ni
    c = 2 + ni * 1            # interior cell (i=2, j=1)
    for d, side in ((0, -1), (0, 1), (1, -1), (1, 1)):
        B, nb = g.coupling_block(c, d, side, scheme)
        i, j = c % ni, c // ni
        if d == 0:
            Sf = S0[j * (ni + 1) + i + (side > 0)]
        else:
            Sf = S1[(j + (side > 0)) * ni + i]
        A = fd_jacobian(g.mech, 2, Q[:, nb], Sf, 1 if scheme == 0 else 2)
        l = lam[nb, d]
        ref = -0.5 * (A + l * np.eye(len(A))) if side < 0 else 0.5 * (A - l * np.eye(len(A)))
        scale = np.max(np.abs(ref), axis=1, keepdims=True)
        assert np.max(np.abs(B - ref) / scale) < 1e-5


def test_corrections_identities():
    g, Q = make_case("box2d_air5", seed=7)
    N, ns, nF = g.ncell, g.ns, g.nF
    rng = np.random.default_rng(3)
    rho = Q[:ns].sum(axis=0)
    dQ = np.zeros((g.nsplit, N))
    dQ[0] = 0.05 * rho * rng.uniform(-1, 1, N)
    dQ[1:nF] = 0.01 * Q[ns:] * rng.uniform(-1, 1, (nF - 1, N))
    dQ[nF:] = 0.03 * Q[:ns] * rng.uniform(-1, 1, (ns, N))   # species increments inconsistent with drho
    # CS-1: sum_s rho_s^{m+1} = rho^m + drho, and only the increment is redistributed
    g.set_state(Q)
    assert g.correct(1, 0, dQ) == 0
    Q1 = g.get_state()
    assert np.max(np.abs(Q1[:ns].sum(axis=0) - (rho + dQ[0])) / rho) < 1e-14
    W = Q[:ns] / rho
    expect = Q[:ns] + dQ[nF:] + W * (dQ[0] - dQ[nF:].sum(axis=0))
    assert np.max(np.abs(Q1[:ns] - expect) / rho) < 1e-15
    assert np.max(np.abs(Q1[ns:] - (Q[ns:] + dQ[1:nF])) / np.abs(Q[ns:]).max(axis=1, keepdims=True)) < 1e-15
    # CS-2: mass fractions sum to one, total density = rho + drho, ratios of rho_s + dQ_s kept
    g.set_state(Q)
    g.correct(2, 0, dQ)
    Q2 = g.get_state()
    tot = Q2[:ns].sum(axis=0)
    assert np.max(np.abs(tot / (rho + dQ[0]) - 1)) < 1e-15
    t = Q[:ns] + dQ[nF:]
    assert np.max(np.abs(Q2[:ns] / tot - t / t.sum(axis=0))) < 1e-15
    # CS-2 after CS-1 changes nothing (CS-1 already gives the right total)
    g.set_state(Q1)
    zero = np.zeros_like(dQ)
    g.correct(2, 0, zero)
    assert np.max(np.abs(g.get_state()[:ns] - Q1[:ns]) / rho) < 1e-15
    # coupled update: rho_ns is the remainder of the total density
    dci = np.zeros((g.nci, N))
    dci[:nF] = dQ[:nF]
    dci[nF:] = dQ[nF + 1:nF + ns]
    g.set_state(Q)
    g.correct(0, 0, dci)
    Qc = g.get_state()
    assert np.max(np.abs(Qc[1:ns] - (Q[1:ns] + dci[nF:])) / rho) < 1e-15
    assert np.max(np.abs(Qc[:ns].sum(axis=0) / (rho + dQ[0]) - 1)) < 1e-15


def test_clip_counts_negative_densities():
    g, Q = make_case("box2d_air5", seed=8)
    N, ns, nF = g.ncell, g.ns, g.nF
    dQ = np.zeros((g.nsplit, N))
    dQ[nF + 2] = -2.0 * Q[2]          # drive species 2 negative everywhere
    g.set_state(Q)
    n = g.correct(1, 1, dQ)
    assert n >= N
    assert np.all(g.get_state()[:ns] >= 0)
