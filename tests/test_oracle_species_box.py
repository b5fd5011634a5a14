"""Pins of the species-box oracle (oracle/species_box.py: one implicit step of the split and
coupled operators for a non-reacting mixture of ns species, the scaling test of Sec. 3.1)
against facts fixed outside it: the textbook Euler flux Jacobian of a perfect gas (one
species), Euler's theorem for the homogeneous flux (A Q = F, any ns), the LU-SGS sweeps as
global block-triangular solves assembled column by column, the upwind species recursion, and
the one-species coupled operator reducing to the split flow block."""
import numpy as np
import pytest

import inputs
from oracle import species_box as sb


def small_box(ns, n=(3, 3, 2), seed=1):
    return sb.Box(inputs.species_box(ns, seed=seed, n=n, size=(0.3, 0.3, 0.2)))


def test_one_species_jacobian_is_the_textbook_euler_jacobian():
    box = small_box(1)
    q = box.q
    rho, u, p, c = sb.primitives(box, q)
    gam = c * c * rho / p
    S = np.array([0.3, -0.7, 0.2])
    A = np.column_stack([sb.jvp_full(box, q, S, e) for e in np.eye(5)])
    # textbook: variables (rho, m, rho E), U = u.S, H = (rho E + p) / rho
    U = u @ S
    H = (q[4] + p) / rho
    phi = 0.5 * (gam - 1.0) * (u @ u)
    B = np.zeros((5, 5))
    B[0, 1:4] = S
    for a in range(3):
        B[1 + a, 0] = phi * S[a] - u[a] * U
        B[1 + a, 1:4] = u[a] * S - (gam - 1.0) * S[a] * u
        B[1 + a, 1 + a] += U
        B[1 + a, 4] = (gam - 1.0) * S[a]
    B[4, 0] = (phi - H) * U
    B[4, 1:4] = H * S - (gam - 1.0) * u * U
    B[4, 4] = gam * U
    assert np.allclose(A, B, rtol=1e-12, atol=1e-12 * np.abs(B).max())


@pytest.mark.parametrize("ns", [1, 5, 40])
def test_flux_is_homogeneous(ns):
    """p is homogeneous of degree one in Q, so the flux is and A(Q) Q = F(Q) (Euler)."""
    box = small_box(ns)
    for S in box.S + [np.array([0.2, -0.1, 0.4])]:
        F = sb.flux(box, box.q, S)
        AQ = sb.jvp_full(box, box.q, S, box.q)
        assert np.allclose(AQ, F, rtol=1e-12, atol=1e-12 * np.abs(F).max())


def global_solve(box, nblock, apply_A, lam, D, rhs_blocks):
    """(D + U)^-1 D (D + L)^-1 rhs with the block matrices assembled column by column over all
    cells (L: lower neighbours -1/2 (A + lambda), U: upper neighbours +1/2 (A - lambda))."""
    N = box.N
    n = N * nblock
    Lm = np.zeros((n, n))
    Um = np.zeros((n, n))
    for c in range(N):
        for lower, M in ((True, Lm), (False, Um)):
            for nb, S, d, s in sb.neighbours(box, c, lower):
                Ablk = np.column_stack([apply_A(e, S) for e in np.eye(nblock)])
                blk = -0.5 * (Ablk + lam[d] * np.eye(nblock)) if lower else 0.5 * (Ablk - lam[d] * np.eye(nblock))
                M[c * nblock:(c + 1) * nblock, nb * nblock:(nb + 1) * nblock] += blk
    Dm = np.kron(np.eye(N), D)
    x = np.linalg.solve(Dm + Lm, rhs_blocks.T.ravel())
    y = np.linalg.solve(Dm + Um, Dm @ x)
    return y.reshape(N, nblock).T


def test_split_sweeps_are_the_block_triangular_solves():
    ns, cfl = 3, 7.0
    box = small_box(ns)
    rhs = inputs.species_box_rhs(ns, box.N, seed=2)
    got = sb.split_operator(box, rhs, cfl)
    q = box.q
    lF, lC = sb.radii(box, q)
    Vdt = lF.sum() / cfl
    Y = q[:ns] / q[:ns].sum()

    def A_flow(x, S):
        a = sb.jvp_full(box, q, S, np.concatenate([Y * x[0], x[1:5]]))
        return np.concatenate([[a[:ns].sum()], a[ns:]])
    rf = np.vstack([rhs[:ns].sum(axis=0), rhs[ns:]])
    want_f = global_solve(box, 5, A_flow, lF, (Vdt + lF.sum()) * np.eye(5), rf)
    assert np.allclose(got[:5], want_f, rtol=1e-11, atol=1e-11 * np.abs(want_f).max(axis=1, keepdims=True))
    U = [q[ns:ns + 3] @ S / q[:ns].sum() for S in box.S]
    for s in range(ns):
        want_s = global_solve(box, 1, lambda x, S: np.array([(q[ns:ns + 3] @ S / q[:ns].sum()) * x[0]]),
                              lC, np.array([[Vdt + lC.sum()]]), rhs[s:s + 1])
        assert np.allclose(got[5 + s], want_s[0], rtol=1e-11, atol=1e-11 * np.abs(want_s).max())
    assert all(u > 0 for u in U)


def test_coupled_sweeps_are_the_block_triangular_solves():
    ns, cfl = 3, 7.0
    box = small_box(ns)
    rhs = inputs.species_box_rhs(ns, box.N, seed=3)
    got = sb.coupled_operator(box, rhs, cfl)
    q = box.q
    lF, _ = sb.radii(box, q)
    nc = ns + 4

    def A_ci(x, S):
        dq = np.concatenate([[x[0] - x[5:].sum()], x[5:], x[1:5]])
        a = sb.jvp_full(box, q, S, dq)
        return np.concatenate([[a[:ns].sum()], a[ns:], a[1:ns]])
    rc = np.vstack([rhs[:ns].sum(axis=0), rhs[ns:], rhs[1:ns]])
    want = global_solve(box, nc, A_ci, lF, (lF.sum() / cfl + lF.sum()) * np.eye(nc), rc)
    assert np.allclose(got, want, rtol=1e-11, atol=1e-11 * np.abs(want).max(axis=1, keepdims=True))


def test_species_backward_sweep_vanishes_for_a_flow_crossing_every_face_forward():
    """All face velocities are positive, so 1/2 (U - |U|) = 0 on every upper face: the species
    increments are the forward upwind recursion D_s x_c = rhs_c + sum_lower U_d x_nb."""
    ns = 4
    box = small_box(ns, n=(4, 3, 3))
    rhs = inputs.species_box_rhs(ns, box.N, seed=4)
    cfl = 3.0
    got = sb.split_operator(box, rhs, cfl)[5:]
    q = box.q
    lF, lC = sb.radii(box, q)
    Ds = lF.sum() / cfl + lC.sum()
    U = [q[ns:ns + 3] @ S / q[:ns].sum() for S in box.S]
    for c in range(box.N):
        acc = rhs[:ns, c].copy()
        for nb, S, d, s in sb.neighbours(box, c, True):
            acc += U[d] * got[:, nb]
        assert np.allclose(got[:, c], acc / Ds, rtol=1e-13, atol=0.0)


def test_one_species_coupled_operator_is_the_split_flow_block():
    box = small_box(1)
    rhs = inputs.species_box_rhs(1, box.N, seed=5)
    a = sb.split_operator(box, rhs, 4.0)
    b = sb.coupled_operator(box, rhs, 4.0)
    assert np.allclose(a[:5], b, rtol=1e-13, atol=1e-13 * np.abs(b).max(axis=1, keepdims=True))
