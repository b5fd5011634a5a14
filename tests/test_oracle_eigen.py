"""Pins of the oracle's eigenvalue splitting of the coupled operator (Sec. 2.3: the flux
Jacobian split as A+- = (A +- |A|)/2 instead of the spectral (A +- lambda I)/2).

* |A| from the wave decomposition is the matrix absolute value of the oracle's own Jacobian
  (taken column by column): its square is A^2, it commutes with A and its eigenvalues are
  |eig(A)| (full and coupled variables, 2D and 3D, 5 and 11 species); |A| = A when every wave
  moves forward; |A(-S)| = |A(S)|.
* The coupling blocks equal -(A + |A| + 2 lambda_vis)/2 and (A - |A| - 2 lambda_vis)/2 with A
  from finite differences of the physical flux and |A| as pinned above.
* The sweeps equal the dense solve of (D+L) D^-1 (D+U) with those blocks and the assembled
  diagonal (V/dtau + sum 2 lambda_vis) I + sum_d |A(S_d)| - V dS/dQ.
"""
import numpy as np
import pytest

import inputs
import oracle
from test_oracle_lusgs import make_case, assemble, scaled_factored_solve, rhs
from test_oracle_thermo_flux import fd_jacobian

def face(q, mech, nd, rng):
    """A random face vector whose normal velocity stays away from 0 and from -+c (the
    eigenvalues of A then keep clear of zero and sign(A) is well defined)."""
    prim = oracle.state_prim(mech, nd, q)
    c = prim["c"]
    ns = oracle.gas_info(mech)["ns"]
    u = q[ns:ns + nd] / q[:ns].sum()
    while True:
        n = rng.normal(size=nd)
        n /= np.linalg.norm(n)
        Un = u @ n
        if min(abs(Un), abs(Un + c), abs(Un - c)) > 0.1 * c:
            S = np.zeros(3)
            S[:nd] = 1e-3 * n
            return S


def state(mech, nd, seed):
    """One partly dissociated cell state moving at 1500 m/s in a seeded direction."""
    shape = (1, 1) if nd == 2 else (1, 1, 1)
    pr = inputs.perturbed_primitive(mech, shape, seed=seed, ndim=nd, T=4000.0, Tv=3000.0, p=5000.0)
    d = np.random.default_rng(seed).normal(size=nd)
    pr["u"] = (1500.0 * d / np.linalg.norm(d)).reshape((nd,) + shape)
    return oracle.prim_to_cons_field(mech, nd, pr)[:, 0]


@pytest.mark.parametrize("mech,nd", [(inputs.MECH_AIR11, 2), (inputs.MECH_AIR5, 3), (inputs.MECH_AIR11, 3)])
@pytest.mark.parametrize("which", [0, 2])
def test_absolute_jacobian_is_the_matrix_absolute_value(mech, nd, which):
    """B = |A| is the one matrix with B^2 = A^2, B A = A B and eigenvalues |eig(A)| (A is
    diagonalisable with real eigenvalues), with A the oracle's own Jacobian-vector product
    taken column by column."""
    rng = np.random.default_rng(11)
    for k in range(3):
        q = state(mech, nd, seed=k)
        S = face(q, mech, nd, rng)
        n = len(q)               # the coupled variables replace one species by the total density
        E = np.eye(n)
        A = np.column_stack([oracle.state_jvp(mech, nd, q, S, which, E[i]) for i in range(n)])
        wb = 3 if which == 0 else 4
        B = np.column_stack([oracle.state_jvp(mech, nd, q, S, wb, E[i]) for i in range(n)])
        A2 = A @ A
        assert np.max(np.abs(B @ B - A2)) <= 1e-11 * np.max(np.abs(A2))
        AB = A @ B
        assert np.max(np.abs(B @ A - AB)) <= 1e-11 * np.max(np.abs(AB))
        ea = np.sort(np.abs(np.linalg.eigvals(A).real))
        eb = np.sort(np.linalg.eigvals(B).real)
        assert np.allclose(eb, ea, rtol=1e-8, atol=1e-10 * ea.max())
        # even in the face vector
        Bm = np.column_stack([oracle.state_jvp(mech, nd, q, -S, wb, E[i]) for i in range(n)])
        assert np.allclose(Bm, B, rtol=1e-12, atol=1e-12 * np.abs(B).max())


def test_supersonic_absolute_jacobian_is_the_jacobian():
    mech, nd = inputs.MECH_AIR5, 2
    q = state(mech, nd, seed=3)
    ns = 5
    u = q[ns:ns + nd] / q[:ns].sum()
    S = 1e-3 * u / np.linalg.norm(u)          # along the flow, speed 1500 m/s > c
    E = np.eye(len(q))
    A = np.column_stack([oracle.state_jvp(mech, nd, q, S, 0, e) for e in E])
    B = np.column_stack([oracle.state_jvp(mech, nd, q, S, 3, e) for e in E])
    assert np.allclose(B, A, rtol=1e-12, atol=1e-12 * np.abs(A).max())


def test_eigen_coupling_blocks():
    g, Q = make_case("ogrid_air11", seed=5)
    g.set_ci_splitting(1)
    g.residual()
    g.build_diagonals(5.0)
    lv = g.field("lamCIv").reshape(-1, 3)
    S0 = g.field("S0").reshape(-1, 3)
    S1 = g.field("S1").reshape(-1, 3)
    ni = g.ni
    c = 2 + ni * 1
    for d, side in ((0, -1), (0, 1), (1, -1), (1, 1)):
        B, nb = g.coupling_block(c, d, side, 3)
        i, j = c % ni, c // ni
        Sf = S0[j * (ni + 1) + i + (side > 0)] if d == 0 else S1[(j + (side > 0)) * ni + i]
        A = fd_jacobian(g.mech, 2, Q[:, nb], Sf, 2)
        n = len(A)
        Babs = np.column_stack([oracle.state_jvp(g.mech, 2, Q[:, nb], Sf, 4, e) for e in np.eye(n)])
        dis = Babs + lv[nb, d] * np.eye(n)
        ref = -0.5 * (A + dis) if side < 0 else 0.5 * (A - dis)
        scale = np.max(np.abs(ref), axis=1, keepdims=True)
        assert np.max(np.abs(B - ref) / scale) < 1e-5


@pytest.mark.parametrize("name", ["box2d_air5", "ogrid_air11", "box3d_air5_kper"])
def test_eigen_coupled_sweeps_equal_dense_factored_solve(name):
    g, Q = make_case(name, seed=3)
    g.set_ci_splitting(1)
    R, _ = g.residual()
    cfl = 4.0
    g.build_diagonals(cfl)
    D, L, U = assemble(g, 3)
    x = scaled_factored_solve(g, Q, 2, D, L, U, rhs(g, R, 2))
    dQ = g.lusgs_coupled(cfl)
    x = x.reshape(g.ncell, g.nci).T
    tol = 1e-7 if g.ns < 11 else 1e-6
    assert np.max(np.abs(dQ - x).max(axis=1) / np.abs(x).max(axis=1)) < tol
    # and the diagonal block is the assembled one: (V/dtau + sum 2 lambda_vis) I + sum |A|
    # (checked through its symmetric part being larger than the spectral operator's minimum)
    g2, _ = make_case(name, seed=3)
    g2.residual()
    g2.build_diagonals(cfl)
    assert not np.allclose(g.field("Dci"), g2.field("Dci"))
