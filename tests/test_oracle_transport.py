"""Pins of the oracle's species transport model (Sec. 2.1 defers viscosity, conductivity and
the effective diffusion coefficient D_s of each species to its references; the model read
here: Blottner viscosity fits, Eucken conductivities, Wilke mixing, hard-sphere binary
diffusion and Blanc's law, with a correction velocity) against what kinetic theory and the
mixture rules fix:

* a single species: Wilke's rule returns the species' own values, so Eucken's relation shows
  directly: k = 15/4 mu R for an atom, k = mu (c_v + 9/4 R) for a molecule (1T);
* a single species: the effective diffusion coefficient is the hard-sphere self-diffusion
  coefficient, rho D / mu = 6/5 exactly (first Chapman-Enskog approximation for rigid spheres
  whose diameter reproduces mu);
* a binary mixture of any composition: Blanc's law gives both species the binary coefficient;
* the diffusive mass fluxes of a non-uniform ionised mixture sum to zero at every face, and so
  does the charge they carry (electrons follow the ions);
* the viscous radius equals the weight of the discrete viscous stencil with the new transport
  (flow block), and the species radius max_s D_s |S|^2/V (Eq. (vislambda)) bounds the species
  diffusion stencil, whose spectral radius lies between the two largest D_s."""
import numpy as np
import pytest

import inputs
import oracle
from test_oracle_spectral import _flow_block, _fd_residual_jacobian

RU = 8314.462618


def _uniform_box(mech, Y, T, Tv=None, u=(0.0, 0.0), p=2000.0, n=2, h=1e-3, transport=1):
    nodes = inputs.box_grid(n, n, lx=n * h, ly=n * h)
    bc = [inputs.BC_PERIODIC] * 4 + [inputs.BC_FARFIELD] * 2
    g = oracle.OracleGrid(nodes, bc, mech, limiter=0)
    g.set_transport(transport)
    g.set_reacting(False)
    g.set_boundary(inputs.freestream(mech, T=T, p=p, mach=2.0), Tw=T)
    M = oracle.gas_info(mech)["M"]
    Y = np.asarray(Y, dtype=float)
    rho = p / (RU * np.sum(Y / M) * T)
    q = oracle.state_cons(mech, 2, rho * Y, np.asarray(u, dtype=float), T, T if Tv is None else Tv)
    Q = np.repeat(q[:, None], g.ncell, axis=1)
    g.set_state(Q)
    g.residual()
    return g, Q


@pytest.mark.parametrize("T", [500.0, 3000.0, 9000.0])
def test_single_species_eucken_and_self_diffusion(T):
    mech = inputs.MECH_AIR5
    M = oracle.gas_info(mech)["M"]
    for s in range(5):
        Y = np.zeros(5)
        Y[s] = 1.0
        g, _ = _uniform_box(mech, Y, T)
        mu, kt, cv = g.field("mu")[0], g.field("kt")[0], g.field("cv")[0]
        R = RU / M[s]
        if s >= 3:                                   # N, O: atoms
            assert abs(kt - 3.75 * mu * R) <= 1e-13 * kt
        else:                                        # N2, O2, NO: molecules
            assert abs(kt - mu * (cv + 2.25 * R)) <= 1e-13 * kt
        rhoD = g.field("rhoDs").reshape(5, -1)[s, 0]
        assert abs(rhoD / mu - 1.2) <= 1e-13


def test_binary_mixture_gives_the_binary_coefficient():
    """Blanc's law in a binary mixture: D_1 = (1 - X_1) / (X_2 / D_12) = D_12 and likewise D_2,
    whatever the composition (D_12 depends on T and the number density only, fixed here by
    T and p)."""
    mech = inputs.MECH_AIR5
    M = oracle.gas_info(mech)["M"]
    D = []
    for x1 in (0.5, 0.2, 0.85):
        Y = np.zeros(5)
        Y[0], Y[1] = x1 * M[0], (1 - x1) * M[1]       # mole fractions x1, 1 - x1 of N2, O2
        Y /= Y.sum()
        g, Q = _uniform_box(mech, Y, 2500.0)
        rho = Q[:5, 0].sum()
        rD = g.field("rhoDs").reshape(5, -1)[:, 0]
        assert abs(rD[0] - rD[1]) <= 1e-14 * rD[0]
        D.append(rD[0] / rho)
    assert max(D) - min(D) <= 1e-12 * max(D), D


def test_diffusive_fluxes_conserve_mass_and_charge():
    mech = inputs.MECH_AIR11
    nodes = inputs.cylinder_ogrid(10, 6)
    g = oracle.OracleGrid(nodes, inputs.cylinder_bc(), mech, limiter=0)
    g.set_transport(1)
    g.set_reacting(False)
    g.set_boundary(inputs.freestream(mech, mach=10.0), Tw=500.0)
    pr = inputs.perturbed_primitive(mech, (g.nj, g.ni), seed=5, ndim=2, T=6000.0, Tv=4500.0, p=8000.0)
    M = oracle.gas_info(mech)["M"]
    rs = pr["rho_s"]
    rs[10] = M[10] * sum(rs[i] / M[i] for i in range(5, 10))      # a neutral mixture
    Q = oracle.prim_to_cons_field(mech, 2, pr)
    g.set_state(Q)
    g.residual()
    Fon = [g.field(f"F{d}").reshape(-1, g.nq) for d in range(2)]
    g.set_viscous(False)
    g.set_state(Q)
    g.residual()
    Foff = [g.field(f"F{d}").reshape(-1, g.nq) for d in range(2)]
    charge = np.array([0, 0, 0, 0, 0, 1, 1, 1, 1, 1, -1], dtype=float)
    for d in range(2):
        J = (Fon[d] - Foff[d])[:, :g.ns]             # diffusive mass fluxes per face
        # the difference of the two runs carries the rounding of the inviscid fluxes
        tol = 1e-14 * np.abs(Fon[d][:, :g.ns]).max()
        assert np.abs(J).max() > 1e4 * tol
        assert np.abs(J.sum(axis=1)).max() <= tol
        assert np.abs((J / M) @ charge).max() <= tol / M.min()


@pytest.mark.parametrize("mech,T,Tv,Y", [
    (inputs.MECH_AIR5, 2000.0, 2000.0, [0.6, 0.15, 0.05, 0.1, 0.1]),
    (inputs.MECH_AIR11, 3000.0, 2200.0, [0.55, 0.12, 0.06, 0.12, 0.15, 0, 0, 0, 0, 0, 0]),
])
def test_viscous_radius_with_species_transport(mech, T, Tv, Y):
    Y = np.asarray(Y) / np.sum(Y)
    h = 2.5e-5
    g, Q = _uniform_box(mech, Y, T, Tv=Tv, p=200.0, n=4, h=h)
    ns, nq = g.ns, g.nq
    rho = Q[:ns, 0].sum()
    c_snd = oracle.state_prim(mech, 2, Q[:, 0])["c"]
    scales = np.concatenate([np.full(ns, rho), np.full(2, rho * c_snd),
                             np.abs(Q[ns:, 0]).max() * np.ones(nq - ns - 2)])
    c, nb = 5, 6
    jac, lam = {}, {}
    for visc in (True, False):
        g.set_viscous(visc)
        jac[visc] = _fd_residual_jacobian(g, Q, c, nb, scales)
        g.set_state(Q)
        g.residual()
        g.build_diagonals(5.0)
        lam[visc] = (g.field("lamF").reshape(-1, 3)[c, 0], g.field("lamC").reshape(-1, 3)[c, 0])
    Jnb = jac[True] - jac[False]
    lvF = 0.5 * (lam[True][0] - lam[False][0])
    lvC = 0.5 * (lam[True][1] - lam[False][1])
    radius = lambda A: np.max(np.abs(np.linalg.eigvals(A)))     # noqa: E731
    assert abs(radius(_flow_block(Jnb, Y, ns)) - lvF) <= 1e-5 * lvF
    # species: max_s D_s |S|^2/V, the radius the operator takes, bounds the stencil's radius
    rD = np.sort(g.field("rhoDs").reshape(ns, -1)[:, c])
    present = Y > 0
    rDp = np.sort(g.field("rhoDs").reshape(ns, -1)[present, c])
    assert abs(lvC - rD[-1] / rho) <= 1e-12 * lvC          # |S|^2/V = 1 on this machine
    rs = radius(Jnb[:ns, :ns])
    assert rDp[-2] / rho * (1 - 1e-6) <= rs <= lvC * (1 + 1e-6), (rs, rDp / rho, lvC)
