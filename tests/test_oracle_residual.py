"""Pins of the oracle's geometry and residual R(Q) (Sec. 2.2 Eq. (iterate) in finite-volume
form; Sec. 3.2 MUSCL/Roe and central viscous fluxes): closure of the cell faces, exact
volumes, freestream preservation, telescoping conservation, mirror symmetry, exact gradients
of linear fields, Couette shear stress and zero net diffusive mass flux."""
import math

import numpy as np
import pytest

import inputs
import oracle
from _helpers import rel_err

BOX_BC = [inputs.BC_FARFIELD] * 6


def face_closure(g):
    """max over cells of |sum_out S| / max |S|."""
    nd, ni, nj, nk = g.nd, g.ni, g.nj, g.nk
    S = [g.field(f"S{d}").reshape(-1, 3) for d in range(nd)]
    if nd == 2:
        Si = S[0].reshape(nj, ni + 1, 3)
        Sj = S[1].reshape(nj + 1, ni, 3)
        tot = Si[:, 1:] - Si[:, :-1] + Sj[1:] - Sj[:-1]
    else:
        Si = S[0].reshape(nk, nj, ni + 1, 3)
        Sj = S[1].reshape(nk, nj + 1, ni, 3)
        Sk = S[2].reshape(nk + 1, nj, ni, 3)
        tot = Si[:, :, 1:] - Si[:, :, :-1] + Sj[:, 1:] - Sj[:, :-1] + Sk[1:] - Sk[:-1]
    scale = max(np.max(np.abs(s)) for s in S)
    return np.max(np.abs(tot)) / scale


def test_geometry_cylinder_closure_and_area():
    ni, nj = 48, 32
    nodes = inputs.cylinder_ogrid(ni, nj)
    g = oracle.OracleGrid(nodes, inputs.cylinder_bc(), inputs.MECH_AIR5)
    assert face_closure(g) < 1e-14
    V = g.field("V")
    assert np.all(V > 0)

    def ring_area(j):   # shoelace over the node ring j (independent of the cell split)
        x, y = nodes[0, j, :ni], nodes[1, j, :ni]
        return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))
    assert abs(V.sum() / (ring_area(nj) - ring_area(0)) - 1) < 1e-13


def test_geometry_3d_box_and_sphere_cone():
    nodes = inputs.box_grid(4, 3, 5, lx=1.0, ly=2.0, lz=0.5, seed=1, wiggle=0.3)
    g = oracle.OracleGrid(nodes, BOX_BC, inputs.MECH_AIR5)
    assert face_closure(g) < 1e-14
    assert abs(g.field("V").sum() - 1.0) < 1e-13
    nodes = inputs.sphere_cone(8, 6, 8)
    g = oracle.OracleGrid(nodes, inputs.sphere_cone_bc(), inputs.MECH_AIR11)
    assert face_closure(g) < 1e-14
    assert np.all(g.field("V") > 0)
    # i-faces on the axis are degenerate (zero area)
    Si = g.field("S0").reshape(8, 6, 9, 3)
    assert np.max(np.abs(Si[:, :, 0])) == 0.0


@pytest.mark.parametrize("nd,mech", [(2, inputs.MECH_AIR5), (2, inputs.MECH_AIR11),
                                     (3, inputs.MECH_AIR5), (3, inputs.MECH_AIR11)])
def test_freestream_preservation(nd, mech):
    if nd == 2:
        nodes = inputs.box_grid(7, 6, seed=3, wiggle=0.4)
    else:
        nodes = inputs.box_grid(4, 5, 3, seed=3, wiggle=0.4)
    g = oracle.OracleGrid(nodes, BOX_BC, mech, limiter=1)
    fs = inputs.freestream(mech, T=800.0, p=3000.0, mach=3.0, direction=(0.8, 0.5, 0.3))
    g.set_boundary(fs, Tw=500.0)
    g.set_reacting(False)
    Q = g.freestream_state()
    g.set_state(Q)
    R, _ = g.residual()
    F = g.field("F0").reshape(-1, g.nq)
    scale = np.max(np.abs(F), axis=0)          # flux magnitude per variable
    scale[:g.ns] = np.max(scale[:g.ns])        # species: relative to the mass flux
    assert np.max(np.abs(R).max(axis=1) / scale) < 1e-12
    # a full CS step keeps the uniform state
    g.step(scheme=0, correction=1, cfl=20.0)
    assert rel_err(g.get_state(), Q) < 1e-13


def random_cylinder_state(mech, ni, nj, seed, limiter=1):
    nodes = inputs.cylinder_ogrid(ni, nj)
    g = oracle.OracleGrid(nodes, inputs.cylinder_bc(), mech, limiter=limiter)
    fs = inputs.freestream(mech, T=300.0, p=500.0, mach=10.0)
    g.set_boundary(fs, Tw=500.0)
    pr = inputs.perturbed_primitive(mech, (nj, ni), seed=seed, ndim=2)
    return g, pr


@pytest.mark.parametrize("mech", [inputs.MECH_AIR5, inputs.MECH_AIR11])
def test_mirror_symmetry(mech):
    """The O-grid is symmetric about the stagnation line (cell i <-> (ni - i) mod ni): a
    mirror-symmetric state has a mirror-symmetric residual."""
    ni, nj = 24, 10
    g, pr = random_cylinder_state(mech, ni, nj, 5)
    mi = (ni - np.arange(ni)) % ni
    for k in pr:
        if k == "u":
            pr[k][0] = 0.5 * (pr[k][0] + pr[k][0][:, mi])
            pr[k][1] = 0.5 * (pr[k][1] - pr[k][1][:, mi])
        else:
            pr[k] = 0.5 * (pr[k] + pr[k][..., mi])
    g.set_state(oracle.prim_to_cons_field(mech, 2, pr))
    R, _ = g.residual()
    R = R.reshape(g.nq, nj, ni)
    Rm = R[:, :, mi].copy()
    Rm[g.ns + 1] *= -1
    assert np.max(rel_err(R, Rm, axis=(1, 2))) < 1e-12


@pytest.mark.parametrize("mech", [inputs.MECH_AIR5, inputs.MECH_AIR11])
def test_mirror_symmetry_half_grid(mech):
    """The windward half grid with odd ni is symmetric about the stagnation line (cell i <->
    ni - 1 - i) and ends in outflow boundaries on both sides: a mirror-symmetric state has a
    mirror-symmetric residual, with the H-correction of the entropy fix switched on."""
    ni, nj = 15, 10
    nodes = inputs.cylinder_half(ni, nj)
    g = oracle.OracleGrid(nodes, inputs.cylinder_half_bc(), mech, limiter=1)
    g.set_boundary(inputs.freestream(mech, T=300.0, p=500.0, mach=10.0), Tw=500.0)
    pr = inputs.perturbed_primitive(mech, (nj, ni), seed=6, ndim=2)
    mi = ni - 1 - np.arange(ni)
    for k in pr:
        if k == "u":
            pr[k][0] = 0.5 * (pr[k][0] + pr[k][0][:, mi])
            pr[k][1] = 0.5 * (pr[k][1] - pr[k][1][:, mi])
        else:
            pr[k] = 0.5 * (pr[k] + pr[k][..., mi])
    g.set_state(oracle.prim_to_cons_field(mech, 2, pr))
    R, _ = g.residual()
    R = R.reshape(g.nq, nj, ni)
    Rm = R[:, :, mi].copy()
    Rm[g.ns + 1] *= -1
    assert np.max(rel_err(R, Rm, axis=(1, 2))) < 1e-11


def test_h_correction_closed_form():
    """H-correction of the entropy fix (Sanders, Morano and Druguet 1998) on a 2 x 3 Cartesian
    box, first order, eps = 0.  Across each i-face only the density jumps (same p, u = (0, v)
    on both sides), so Roe's dissipation is l2 * (rho_R - rho_L) with l2 the fixed modulus of
    the zero wave speed u_n = 0, and the mass flux is -|S| l2 (rho_R - rho_L) / 2.  With the
    width 2 eta_H, l2 = eta_H: the largest of (|jump of u.n| + |jump of c|) / 2 over the face
    and the j-faces bounding its two cells, boundary faces counting 0.  Without the
    correction, l2 = 0 and the flux vanishes."""
    mech = inputs.MECH_PERFECT
    ni, nj = 2, 3
    nodes = inputs.box_grid(ni, nj, lx=2.0, ly=3.0)
    p = np.array([1000.0, 1000.0, 2000.0])                   # per row j
    v = np.array([0.0, 300.0, -100.0])                       # per row j
    rho = np.array([[0.010, 0.012], [0.010, 0.011], [0.020, 0.0205]])   # [j, i]
    Rgas = 8314.462618 / 28.9647
    pr = {"rho_s": rho[None], "u": np.zeros((2, nj, ni)), "T": p[:, None] / (rho * Rgas)}
    pr["u"][1] = v[:, None]
    pr["Tv"] = pr["T"]
    c = np.sqrt(1.4 * p[:, None] / rho)                      # diatomic perfect gas, gamma 1.4

    def eta_j(i, j):                                         # j-face between rows j and j+1
        if j < 0 or j + 1 >= nj:
            return 0.0
        return 0.5 * (abs(v[j + 1] - v[j]) + abs(c[j + 1, i] - c[j, i]))

    for hcorr in (True, False):
        g = oracle.OracleGrid(nodes, BOX_BC, mech, limiter=0, efix=0.0)
        g.set_hcorr(hcorr)
        g.set_boundary(inputs.freestream(mech, T=300.0, p=1000.0, mach=0.0))
        g.set_state(oracle.prim_to_cons_field(mech, 2, pr))
        g.set_reacting(False)
        g.residual()
        F0 = g.field("F0").reshape(-1, g.nq)
        for j in range(nj):
            etaH = max(0.5 * abs(c[j, 1] - c[j, 0]), eta_j(0, j), eta_j(0, j - 1),
                       eta_j(1, j), eta_j(1, j - 1))
            want = -0.5 * 1.0 * (etaH if hcorr else 0.0) * (rho[j, 1] - rho[j, 0])
            got = F0[1 + (ni + 1) * j, 0]
            assert abs(got - want) <= 1e-9 * 0.5 * etaH * abs(rho[j, 1] - rho[j, 0]), (hcorr, j, got, want)


@pytest.mark.parametrize("mech", [inputs.MECH_AIR5, inputs.MECH_AIR11])
def test_telescoping_conservation(mech):
    """sum over cells of R equals the net outward flux through the boundary faces (the
    interior faces cancel), with the sources switched off."""
    ni, nj = 12, 8
    g, pr = random_cylinder_state(mech, ni, nj, 6)
    g.set_reacting(False)
    g.set_state(oracle.prim_to_cons_field(mech, 2, pr))
    R, _ = g.residual()
    F1 = g.field("F1").reshape(nj + 1, ni, g.nq)
    boundary = F1[nj].sum(axis=0) - F1[0].sum(axis=0)
    tot = R.sum(axis=1)
    scale = np.abs(g.field("F1")).reshape(-1, g.nq).max(axis=0)
    assert np.max(np.abs(tot - boundary) / scale) < 1e-12


def test_linear_field_gradient_exact():
    """Green-Gauss gradients are exact for linear fields on parallelogram cells."""
    mech = inputs.MECH_AIR5
    ni, nj = 6, 5
    x = np.linspace(0, 1, ni + 1)
    y = np.linspace(0, 1, nj + 1)
    X, Y = np.meshgrid(x, y)
    nodes = np.stack([X + 0.3 * Y, Y])           # sheared grid: parallelograms
    g = oracle.OracleGrid(nodes, BOX_BC, mech)
    fs = inputs.freestream(mech, T=500.0, p=1000.0, mach=0.5)
    g.set_boundary(fs)
    xc = g.field("xc").reshape(-1, 3)
    T = 1000.0 + 300.0 * xc[:, 0] - 200.0 * xc[:, 1]
    u = np.stack([50.0 + 10 * xc[:, 0] + 20 * xc[:, 1], -5.0 + 40 * xc[:, 0]])
    rhos = np.tile(np.array([0.7, 0.2, 0.05, 0.03, 0.02])[:, None] * 0.01, (1, ni * nj))
    Q = oracle.prim_to_cons_field(mech, 2, dict(rho_s=rhos, u=u, T=T, Tv=T))
    g.set_state(Q)
    g.set_reacting(False)
    g.residual()
    gr = g.field("grad").reshape(ni * nj, -1, 3)
    inner = [i + ni * j for j in range(1, nj - 1) for i in range(1, ni - 1)]
    # variables: u, v, T, Y_s
    np.testing.assert_allclose(gr[inner, 0, :2], np.tile([10.0, 20.0], (len(inner), 1)), rtol=0, atol=1e-9)
    np.testing.assert_allclose(gr[inner, 1, :2], np.tile([40.0, 0.0], (len(inner), 1)), rtol=0, atol=1e-9)
    np.testing.assert_allclose(gr[inner, 2, :2], np.tile([300.0, -200.0], (len(inner), 1)), rtol=0, atol=1e-8)


def test_couette_shear_stress():
    """Uniform shear u = a y: the viscous momentum flux through interior j-faces is
    -mu a dx and the viscous work term is -u_f mu a dx (Stokes shear stress, Sec. 2.1)."""
    mech = inputs.MECH_PERFECT
    ni, nj = 5, 6
    nodes = inputs.box_grid(ni, nj, lx=0.5, ly=0.3)
    g = oracle.OracleGrid(nodes, BOX_BC, mech, limiter=1, efix=1e-12)
    fs = inputs.freestream(mech, T=400.0, p=2000.0, mach=0.3)
    g.set_boundary(fs)
    xc = g.field("xc").reshape(-1, 3)
    a = 800.0
    T = np.full(ni * nj, 400.0)
    u = np.stack([a * xc[:, 1], np.zeros(ni * nj)])
    p = 2000.0
    rho = p / (8314.462618 / 28.9647 * 400.0)
    Q = oracle.prim_to_cons_field(mech, 2, dict(rho_s=np.full((1, ni * nj), rho), u=u, T=T))
    g.set_state(Q)
    g.residual()
    F1 = g.field("F1").reshape(nj + 1, ni, g.nq)
    mu = g.field("mu")[0]
    dx = 0.5 / ni
    for j in range(2, nj - 1):
        yf = 0.3 * j / nj
        for i in range(1, ni - 1):      # away from the side boundaries' one-sided gradients
            assert abs(F1[j, i, 1] - (-mu * a * dx)) < 1e-10 * mu * a * dx
            assert abs(F1[j, i, 2] - p * dx) < 1e-10 * p * dx
            assert abs(F1[j, i, 3] - (-(a * yf) * mu * a * dx)) < 1e-9 * abs(a * yf * mu * a * dx)


def test_species_diffusion_sums_to_zero():
    """Fick diffusion with one coefficient and no correction velocity (Sec. 2.1) carries no
    net mass: sum_s of the species face fluxes vanishes for a fluid at rest."""
    mech = inputs.MECH_AIR11
    ni, nj = 6, 5
    nodes = inputs.box_grid(ni, nj, seed=2, wiggle=0.3)
    g = oracle.OracleGrid(nodes, BOX_BC, mech, limiter=1, efix=0.0)
    g.set_hcorr(False)      # no entropy fix at all: Roe adds no dissipation at rest
    fs = inputs.freestream(mech, T=300.0, p=1000.0, mach=0.0)
    g.set_boundary(fs)
    pr = inputs.perturbed_primitive(mech, (nj, ni), seed=8, ndim=2)
    rho = pr["rho_s"].sum(axis=0)
    Y = pr["rho_s"] / rho
    T = pr["T"]
    # constant pressure, zero velocity, varying composition and temperature
    M = oracle.gas_info(mech)["M"]
    Rmix = (Y / M[:, None, None]).sum(axis=0) * 8314.462618
    rho = 1000.0 / (Rmix * T)
    pr["rho_s"] = Y * rho
    pr["u"] = np.zeros_like(pr["u"])
    pr["Tv"] = T
    g.set_state(oracle.prim_to_cons_field(mech, 2, pr))
    g.set_reacting(False)
    g.residual()
    for d in range(2):
        F = g.field(f"F{d}").reshape(-1, g.nq)
        tot = F[:, :g.ns].sum(axis=1)
        scale = np.max(np.abs(F[:, :g.ns]))
        assert scale > 0
        assert np.max(np.abs(tot)) / scale < 1e-9
