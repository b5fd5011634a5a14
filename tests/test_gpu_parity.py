"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element, on
seeded inputs: residual and its intermediate fields, split and coupled LU-SGS increments,
corrections, multi-iteration steps, and edge cases.

Tolerance: 1e-10 relative per iteration (per variable, normalised by the variable's largest
magnitude on the grid; species by the largest species density), the figure the method's FP64
path is held to.  Both sides compute in FP64; the differences are rounding-order only
(fused multiply-add on the GPU, -ffp-contract=off in the oracle, different but equivalent
reduction orders)."""
import numpy as np
import pytest

import inputs
import oracle
import paper_2403_03440_gb300 as P
from _helpers import rel

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    P.build()
    P.lib()
    yield


CASES = {
    # name: (nodes, bc, mech, perturbation kwargs)
    "c1_ogrid_air5": (lambda: inputs.cylinder_ogrid(48, 32), inputs.cylinder_bc(), inputs.MECH_AIR5, {}),
    "ogrid_air11": (lambda: inputs.cylinder_ogrid(24, 16), inputs.cylinder_bc(), inputs.MECH_AIR11,
                    dict(T=6000.0, Tv=4500.0, p=8000.0)),
    "ragged_box_perfect": (lambda: inputs.box_grid(13, 7, seed=5, wiggle=0.3), [2] * 6,
                           inputs.MECH_PERFECT, {}),
    "box3d_air5_kper": (lambda: inputs.box_grid(6, 5, 4, seed=2, wiggle=0.3), [2, 3, 1, 2, 0, 0],
                        inputs.MECH_AIR5, {}),
    "sphere_cone_air11": (lambda: inputs.sphere_cone(9, 6, 8), inputs.sphere_cone_bc(),
                          inputs.MECH_AIR11, dict(T=5000.0, Tv=4000.0, p=5000.0)),
    "tiny_periodic_air5": (lambda: inputs.cylinder_ogrid(3, 2), inputs.cylinder_bc(), inputs.MECH_AIR5, {}),
    "half_cyl_air11": (lambda: inputs.cylinder_half(25, 16), inputs.cylinder_half_bc(),
                       inputs.MECH_AIR11, dict(T=6000.0, Tv=4500.0, p=8000.0)),
}


def make_pair(name, seed=1, limiter=1, reacting=True, mach=10.0):
    nodes_fn, bc, mech, kw = CASES[name]
    nodes = nodes_fn()
    nd = nodes.shape[0]
    fs = inputs.freestream(mech, T=300.0, p=500.0, mach=mach)
    ref = oracle.OracleGrid(nodes, bc, mech, limiter=limiter)
    ref.set_reacting(reacting)
    ref.set_boundary(fs, Tw=500.0)
    gpu = P.Grid(nodes, bc, mech, limiter=limiter, reacting=reacting)
    gpu.set_boundary(fs, Tw=500.0)
    shape = (ref.nj, ref.ni) if nd == 2 else (ref.nk, ref.nj, ref.ni)
    pr = inputs.perturbed_primitive(mech, shape, seed=seed, ndim=nd, **kw)
    Q = oracle.prim_to_cons_field(mech, nd, pr)
    ref.set_state(Q)
    gpu.set_state(Q)
    return ref, gpu, Q


@pytest.mark.parametrize("name", list(CASES))
def test_geometry_and_freestream(name):
    ref, gpu, _ = make_pair(name)
    assert rel(gpu.field("V"), ref.field("V")) < 1e-14
    for d in range(ref.nd):
        assert rel(gpu.field(f"S{d}"), ref.field(f"S{d}")) < 1e-13
    assert gpu.stag_cell == ref.stag_cell
    gpu.init_freestream()
    # the temperature solve stops at |dT| <= 1e-12 T, which bounds the freestream velocity's
    # agreement (it is Mach times the sound speed at that temperature)
    assert rel(gpu.get_state(), ref.freestream_state(), ns=ref.ns) < 1e-11


@pytest.mark.parametrize("name", list(CASES))
def test_residual_parity(name):
    ref, gpu, _ = make_pair(name)
    Rr, nr = ref.residual()
    Rg, ng = gpu.residual()
    for f in ("T", "Tv", "p", "c", "mu", "rho"):
        assert rel(gpu.field(f), ref.field(f)) < TOL, f
    assert rel(gpu.field("omega").reshape(ref.ns, -1), ref.field("omega").reshape(ref.ns, -1), ns=ref.ns) < TOL
    assert rel(gpu.field("dom").reshape(ref.ns, -1), ref.field("dom").reshape(ref.ns, -1)) < TOL
    for d in range(ref.nd):
        Fo = ref.field(f"F{d}").reshape(-1, ref.nq).T
        Fg = gpu.field(f"F{d}").reshape(ref.nq, -1)
        assert rel(Fg, Fo, ns=ref.ns) < TOL, f"face flux {d}"
    assert rel(Rg, Rr, ns=ref.ns) < TOL
    np.testing.assert_allclose(ng, nr, rtol=TOL, atol=0)


@pytest.mark.parametrize("name", ["c1_ogrid_air5", "half_cyl_air11", "box3d_air5_kper"])
def test_residual_parity_without_h_correction(name):
    """The option that switches the H-correction of the entropy fix off acts on both sides
    alike, and changes the face fluxes."""
    ref, gpu, _ = make_pair(name)
    Fon = gpu.residual()[0].copy()
    ref.set_hcorr(False)
    gpu.set_option("h_correction", 0)
    Rr, nr = ref.residual()
    Rg, ng = gpu.residual()
    assert rel(Rg, Rr, ns=ref.ns) < TOL
    np.testing.assert_allclose(ng, nr, rtol=TOL, atol=0)
    assert rel(Rg, Fon, ns=ref.ns) > 1e-6


@pytest.mark.parametrize("name", list(CASES))
def test_split_operator_parity(name):
    ref, gpu, _ = make_pair(name, seed=2)
    ref.residual()
    gpu.residual(want_R=False)
    cfl = 6.0
    dr = ref.lusgs_split(cfl)
    dg = gpu.lusgs_split(cfl)
    nd = ref.nd
    assert rel(gpu.field("lamF").reshape(nd, -1), ref.field("lamF").reshape(-1, 3)[:, :nd].T) < TOL
    assert rel(gpu.field("lamC").reshape(nd, -1), ref.field("lamC").reshape(-1, 3)[:, :nd].T) < TOL
    assert rel(gpu.field("DF"), ref.field("DF")) < TOL
    assert rel(gpu.field("Ds").reshape(ref.ns, -1), ref.field("Ds").reshape(ref.ns, -1)) < TOL
    # flow rows and species rows of the increment
    assert rel(dg[:ref.nF], dr[:ref.nF]) < TOL
    assert rel(dg[ref.nF:], dr[ref.nF:], ns=ref.ns) < TOL


@pytest.mark.parametrize("name", ["c1_ogrid_air5", "half_cyl_air11", "sphere_cone_air11"])
@pytest.mark.parametrize("scheme", [0, 1])
def test_operator_parity_with_source_radius_in_dtau(name, scheme):
    """Option dtau_source (Sec. 2.2's local time step with lambda_S in its denominator) acts on
    both sides alike and changes the diagonals of both operators."""
    ref, gpu, _ = make_pair(name, seed=2)
    ref.residual()
    gpu.residual(want_R=False)
    cfl = 6.0
    base = gpu.lusgs_split(cfl) if scheme == 0 else gpu.lusgs_coupled(cfl)
    DF0 = gpu.field("DF")
    ref.set_dtau_source(1)
    gpu.set_option("dtau_source", 1)
    dr = ref.lusgs_split(cfl) if scheme == 0 else ref.lusgs_coupled(cfl)
    dg = gpu.lusgs_split(cfl) if scheme == 0 else gpu.lusgs_coupled(cfl)
    assert rel(gpu.field("DF"), ref.field("DF")) < TOL
    assert rel(gpu.field("Ds").reshape(ref.ns, -1), ref.field("Ds").reshape(ref.ns, -1)) < TOL
    assert np.all(gpu.field("DF") >= DF0) and np.any(gpu.field("DF") > DF0 * (1 + 1e-6))
    # (coupled: the tolerance of test_coupled_operator_parity, set by the blocks' condition)
    tol = TOL if scheme == 0 else (1e-8 if ref.ns < 11 else 1e-6)
    nF = ref.nF
    assert rel(dg[:nF], dr[:nF]) < tol
    assert rel(dg[nF:], dr[nF:], ns=(ref.ns if scheme == 0 else ref.nci - nF)) < tol
    assert rel(dg, base) > 1e-8


@pytest.mark.parametrize("name", list(CASES))
def test_coupled_operator_parity(name):
    ref, gpu, _ = make_pair(name, seed=3)
    ref.residual()
    gpu.residual(want_R=False)
    cfl = 4.0
    dr = ref.lusgs_coupled(cfl)
    dg = gpu.lusgs_coupled(cfl)
    assert rel(gpu.field("lamCI").reshape(ref.nd, -1), ref.field("lamCI").reshape(-1, 3)[:, :ref.nd].T) < TOL
    # the coupled blocks carry the chemical source Jacobian: their equilibrated condition
    # number (up to ~4e7 for the ionised mixture, measured on the oracle) bounds how far two
    # correct FP64 LU solves can differ; the non-reacting case below is held to TOL
    tol = 1e-8 if ref.ns < 11 else 1e-6
    assert rel(dg[:ref.nF], dr[:ref.nF]) < tol
    if ref.nci > ref.nF:
        assert rel(dg[ref.nF:], dr[ref.nF:], ns=ref.nci - ref.nF) < tol


@pytest.mark.parametrize("name", ["c1_ogrid_air5", "ogrid_air11", "box3d_air5_kper", "sphere_cone_air11"])
@pytest.mark.parametrize("reacting", [False, True])
def test_coupled_operator_parity_eigenvalue_splitting(name, reacting):
    """The coupled operator with the eigenvalue splitting A+- = (A +- |A|)/2: dense diagonal
    blocks with sum_d |A(S_d)|, |A| x in the sweeps; the non-reacting blocks at the FP64
    tolerance, the reacting ones at the conditioning bound of the spectral case."""
    ref, gpu, _ = make_pair(name, seed=6, reacting=reacting)
    ref.set_ci_splitting(1)
    gpu.set_option("ci_splitting", 1)
    ref.residual()
    gpu.residual(want_R=False)
    dr = ref.lusgs_coupled(4.0)
    dg = gpu.lusgs_coupled(4.0)
    assert rel(gpu.field("lamCI").reshape(ref.nd, -1), ref.field("lamCIv").reshape(-1, 3)[:, :ref.nd].T) < TOL
    tol = TOL * 10 if not reacting else (1e-8 if ref.ns < 11 else 1e-6)
    assert rel(dg[:ref.nF], dr[:ref.nF]) < tol
    assert rel(dg[ref.nF:], dr[ref.nF:], ns=ref.nci - ref.nF) < tol
    # and it is a different operator from the spectral one
    gpu.set_option("ci_splitting", 0)
    gpu.residual(want_R=False)
    ds = gpu.lusgs_coupled(4.0)
    assert rel(ds[:ref.nF], dr[:ref.nF]) > 1e-4


def test_eigenvalue_splitting_multi_iteration_parity():
    """20 coupled iterations with the eigenvalue splitting from the freestream (C1 grid; CFL
    ramped from 0.5 to 5: at CFL 10 this operator, with less diagonal weight than the
    spectral one, loses the impulsive start on both sides)."""
    nodes_fn, bc, mech, _ = CASES["c1_ogrid_air5"]
    nodes = nodes_fn()
    fs = inputs.freestream(mech, T=300.0, p=500.0, mach=10.0)
    ref = oracle.OracleGrid(nodes, bc, mech)
    ref.set_boundary(fs, Tw=500.0)
    ref.set_ci_splitting(1)
    gpu = P.Grid(nodes, bc, mech)
    gpu.set_boundary(fs, Tw=500.0)
    gpu.set_option("ci_splitting", 1)
    Q0 = ref.freestream_state()
    ref.set_state(Q0)
    gpu.set_state(Q0)
    kw = dict(scheme=1, correction=1, clip=1, cfl=5.0, cfl_start=0.5, ramp_iters=50, iters=20)
    sr = ref.step(**kw)
    sg = gpu.step(**kw)
    assert sr["iters_done"] == sg["iters_done"] == 20
    assert rel(gpu.get_state(), ref.get_state(), ns=ref.ns) < 1e-9
    with pytest.raises(P.CSError):
        gpu.set_option("ci_splitting", 2)


@pytest.mark.parametrize("name", ["c1_ogrid_air5", "ogrid_air11", "sphere_cone_air11"])
def test_coupled_operator_parity_nonreacting(name):
    """Without the source Jacobian the coupled blocks are well conditioned: exact sweep
    structure, coupled Jacobian and LU at the FP64 tolerance."""
    ref, gpu, _ = make_pair(name, seed=3, reacting=False)
    ref.residual()
    gpu.residual(want_R=False)
    dr = ref.lusgs_coupled(4.0)
    dg = gpu.lusgs_coupled(4.0)
    assert rel(dg[:ref.nF], dr[:ref.nF]) < TOL
    assert rel(dg[ref.nF:], dr[ref.nF:], ns=ref.nci - ref.nF) < TOL


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("clip", [0, 1])
def test_correction_parity(mode, clip):
    ref, gpu, Q = make_pair("c1_ogrid_air5", seed=4)
    rng = np.random.default_rng(9)
    n = ref.nci if mode == 0 else ref.nsplit
    dQ = np.zeros((n, ref.ncell))
    rho = Q[:ref.ns].sum(axis=0)
    dQ[0] = 0.05 * rho * rng.uniform(-1, 1, ref.ncell)
    dQ[1:ref.nF] = 0.01 * Q[ref.ns:] * rng.uniform(-1, 1, (ref.nF - 1, ref.ncell))
    k = n - ref.nF
    dQ[ref.nF:] = 0.5 * Q[:k] * rng.uniform(-1.5, 1, (k, ref.ncell))   # some go negative
    nr = ref.correct(mode, clip, dQ)
    ng = gpu.correct(mode, clip, dQ)
    assert nr == ng
    assert rel(gpu.get_state(), ref.get_state(), ns=ref.ns) < 1e-14


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_correction_parity_with_update_limit(mode):
    """The update limit scales a cell's whole increment by min(1, f rho / |d rho|), then
    halves it while the thermal band is left, on both sides alike; the increments here exceed
    f = 0.02 of the density in most cells."""
    ref, gpu, Q = make_pair("c1_ogrid_air5", seed=5)
    rng = np.random.default_rng(11)
    n = ref.nci if mode == 0 else ref.nsplit
    dQ = np.zeros((n, ref.ncell))
    rho = Q[:ref.ns].sum(axis=0)
    dQ[0] = 0.05 * rho * rng.uniform(-1, 1, ref.ncell)
    dQ[1:ref.nF] = 0.01 * Q[ref.ns:] * rng.uniform(-1, 1, (ref.nF - 1, ref.ncell))
    k = n - ref.nF
    dQ[ref.nF:] = 0.5 * Q[:k] * rng.uniform(-1.5, 1, (k, ref.ncell))
    Qlim = ref.get_state()
    ref.set_update_limit(0.02)
    gpu.set_option("update_limit", 0.02)
    nr = ref.correct(mode, 0, dQ)      # no clipping: the new density is exactly rho + alpha d rho
    ng = gpu.correct(mode, 0, dQ)
    assert nr == ng
    Qr = ref.get_state()
    assert rel(gpu.get_state(), Qr, ns=ref.ns) < 1e-14
    # no cell's density moved by more than 2 % (plus rounding), and the limit acted in most
    # cells (the density moved by less than the raw increment)
    drho = np.abs(Qr[:ref.ns].sum(axis=0) - Qlim[:ref.ns].sum(axis=0))
    assert np.all(drho <= 0.02 * rho * (1 + 1e-12))
    assert np.mean(drho < 0.99 * np.abs(dQ[0])) > 0.3


@pytest.mark.parametrize("scheme,corr", [(0, 1), (0, 2), (1, 0)])
def test_multi_iteration_parity(scheme, corr):
    """20 iterations from the freestream (impulsive start, CFL ramp) on the C1 grid."""
    nodes_fn, bc, mech, _ = CASES["c1_ogrid_air5"]
    nodes = nodes_fn()
    fs = inputs.freestream(mech, T=300.0, p=500.0, mach=10.0)
    ref = oracle.OracleGrid(nodes, bc, mech)
    ref.set_boundary(fs, Tw=500.0)
    gpu = P.Grid(nodes, bc, mech)
    gpu.set_boundary(fs, Tw=500.0)
    Q0 = ref.freestream_state()
    ref.set_state(Q0)
    gpu.set_state(Q0)
    kw = dict(scheme=scheme, correction=max(corr, 1), clip=1, cfl=10.0, cfl_start=1.0,
              ramp_iters=50, iters=20)
    sr = ref.step(**kw)
    sg = gpu.step(**kw)
    assert sr["iters_done"] == sg["iters_done"] == 20
    assert rel(gpu.get_state(), ref.get_state(), ns=ref.ns) < 1e-9
    for k in ("r_species", "r_energy", "q_stag"):
        assert abs(sg[k] - sr[k]) <= 1e-8 * abs(sr[k]), k


def test_multi_iteration_parity_with_source_radius_in_dtau():
    """20 iterations from the freestream with the local time step of Sec. 2.2 carrying the
    source radius (option dtau_source) on the 11-species two-temperature half cylinder."""
    nodes_fn, bc, mech, _ = CASES["half_cyl_air11"]
    nodes = nodes_fn()
    fs = inputs.freestream(mech, T=300.0, p=500.0, mach=15.0)
    ref = oracle.OracleGrid(nodes, bc, mech, limiter=0)
    ref.set_boundary(fs, Tw=500.0)
    ref.set_dtau_source(1)
    gpu = P.Grid(nodes, bc, mech, limiter=0)
    gpu.set_boundary(fs, Tw=500.0)
    gpu.set_option("dtau_source", 1)
    Q0 = ref.freestream_state()
    ref.set_state(Q0)
    gpu.set_state(Q0)
    kw = dict(scheme=0, correction=1, clip=1, cfl=20.0, cfl_start=0.5, ramp_iters=10, iters=20)
    sr = ref.step(**kw)
    sg = gpu.step(**kw)
    assert sr["iters_done"] == sg["iters_done"] == 20
    assert rel(gpu.get_state(), ref.get_state(), ns=ref.ns) < 1e-9
    for k in ("r_species", "r_energy", "q_stag"):
        assert abs(sg[k] - sr[k]) <= 1e-8 * abs(sr[k]), k


def test_full_size_c2_parity():
    """The 384 x 256 11-species two-temperature cylinder (the benchmark's grid and launch
    configuration): full residual, split increments and CS-1 update against the oracle on a
    seeded non-uniform state."""
    mech = inputs.MECH_AIR11
    ni, nj = 384, 256
    nodes = inputs.cylinder_ogrid(ni, nj, dr1=5e-5 / 8)
    fs = inputs.freestream(mech, T=300.0, p=500.0, mach=15.0)
    ref = oracle.OracleGrid(nodes, inputs.cylinder_bc(), mech)
    ref.set_boundary(fs, Tw=500.0)
    gpu = P.Grid(nodes, inputs.cylinder_bc(), mech)
    gpu.set_boundary(fs, Tw=500.0)
    pr = inputs.perturbed_primitive(mech, (nj, ni), seed=11, ndim=2, T=5000.0, Tv=4000.0, p=6000.0)
    Q = oracle.prim_to_cons_field(mech, 2, pr)
    ref.set_state(Q)
    gpu.set_state(Q)
    Rr, nr = ref.residual()
    Rg, ng = gpu.residual()
    assert rel(Rg, Rr, ns=ref.ns) < TOL
    dr = ref.lusgs_split(10.0)
    dg = gpu.lusgs_split(10.0)
    assert rel(dg[:ref.nF], dr[:ref.nF]) < TOL
    assert rel(dg[ref.nF:], dr[ref.nF:], ns=ref.ns) < TOL
    ref.correct(1, 1)
    gpu.correct(1, 1)
    assert rel(gpu.get_state(), ref.get_state(), ns=ref.ns) < TOL


def test_uniform_freestream_is_fixed_point():
    """Degenerate case: uniform freestream on an all-far-field grid gives R = 0 and dQ = 0."""
    nodes = inputs.box_grid(9, 7, seed=1, wiggle=0.3)
    mech = inputs.MECH_AIR11
    fs = inputs.freestream(mech, T=800.0, p=3000.0, mach=3.0, direction=(0.8, 0.6, 0.0))
    gpu = P.Grid(nodes, [2] * 6, mech, reacting=False)
    gpu.set_boundary(fs)
    gpu.init_freestream()
    Q0 = gpu.get_state()
    R, _ = gpu.residual()
    F = gpu.field("F0").reshape(gpu.nq, -1)
    scale = np.abs(F).max(axis=1)
    scale[:gpu.ns] = scale[:gpu.ns].max()
    assert np.max(np.abs(R).max(axis=1) / scale) < 1e-12
    gpu.step(scheme=0, correction=2, cfl=50.0, iters=3)
    assert rel(gpu.get_state(), Q0, ns=gpu.ns) < 1e-13


def test_error_paths():
    import torch
    ref, gpu, Q = make_pair("c1_ogrid_air5")
    fresh = P.Grid(inputs.cylinder_ogrid(8, 4), inputs.cylinder_bc(), inputs.MECH_AIR5)
    with pytest.raises(P.CSError) as e:
        fresh.residual()                              # no boundary data yet
    assert e.value.status == P.CS_ERR_STATE
    with pytest.raises(P.CSError) as e:
        gpu.lusgs_split(5.0)                          # no residual yet
    assert e.value.status == P.CS_ERR_STATE
    with pytest.raises(P.CSError) as e:
        gpu.residual()
        gpu.lusgs_split(-1.0)                         # bad CFL
    assert e.value.status == P.CS_ERR_ARG
    # a negative species density is caught by the primitive kernel's own check
    Qbad = Q.copy()
    Qbad[0, 17] = -1.0
    gpu.set_state(torch.from_numpy(Qbad).cuda())
    with pytest.raises(P.CSError) as e:
        gpu.residual()
    assert e.value.status == P.CS_ERR_NONPHYSICAL
    # the grid stays usable after the error
    gpu.set_state(Q)
    gpu.residual()


def test_device_and_host_buffers_agree():
    """The same call with device (torch) and host (numpy) buffers gives identical results."""
    import torch
    ref, gpu, Q = make_pair("ogrid_air11", seed=6)
    Rh, _ = gpu.residual()
    Rd = torch.empty((gpu.nq, gpu.ncell), dtype=torch.float64, device="cuda")
    gpu.set_state(torch.from_numpy(Q).cuda())      # same temperature warm start as the first call
    gpu.residual(R_out=Rd)
    assert np.array_equal(Rd.cpu().numpy(), Rh)


@pytest.mark.parametrize("name", ["c1_ogrid_air5", "ogrid_air11", "ragged_box_perfect", "tiny_periodic_air5"])
def test_cluster_sweep_equals_hyperplane_sweep(name):
    """The one-launch cluster sweep (2D) and the one-launch-per-hyperplane sweep perform the
    same arithmetic in the same order (the compiler may contract multiply-adds differently
    in the two kernels, so they agree to rounding)."""
    ref, gpu, Q = make_pair(name, seed=7)
    out = {}
    # wavefront-record cluster, direct cluster, assembled couplings (point to point between
    # CTAs; with a cluster barrier), per hyperplane
    for mode in (2, 1, 5, 6, 0):
        gpu.set_option("cluster_sweep", mode)
        gpu.set_state(Q)
        gpu.residual(want_R=False)
        out[mode] = gpu.lusgs_split(8.0)
    # the assembled couplings with every cluster size that holds the rows (at most 32 per CTA;
    # C above the row count leaves CTAs without rows)
    for mode in (5, 6):
        for C in (2, 4, 16):
            if -(-ref.nj // C) > 32:
                continue
            gpu.set_option("cluster_sweep", mode)
            gpu.set_option("cluster_size", C)
            gpu.set_state(Q)
            gpu.residual(want_R=False)
            out[(mode, C)] = gpu.lusgs_split(8.0)
    gpu.set_option("cluster_size", 0)
    gpu.set_option("cluster_sweep", 3)
    a, b = out[2], out[0]
    for m in (1, 2):
        assert rel(out[m][:ref.nF], b[:ref.nF]) < 1e-13, m
        assert rel(out[m][ref.nF:], b[ref.nF:], ns=ref.ns) < 1e-13, m
    # the couplings are multiplied by D^-1 before the sweep (another rounding order)
    for m in [5, 6] + [k for k in out if isinstance(k, tuple)]:
        assert rel(out[m][:ref.nF], b[:ref.nF]) < 1e-12, m
        assert rel(out[m][ref.nF:], b[ref.nF:], ns=ref.ns) < 1e-12, m
    ref.residual()
    d = ref.lusgs_split(8.0)
    for m in (2, 5, 6):
        assert rel(out[m][:ref.nF], d[:ref.nF]) < TOL, m
        assert rel(out[m][ref.nF:], d[ref.nF:], ns=ref.ns) < TOL, m


@pytest.mark.parametrize("nodes_fn,bc,mech", [
    (lambda: inputs.cylinder_half(40, 100), inputs.cylinder_half_bc(), inputs.MECH_AIR5),
    (lambda: inputs.cylinder_half(25, 16), inputs.cylinder_half_bc(), inputs.MECH_AIR11),
    (lambda: inputs.cylinder_ogrid(24, 16), inputs.cylinder_bc(), inputs.MECH_AIR11),
])
def test_block_sweep_equals_cluster_sweep_fp32(nodes_fn, bc, mech):
    """FP32 operator: the one-CTA-per-component sweep (every row in one CTA, __syncthreads
    between hyperplanes) performs the record cluster kernel's arithmetic; 100 rows span 4
    warps.  Both, and the sweep over FP32 couplings assembled in FP64 (point-to-point cluster
    exchange), agree with the FP64 oracle to FP32 rounding."""
    nodes = nodes_fn()
    fs = inputs.freestream(mech, T=300.0, p=500.0, mach=10.0)
    ref = oracle.OracleGrid(nodes, bc, mech)
    ref.set_boundary(fs, Tw=500.0)
    gpu = P.Grid(nodes, bc, mech)
    gpu.set_boundary(fs, Tw=500.0)
    pr = inputs.perturbed_primitive(mech, (ref.nj, ref.ni), seed=9, ndim=2)
    Q = oracle.prim_to_cons_field(mech, 2, pr)
    ref.set_state(Q)
    out = {}
    # one CTA per component, wavefront records, assembled couplings point to point (FP32
    # records)
    for mode in (4, 2, 5):
        gpu.set_option("cluster_sweep", mode)
        gpu.set_state(Q)
        gpu.residual(want_R=False)
        out[mode] = gpu.lusgs_split(8.0, precision=1)
    gpu.set_option("cluster_sweep", 3)
    assert rel(out[4][:ref.nF], out[2][:ref.nF]) < 1e-6
    assert rel(out[4][ref.nF:], out[2][ref.nF:], ns=ref.ns) < 1e-6
    ref.residual()
    d = ref.lusgs_split(8.0)
    for m in (4, 5):
        assert rel(out[m][:ref.nF], d[:ref.nF]) < 1e-4, m
        assert rel(out[m][ref.nF:], d[ref.nF:], ns=ref.ns) < 1e-4, m


@pytest.mark.parametrize("name", ["c1_ogrid_air5", "ogrid_air11", "box3d_air5_kper"])
def test_mixed_precision_split_operator(name):
    """Mixed precision: the split sweeps compute in FP32 from FP64 radii, diagonals and
    right-hand side.  Against the FP64 oracle the increments agree to FP32 rounding carried
    through the sweep recurrence (bound 1e-4 per variable, measured ~1e-6)."""
    ref, gpu, _ = make_pair(name, seed=2)
    ref.residual()
    gpu.residual(want_R=False)
    dr = ref.lusgs_split(6.0)
    dg = gpu.lusgs_split(6.0, precision=1)
    e1 = rel(dg[:ref.nF], dr[:ref.nF])
    e2 = rel(dg[ref.nF:], dr[ref.nF:], ns=ref.ns)
    assert e1 < 1e-4 and e2 < 1e-4, (e1, e2)
    assert e1 > 0.0          # it really ran in FP32
