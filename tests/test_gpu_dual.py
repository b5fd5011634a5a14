"""Dual time stepping (Sec. 2.3) on the CUDA path against the oracle: physical steps of a
moving, non-uniform half-cylinder flow (split and coupled operators), the periodic
zero-dimensional reactor (the converged inner iterate, FP64 and FP32 operator), batches whose
captured graph reads the physical-time coefficients from device memory, and argument errors.
Tolerance: the FP64 path's 1e-10 per iteration, grown with the iteration count as in the
steady multi-iteration tests."""
import numpy as np
import pytest

import inputs
import oracle
import paper_2403_03440_gb300 as P
from _helpers import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    P.build()
    P.lib()
    yield


MECH = inputs.MECH_AIR11


def half_cylinder_pair(mech):
    """Impulsive start of a Mach 10 flow over the half cylinder (a moving, strongly unsteady
    start-up), oracle and CUDA path from the same freestream state."""
    nodes = inputs.cylinder_half(25, 16)
    bc = inputs.cylinder_half_bc()
    fs = inputs.freestream(mech, T=300.0, p=500.0, mach=10.0)
    ref = oracle.OracleGrid(nodes, bc, mech)
    ref.set_boundary(fs, Tw=500.0)
    gpu = P.Grid(nodes, bc, mech)
    gpu.set_boundary(fs, Tw=500.0)
    Q = ref.freestream_state()
    ref.set_state(Q)
    gpu.set_state(Q)
    return ref, gpu


@pytest.mark.parametrize("mech,scheme,corr,theta", [(MECH, 0, 1, 0.5), (inputs.MECH_AIR5, 0, 2, 0.0),
                                                    (inputs.MECH_AIR5, 1, 1, 0.5)])
def test_physical_steps_match_oracle(mech, scheme, corr, theta):
    """Three physical steps of 4 inner iterations each (the later ones with theta active).
    dt = 1 us is below the pseudo time step of the outer cells and above that of the wall
    cells, so both terms of the diagonal matter."""
    ref, gpu = half_cylinder_pair(mech)
    dt = 1e-6
    ref.set_dual(dt, theta)
    gpu.set_dual(dt, theta)
    cfl = 2.0 if mech == MECH else 5.0
    kw = dict(scheme=scheme, correction=corr, clip=1, cfl=cfl, cfl_start=0.5, ramp_iters=8,
              iters=4)
    for _ in range(3):
        ref.dual_advance()
        gpu.dual_advance()
        sr = ref.step(**kw)
        sg = gpu.step(**kw)
        assert rel(gpu.get_state(), ref.get_state(), ns=ref.ns) < 1e-9
        for k in ("r_species", "r_energy"):
            assert abs(sg[k] - sr[k]) <= 1e-8 * abs(sr[k]), k
    # the residual of cs_residual carries the physical-time term as well
    Rr, nr = ref.residual()
    Rg, ng = gpu.residual()
    assert rel(Rg, Rr, ns=ref.ns) < 1e-9


def reactor_pair(dt, theta):
    from test_oracle_dual import NODES, BC, reactor_freestream
    fs = reactor_freestream()
    ref = oracle.OracleGrid(NODES, BC, MECH)
    ref.set_boundary(fs, Tw=500.0)
    ref.set_state(ref.freestream_state())
    gpu = P.Grid(NODES, BC, MECH)
    gpu.set_boundary(fs, Tw=500.0)
    gpu.set_state(ref.freestream_state())
    ref.set_dual(dt, theta)
    gpu.set_dual(dt, theta)
    return ref, gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_reactor_converged_steps_match_oracle(precision):
    """Four physical steps of the periodic reactor, each converged by 25 inner iterations: the
    fixed point does not depend on the operator's precision, so the FP32 operator lands on the
    oracle's FP64 iterate too."""
    ref, gpu = reactor_pair(5e-7, 0.5)
    kw = dict(scheme=0, correction=1, clip=1, cfl=1e3, cfl_start=1e3, ramp_iters=0, iters=25)
    for _ in range(4):
        ref.dual_advance()
        gpu.dual_advance()
        ref.step(**kw)
        gpu.step(precision=precision, **kw)
    tol = 1e-10 if precision == 0 else 1e-8
    a, b = gpu.get_state(), ref.get_state()
    # the flow moves along x: the y momentum is zero up to rounding noise on both sides, so
    # the momentum rows share the momentum magnitude as their scale
    ns = ref.ns
    scale = np.abs(b).max(axis=1)
    scale[:ns] = scale[:ns].max()
    scale[ns:ns + 2] = np.abs(b[ns:ns + 2]).max()
    assert np.max(np.abs(a - b).max(axis=1) / scale) < tol


def test_dual_in_a_batch_equals_stepping_alone():
    """Physical steps of two grids through a batch (one captured graph reused across physical
    steps: the coefficients change in device memory between replays) equal cs_step alone."""
    def make():
        g = P.Grid(inputs.cylinder_half(24, 16), inputs.cylinder_half_bc(), inputs.MECH_AIR5)
        g.set_boundary(inputs.freestream(inputs.MECH_AIR5, T=300.0, p=500.0, mach=8.0), Tw=500.0)
        g.init_freestream()
        return g
    grids = [make(), make()]
    alone = make()
    for g in grids + [alone]:
        g.set_option("cluster_sweep", 1)
        g.set_option("cluster_size", 2)
    batch = P.Batch(grids)
    o = dict(scheme=0, correction=1, clip=1, cfl=5.0, cfl_start=5.0, ramp_iters=0, precision=0)
    for g in grids + [alone]:
        g.set_dual(1e-5, 0.5)
    for _ in range(3):
        for g in grids + [alone]:
            g.dual_advance()
        batch.step([o, o], iters=4, iters_per_graph=2)
        alone.step(iters=4, **o)
    assert rel(grids[0].get_state(), alone.get_state(), ns=5) < 1e-12
    assert rel(grids[1].get_state(), alone.get_state(), ns=5) < 1e-12


def test_dual_arguments_and_state():
    g = P.Grid(inputs.cylinder_half(8, 6), inputs.cylinder_half_bc(), inputs.MECH_AIR5)
    g.set_boundary(inputs.freestream(inputs.MECH_AIR5), Tw=500.0)
    g.init_freestream()
    with pytest.raises(P.CSError):
        g.dual_advance()                    # off
    with pytest.raises(P.CSError):
        g.set_dual(-1e-6, 0.0)
    with pytest.raises(P.CSError):
        g.set_dual(1e-6, float("nan"))
    # on, but no physical step begun: the steady scheme, bit for bit
    Q0 = g.get_state()
    h = P.Grid(inputs.cylinder_half(8, 6), inputs.cylinder_half_bc(), inputs.MECH_AIR5)
    h.set_boundary(inputs.freestream(inputs.MECH_AIR5), Tw=500.0)
    h.set_state(Q0)
    g.set_dual(1e-6, 0.5)
    kw = dict(scheme=0, correction=1, clip=1, cfl=3.0, iters=3)
    g.step(**kw)
    h.step(**kw)
    assert np.array_equal(g.get_state(), h.get_state())
    g.set_dual(0.0, 0.0)
    with pytest.raises(P.CSError):
        g.dual_advance()
