"""GPU parity of the species transport model (option transport = 1; Sec. 2.1 defers the
transport data to its references, Eq. (vislambda) takes max_s D_s in the species radius):
Blottner / Eucken / Wilke mixture values, per-species effective diffusion by Blanc's law with
the electrons following the ions and a correction velocity, against the oracle with the same
model, element by element at the FP64 tolerance: the transport fields, the residual, the split
and coupled increments and five CS-1 iterations from a perturbed state."""
import numpy as np
import pytest

import inputs
import oracle
import paper_2403_03440_gb300 as P
from _helpers import rel

pytestmark = pytest.mark.gpu
TOL = 1e-10

CASES = {
    "ogrid_air5": (lambda: inputs.cylinder_ogrid(24, 16), inputs.cylinder_bc(), inputs.MECH_AIR5, {}),
    "half_cyl_air11": (lambda: inputs.cylinder_half(25, 16), inputs.cylinder_half_bc(), inputs.MECH_AIR11,
                       dict(T=6000.0, Tv=4500.0, p=8000.0)),
    "box3d_air11": (lambda: inputs.box_grid(6, 5, 4, seed=2, wiggle=0.3), [2, 3, 1, 2, 0, 0],
                    inputs.MECH_AIR11, dict(T=5000.0, Tv=4000.0, p=5000.0)),
}


def make_pair(name, seed=1):
    import torch
    assert torch.cuda.is_available()
    P.build()
    nodes_fn, bc, mech, kw = CASES[name]
    nodes = nodes_fn()
    nd = nodes.shape[0]
    fs = inputs.freestream(mech, T=300.0, p=500.0, mach=10.0)
    ref = oracle.OracleGrid(nodes, bc, mech, limiter=1)
    ref.set_transport(1)
    ref.set_boundary(fs, Tw=500.0)
    gpu = P.Grid(nodes, bc, mech, limiter=1)
    gpu.set_option("transport", 1)
    gpu.set_boundary(fs, Tw=500.0)
    shape = (ref.nj, ref.ni) if nd == 2 else (ref.nk, ref.nj, ref.ni)
    pr = inputs.perturbed_primitive(mech, shape, seed=seed, ndim=nd, **kw)
    Q = oracle.prim_to_cons_field(mech, nd, pr)
    ref.set_state(Q)
    gpu.set_state(Q)
    return ref, gpu, Q


@pytest.mark.parametrize("name", list(CASES))
def test_transport_fields_and_residual(name):
    ref, gpu, _ = make_pair(name)
    Rr, nr = ref.residual()
    Rg, ng = gpu.residual()
    for f in ("mu", "kt", "kv", "rhoD"):
        a, b = gpu.field(f), ref.field(f)
        if np.abs(b).max() > 0:
            assert rel(a, b) < TOL, f
    ns = ref.ns
    assert rel(gpu.field("rhoDs").reshape(ns, -1), ref.field("rhoDs").reshape(ns, -1), ns=ns) < TOL
    assert rel(Rg, Rr, ns=ns) < TOL
    np.testing.assert_allclose(ng, nr, rtol=TOL, atol=0)


@pytest.mark.parametrize("name", list(CASES))
def test_transport_operators_and_iterations(name):
    ref, gpu, Q = make_pair(name, seed=2)
    ref.residual()
    gpu.residual(want_R=False)
    dr = ref.lusgs_split(6.0)
    dg = gpu.lusgs_split(6.0)
    assert rel(gpu.field("lamC").reshape(ref.nd, -1), ref.field("lamC").reshape(-1, 3)[:, :ref.nd].T) < TOL
    assert rel(dg[:ref.nF], dr[:ref.nF]) < TOL
    assert rel(dg[ref.nF:], dr[ref.nF:], ns=ref.ns) < TOL
    # five CS-1 iterations from the impulsively started freestream
    ref.set_state(ref.freestream_state())
    gpu.init_freestream()
    kw = dict(scheme=0, correction=1, clip=1, cfl=2.0, cfl_start=0.5, ramp_iters=5, iters=5)
    ref.step(**kw)
    gpu.step(**kw)
    assert rel(gpu.get_state(), ref.get_state(), ns=ref.ns) < 1e-9


def test_transport_model_changes_the_flow_and_is_rejected_for_a_perfect_gas():
    ref, gpu, Q = make_pair("ogrid_air5")
    R1, _ = gpu.residual()
    gpu.set_option("transport", 0)
    R0, _ = gpu.residual()
    assert rel(R1, R0, ns=gpu.ns) > 1e-6
    nodes = inputs.box_grid(4, 4)
    g = P.Grid(nodes, [2] * 6, inputs.MECH_PERFECT)
    with pytest.raises(P.CSError):
        g.set_option("transport", 1)
