"""Batches of independent cases: K iterations of every case captured into one CUDA graph and
replayed (cs_batch_* of the C ABI), with the per-case sweep configuration chosen by the
autotuner.  A batch must give what cs_step gives case by case, and the oracle's iterate."""
import numpy as np
import pytest

import inputs
import oracle
from _helpers import rel

import paper_2403_03440_gb300 as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    P.build()
    P.lib()
    yield


# (nodes, bc, mech, step options)
CASES = [
    (lambda: inputs.cylinder_half(48, 32), inputs.cylinder_half_bc(), inputs.MECH_AIR5,
     dict(scheme=0, correction=1, cfl=10.0, cfl_start=1.0, ramp_iters=20, precision=1)),
    (lambda: inputs.cylinder_half(40, 24, dr1=6e-5), inputs.cylinder_half_bc(), inputs.MECH_AIR11,
     dict(scheme=0, correction=1, cfl=2.0, cfl_start=0.5, ramp_iters=50, precision=0)),
    (lambda: inputs.cylinder_half(30, 20), inputs.cylinder_half_bc(), inputs.MECH_AIR5,
     dict(scheme=0, correction=2, cfl=5.0, cfl_start=1.0, ramp_iters=0, precision=0)),
    (lambda: inputs.box_grid(6, 5, 4, seed=2, wiggle=0.3), [2, 3, 1, 2, 0, 0], inputs.MECH_AIR5,
     dict(scheme=0, correction=1, cfl=3.0, cfl_start=1.0, ramp_iters=10, precision=0)),
    (lambda: inputs.cylinder_half(24, 16), inputs.cylinder_half_bc(), inputs.MECH_AIR5,
     dict(scheme=1, correction=0, cfl=4.0, cfl_start=1.0, ramp_iters=10, precision=0)),
]


def make_grid(k):
    nodes_fn, bc, mech, _ = CASES[k]
    g = P.Grid(nodes_fn(), bc, mech)
    g.set_boundary(inputs.freestream(mech, T=300.0, p=500.0, mach=10.0), Tw=500.0)
    g.init_freestream()
    return g


def test_batch_equals_case_by_case_steps():
    """12 iterations as 3 replays of a 4-iteration graph, then 6 more as 6 replays of a
    1-iteration graph (the ramp counters carry on): every case matches the same case stepped
    alone with cs_step and the tuned sweep configuration."""
    grids = [make_grid(k) for k in range(len(CASES))]
    batch = P.Batch(grids)
    choice = batch.tune(precision=0, trials=2)
    opts = [c[3] for c in CASES]
    batch.step(opts, iters=12, iters_per_graph=4)
    stats = batch.step(opts, iters=6, iters_per_graph=1)
    for k in range(len(CASES)):
        alone = make_grid(k)
        kind, C = choice[k]
        if C:
            alone.set_option("cluster_sweep", {1: 1, 2: 2, 3: 4}[kind])
            alone.set_option("cluster_size", C)
        o = dict(opts[k])
        s = alone.step(iters=18, **o)
        ns = grids[k].ns
        # identical up to the rounding of the device-evaluated CFL ramp, which 18 iterations
        # from the freestream (clipping decisions included) carry to ~1e-9 in FP64; the FP32
        # operator turns it into FP32 rounding differences
        tol = 1e-5 if o.get("precision", 0) == 1 else 1e-8
        assert rel(grids[k].get_state(), alone.get_state(), ns=ns) < tol, k
        assert stats[k]["iters_done"] == 6 and stats[k]["status_cell"] == -1
        assert abs(stats[k]["r_species"] - s["r_species"]) <= tol * 1e2 * s["r_species"]


def test_batch_tune_choices():
    grids = [make_grid(k) for k in range(len(CASES))]
    batch = P.Batch(grids)
    for prec in (0, 1):
        choice = batch.tune(precision=prec, trials=1)
        for k, (kind, C) in enumerate(choice):
            if k == 3:                        # 3D: no cluster sweep
                assert (kind, C) == (0, 0)
            elif kind == 3:                   # FP32 one-CTA-per-component kernel
                assert prec == 1 and C == 1
            else:
                assert kind in (1, 2) and C in (1, 2, 4, 8, 16)
                assert (grids[k].nj + C - 1) // C <= 32
    # tuning does not change the state
    Q = [g.get_state() for g in grids]
    batch.tune(precision=0, trials=1)
    for g, q in zip(grids, Q):
        assert np.array_equal(g.get_state(), q)


def test_batch_matches_oracle():
    """One batch case against the oracle after 10 iterations from the freestream."""
    k = 0
    nodes_fn, bc, mech, o = CASES[k]
    nodes = nodes_fn()
    fs = inputs.freestream(mech, T=300.0, p=500.0, mach=10.0)
    ref = oracle.OracleGrid(nodes, bc, mech)
    ref.set_boundary(fs, Tw=500.0)
    ref.set_state(ref.freestream_state())
    g = P.Grid(nodes, bc, mech)
    g.set_boundary(fs, Tw=500.0)
    g.set_state(ref.freestream_state())
    other = make_grid(2)
    batch = P.Batch([g, other])
    batch.tune(precision=0, trials=1)
    oo = dict(o, precision=0)
    batch.step([oo, CASES[2][3]], iters=10, iters_per_graph=5)
    ref.step(scheme=oo["scheme"], correction=oo["correction"], clip=1, cfl=oo["cfl"],
             cfl_start=oo["cfl_start"], ramp_iters=oo["ramp_iters"], iters=10)
    assert rel(g.get_state(), ref.get_state(), ns=ref.ns) < 1e-9


def test_batch_rejects_bad_arguments():
    grids = [make_grid(0), make_grid(2)]
    batch = P.Batch(grids)
    opts = [CASES[0][3], CASES[2][3]]
    with pytest.raises(P.CSError):
        batch.step(opts, iters=5, iters_per_graph=2)          # not a multiple
    with pytest.raises(P.CSError):
        batch.step([dict(opts[0], correction=3), opts[1]], iters=2)
    with pytest.raises(P.CSError):
        batch.tune(precision=7)
    bare = P.Grid(inputs.cylinder_half(8, 6), inputs.cylinder_half_bc(), inputs.MECH_AIR5)
    with pytest.raises(P.CSError):
        P.Batch([bare])                                        # no boundary conditions yet
