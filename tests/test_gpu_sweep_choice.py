"""Kernel choice of the 2D split sweep must not depend on which other grids the process made.

The point-to-point sweep over assembled couplings needs more than 48 KiB of dynamic shared
memory on grids with ni + nj - 1 > 682 (FP64).  The opt-in limit is a property of the kernel,
shared by every grid, so a smaller grid probing the kernel after a larger one must not lower
it: the larger grid would then fail to launch the kernel and fall back to another sweep.
These tests alternate iterations of two grids of different sizes and check, through
cs_sweep_info, that both keep the chosen kernel (5: point to point between CTAs, the default),
and that the large grid's increments are those of the same grid stepped alone."""
import numpy as np
import pytest

import inputs
import paper_2403_03440_gb300 as P

pytestmark = pytest.mark.gpu

P2P = 5


def _grid(ni, nj, mech, kind=None):
    nodes = inputs.cylinder_half(ni, nj, dr1=5e-5 * 48 / ni)
    g = P.Grid(nodes, inputs.cylinder_half_bc(), mech)
    if kind is not None:
        g.set_option("cluster_sweep", kind)
    g.set_boundary(inputs.freestream(mech, T=300.0, p=500.0, mach=10.0), Tw=500.0)
    g.init_freestream()
    return g


@pytest.mark.parametrize("kind", [P2P])
@pytest.mark.parametrize("precision", [0, 1])
def test_alternating_grids_keep_the_point_to_point_sweep(precision, kind):
    import torch
    assert torch.cuda.is_available()
    P.build()
    mech = inputs.MECH_AIR5
    # FP64 ring 72 B per hyperplane: 640 + 128 - 1 = 767 planes -> 55 KiB (> 48 KiB);
    # FP32 ring 40 B per hyperplane: 1100 + 160 - 1 = 1259 planes -> 49 KiB
    ni, nj = (640, 128) if precision == 0 else (1100, 160)
    big, small = _grid(ni, nj, mech, kind), _grid(48, 32, mech, kind)
    kw = dict(scheme=0, correction=1, clip=1, cfl=2.0, cfl_start=0.5, ramp_iters=10,
              precision=precision, iters=1)
    big.step(**kw)
    assert big.sweep_info()[0] == kind
    small.step(**kw)                     # probes the kernel with a small ring
    assert small.sweep_info()[0] == kind
    for _ in range(2):
        big.step(**kw)
        assert big.sweep_info()[0] == kind, big.sweep_info()
        small.step(**kw)
        assert small.sweep_info()[0] == kind
    # the big grid's iterates equal those of the same grid stepped alone
    alone = _grid(ni, nj, mech, kind)
    for _ in range(3):
        alone.step(**kw)
    a, b = big.get_state(), alone.get_state()
    scale = np.abs(b).max(axis=1, keepdims=True)
    assert np.max(np.abs(a - b) / scale) <= 1e-13
