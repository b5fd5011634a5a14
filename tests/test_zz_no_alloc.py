"""The no-allocation residual-norm entry point (cs_residual_norms_static).

Some callers cannot allocate device memory: their application's memory pool already holds the
device, or they must not let cudaMalloc / cudaFree synchronise the device while a solver runs.
cs_residual_norms_static serves them from a static device scratch array.  These tests call it
through the C ABI and check

* its results against the norms cs_residual reports for the same residual, twice in a row
  (the array keeps the previous call's contents, which must not leak into the next result);
* a case at exactly the largest accepted cell count (the scratch array's last slot), against
  a float64 torch reduction of the same synthetic residual;
* that repeated calls leave the device's free memory unchanged (it allocates nothing).

The file is named so that pytest collects it last: the memory check reads the device's free
memory, which other tests' allocations would disturb if they ran in between, and a failure
here then stops a `-x` run only after every other test has run.  The largest accepted size is
read from include/cs.h, not restated."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import inputs
import oracle
import paper_2403_03440_gb300 as P

TOL = 1e-10
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _max_cells():
    src = open(os.path.join(ROOT, "include", "cs.h")).read()
    blocks = int(re.search(r"#define CS_NORMS_STATIC_MAX_BLOCKS (\d+)", src).group(1))
    per = int(re.search(r"#define CS_NORMS_STATIC_MAX_CELLS \(CS_NORMS_STATIC_MAX_BLOCKS \* (\d+)\)",
                        src).group(1))
    return blocks * per


MAX_CELLS = _max_cells()


def _fn():
    f = P.lib().cs_residual_norms_static
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p,
                  C.POINTER(C.c_double)]
    f.restype = C.c_int
    return f


def test_rejects_sizes_beyond_the_maximum():
    """Host-side argument checks run before any device work (no GPU needed)."""
    P.build()
    out = (C.c_double * 2)()
    dummy = C.c_void_p(16)          # never dereferenced: the size check comes first
    assert _fn()(dummy, dummy, MAX_CELLS + 1, 5, 2, None, out) == P.CS_ERR_ARG
    assert _fn()(dummy, dummy, 0, 5, 2, None, out) == P.CS_ERR_ARG
    assert _fn()(None, dummy, 100, 5, 2, None, out) == P.CS_ERR_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("mech,ni,nj", [(inputs.MECH_AIR5, 48, 32), (inputs.MECH_AIR11, 384, 256)])
def test_static_norms_match_cs_residual_twice(mech, ni, nj):
    import torch
    assert torch.cuda.is_available()
    P.build()
    nodes = inputs.cylinder_ogrid(ni, nj)
    fs = inputs.freestream(mech, T=300.0, p=500.0, mach=10.0)
    g = P.Grid(nodes, inputs.cylinder_bc(), mech)
    g.set_boundary(fs, Tw=500.0)
    f = _fn()
    for seed in (1, 2):                       # two calls in a row, different residuals
        pr = inputs.perturbed_primitive(mech, (nj, ni), seed=seed, ndim=2)
        Q = oracle.prim_to_cons_field(mech, 2, pr)
        g.set_state(Q)
        R = torch.empty((g.nq, g.ncell), dtype=torch.float64, device="cuda")
        _, norms = g.residual(R_out=R)
        V = torch.from_numpy(g.field("V")).cuda()
        out = (C.c_double * 2)()
        st = f(C.c_void_p(R.data_ptr()), C.c_void_p(V.data_ptr()), g.ncell, g.ns, 2, None, out)
        assert st == P.CS_OK
        assert abs(out[0] - norms[0]) <= TOL * abs(norms[0])
        assert abs(out[1] - norms[1]) <= TOL * abs(norms[1])


@pytest.mark.gpu
def test_largest_size_and_no_allocation():
    """ncell = the largest accepted count fills every slot of the scratch array; the result
    equals a float64 reduction, and repeated calls leave the free device memory unchanged."""
    import torch
    assert torch.cuda.is_available()
    P.build()
    ns, nd = 11, 2
    nq = ns + nd + 2
    gen = torch.Generator(device="cpu").manual_seed(3)
    R = (torch.rand((nq, MAX_CELLS), generator=gen, dtype=torch.float64) - 0.5).cuda()
    V = (torch.rand(MAX_CELLS, generator=gen, dtype=torch.float64) + 0.5).cuda()
    ref_s = float(torch.sqrt(((R[:ns] / V) ** 2).sum()))
    ref_e = float(torch.sqrt(((R[ns + nd] / V) ** 2).sum()))
    f = _fn()
    out = (C.c_double * 2)()
    assert f(C.c_void_p(R.data_ptr()), C.c_void_p(V.data_ptr()), MAX_CELLS, ns, nd, None, out) == P.CS_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in range(3):
        # a smaller call in between: the largest call afterwards must not see its leftovers
        assert f(C.c_void_p(R.data_ptr()), C.c_void_p(V.data_ptr()), 1000, ns, nd, None, out) == P.CS_OK
        assert f(C.c_void_p(R.data_ptr()), C.c_void_p(V.data_ptr()), MAX_CELLS, ns, nd, None, out) == P.CS_OK
        assert abs(out[0] - ref_s) <= TOL * ref_s, (k, out[0], ref_s)
        assert abs(out[1] - ref_e) <= TOL * ref_e, (k, out[1], ref_e)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
