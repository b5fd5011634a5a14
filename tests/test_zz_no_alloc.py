"""The no-allocation residual-norm entry point (cs_residual_norms_static).

Some callers cannot allocate device memory (their application's pool already holds the
device, or they must not let cudaMalloc/cudaFree synchronise the device while a solver runs).
cs_residual_norms_static serves them from a static device scratch array.  These tests call it
through the C ABI and check it against the norms cs_residual reports for the same residual,
twice in a row (the array keeps the previous call's contents, which must not leak into the
next result).  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import inputs
import oracle
import paper_2403_03440_gb300 as P

TOL = 1e-10
MAX_CELLS = 16384 * 256


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
