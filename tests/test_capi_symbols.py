"""The C-ABI library builds for sm_103a, loads, exports every function include/cs.h declares,
and carries the same gas-model constants as the oracle (no GPU needed)."""
import os
import re

import numpy as np

import oracle
import paper_2403_03440_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cs_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    P.build()
    L = P.lib()
    names = declared_functions()
    assert "cs_lusgs_split" in names and "cs_step" in names
    for n in names:
        assert hasattr(L, n), n
    assert sorted(P.EXPORTS) == names


def test_gas_constants_match_oracle():
    P.build()
    for mech in (0, 1, 2):
        a, b = P.gas_info(mech), oracle.gas_info(mech)
        assert a["ns"] == b["ns"] and a["nr"] == b["nr"] and a["ntemp"] == b["ntemp"]
        np.testing.assert_allclose(a["M"], b["M"], rtol=1e-15, atol=0)
        np.testing.assert_allclose(a["hf"], b["hf"], rtol=1e-15, atol=0)


def test_invalid_descriptors_rejected_without_gpu_work():
    """Argument checks happen on the host before any device call."""
    import ctypes as C
    P.build()
    d = P.cs_grid_desc()
    d.ndim, d.ni, d.nj, d.nk = 4, 8, 8, 1
    h = C.c_void_p()
    nodes = np.zeros(2 * 9 * 9)
    assert P.lib().cs_grid_create(C.byref(d), C.c_void_p(nodes.ctypes.data), None, C.byref(h)) == P.CS_ERR_ARG
    d.ndim = 2
    for k in range(6):
        d.bc[k] = 0
    d.bc[0], d.bc[1] = 0, 2                # periodic on one side only
    assert P.lib().cs_grid_create(C.byref(d), C.c_void_p(nodes.ctypes.data), None, C.byref(h)) == P.CS_ERR_ARG
