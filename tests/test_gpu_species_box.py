"""The species-count scaling test's implicit step on the CUDA path (cs_species_box_*: any ns,
split and coupled operators) against the numpy oracle (oracle/species_box.py), element by
element: boxes of several shapes (ragged, one cell thick), ns from 1 to 300 (species groups
with a ragged tail, a coupled block far above the 2D/3D solver's), and the full 10 x 10 x 10
box of the test at ns = 64.  Both sides compute in FP64 with the same algorithm; the
tolerance allows rounding-order differences (fused multiply-adds, reduction order)."""
import numpy as np
import pytest

import inputs
from oracle import species_box as sb
import paper_2403_03440_gb300 as P

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    P.build()
    P.lib()
    yield


def rel_rows(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1e-300)))


def run_pair(ns, n, scheme, seed=0, cfl=5.0):
    import torch
    case = inputs.species_box(ns, seed=seed, n=n)
    box = sb.Box(case)
    gbox = P.SpeciesBox(case)
    rhs = inputs.species_box_rhs(ns, box.N, seed=seed + 1)
    want = sb.split_operator(box, rhs, cfl) if scheme == 0 else sb.coupled_operator(box, rhs, cfl)
    got = gbox.step(scheme, cfl, torch.from_numpy(rhs).cuda()).cpu().numpy()
    return box, gbox, got, want


@pytest.mark.parametrize("ns,n", [(1, (4, 3, 3)), (5, (7, 5, 3)), (33, (5, 4, 3)), (16, (6, 1, 4)),
                                  (3, (12, 12, 12))])
@pytest.mark.parametrize("scheme", [0, 1])
def test_step_matches_oracle(ns, n, scheme):
    box, gbox, got, want = run_pair(ns, n, scheme)
    assert got.shape == want.shape
    assert rel_rows(got, want) < TOL


def test_state_matches_oracle():
    case = inputs.species_box(20, seed=4, n=(3, 4, 5))
    box = sb.Box(case)
    Q = P.SpeciesBox(case).state().cpu().numpy()
    assert rel_rows(Q, np.repeat(box.q[:, None], box.N, axis=1)) < 1e-14


def test_many_species_coupled_block():
    """ns = 300: coupled blocks of 304 x 304 per cell, species spread over ten CTAs."""
    for scheme in (0, 1):
        _, _, got, want = run_pair(300, (3, 3, 2), scheme, seed=7)
        assert rel_rows(got, want) < TOL


def test_full_box_of_the_test():
    """The 10 x 10 x 10 box of the test at ns = 64, both operators."""
    for scheme in (0, 1):
        _, _, got, want = run_pair(64, (10, 10, 10), scheme, seed=3)
        assert rel_rows(got, want) < TOL


def test_timing_and_errors():
    import torch
    case = inputs.species_box(16, seed=0)
    g = P.SpeciesBox(case)
    rhs = torch.from_numpy(inputs.species_box_rhs(16, g.ncell)).cuda()
    flush = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    for scheme in (0, 1):
        g.step(scheme, 5.0, rhs)
        assert g.time(scheme, 5.0, rhs, 3) > 0.0
        assert g.time(scheme, 5.0, rhs, 2, flush=flush) > 0.0
    with pytest.raises(P.CSError):
        g.step(2, 5.0, rhs)                            # no such scheme
    with pytest.raises(P.CSError):
        g.step(0, -1.0, rhs)                           # CFL
    with pytest.raises(P.CSError):
        g.step(0, 5.0, rhs.cpu())                      # host pointer
    bad = dict(case, M=-case["M"])
    with pytest.raises(P.CSError):
        P.SpeciesBox(bad)
