"""Pins of the surrogate network's oracle (oracle/mlp.py): bfloat16 rounding, the SiLU pair,
back-propagation against central differences, and Adam's first step in closed form."""
import numpy as np

import inputs
from oracle import mlp


def test_bf16_rounding_ties_to_even():
    one = np.float32(1.0)
    ulp = 2.0 ** -7                      # bf16 spacing at 1
    vals = np.array([1.0, 1.0 + ulp / 2, 1.0 + 1.5 * ulp, 1.0 + 0.75 * ulp, -3.0, 1e-3],
                    dtype=np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2 * ulp, 1.0 + ulp, -3.0], dtype=np.float32)
    got = mlp.bf16(vals)
    assert np.array_equal(got[:5], want)
    # the low 16 bits of every result are zero and the error is within half a spacing
    assert np.all(got.view(np.uint32) & 0xFFFF == 0)
    assert abs(got[5] - vals[5]) <= 2.0 ** -9 * abs(vals[5])
    assert one == 1.0


def test_silu_pair():
    z = np.linspace(-8, 8, 33)
    assert mlp.silu(np.array([0.0]))[0] == 0.0
    assert mlp.dsilu(np.array([0.0]))[0] == 0.5
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.dsilu(z))) < 1e-8
    # silu(z) -> z for large z, -> 0 for very negative z
    assert abs(mlp.silu(np.array([30.0]))[0] - 30.0) < 1e-10


def test_backward_matches_central_differences():
    rng = np.random.default_rng(3)
    p = inputs.mlp_init(5).astype(np.float64)
    X = np.zeros((7, mlp.KIN))
    X[:, :mlp.NIN] = rng.normal(size=(7, mlp.NIN))
    T = rng.normal(size=(7, mlp.NOUT))
    # pad W1 to the 16-column input and W4 to nothing: the oracle takes the real shapes
    L0, g = mlp.backward(p, X[:, :mlp.NIN], T, exact=True)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    for k in idx:
        h = 1e-6 * max(1.0, abs(p[k]))
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (mlp.loss(mlp.forward(pp, X[:, :mlp.NIN], exact=True)[0], T) -
              mlp.loss(mlp.forward(pm, X[:, :mlp.NIN], exact=True)[0], T)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(g).max(), 1e-12), (k, fd, g[k])


def test_bf16_forward_close_to_exact():
    rng = np.random.default_rng(4)
    p = inputs.mlp_init(1)
    X = rng.normal(size=(64, mlp.NIN)).astype(np.float32)
    ye = mlp.forward(p, X, exact=True)[0]
    yb = mlp.forward(p, X)[0]
    assert np.max(np.abs(yb - ye)) < 3e-2 * np.max(np.abs(ye))


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(6)
    p = rng.normal(size=50).astype(np.float32)
    g = rng.normal(size=50).astype(np.float32)
    lr = 1e-3
    p1, m, v = mlp.adam_step(p, g, np.zeros(50, np.float32), np.zeros(50, np.float32), 1, lr)
    # first step: m_hat = g, v_hat = g^2, so the step is -lr g / (|g| + eps)
    want = p - lr * g / (np.abs(g) + 1e-8)
    assert np.max(np.abs(p1 - want)) < 1e-6 * lr
