"""The surrogate network on the tensor cores (tcgen05 GEMMs in bfloat16 with FP32 accumulation)
against its numpy oracle (oracle/mlp.py, which rounds to bfloat16 at the same points):
forward outputs, loss, back-propagated gradients and Adam steps."""
import numpy as np
import pytest

import inputs
import paper_2403_03440_gb300 as P
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    P.build()
    P.lib()
    yield


def data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, mlp.NIN)).astype(np.float32)
    # smooth targets of the inputs
    T = np.tanh(X @ rng.normal(size=(mlp.NIN, mlp.NOUT)) / 3.0).astype(np.float32)
    return X, T


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


# inference runs the fused persistent kernel: 40100 rows are 314 tiles, more than the grid's
# CTAs, so CTAs loop over tiles and the last tile is ragged
@pytest.mark.parametrize("n", [1, 128, 200, 1000, 40100])
def test_forward_matches_oracle(n):
    import torch
    p = inputs.mlp_init(2)
    X, _ = data(n, 1)
    net = P.MLP(p, max_batch=max(n, 1024))
    Y = torch.empty((n, mlp.NOUT), dtype=torch.float32, device="cuda")
    net.forward(dev(X), Y)
    Yo = mlp.forward(p, X)[0]
    y = Y.cpu().numpy()
    assert rel_l2(y, Yo) < 5e-3
    assert np.max(np.abs(y - Yo)) < 2e-2 * np.max(np.abs(Yo))


@pytest.mark.parametrize("n", [128, 300])
def test_gradients_match_oracle(n):
    p = inputs.mlp_init(3)
    X, T = data(n, 2)
    net = P.MLP(p, max_batch=512)
    loss, g = net.grad(dev(X), dev(T))
    lo, go = mlp.backward(p, X, T)
    assert abs(loss - lo) < 1e-3 * lo
    blocks = mlp.unpack(np.arange(mlp.NPARAM))
    for name, idx in blocks.items():
        idx = idx.ravel()
        assert rel_l2(g[idx], go[idx]) < 1e-2, name      # measured: <= 4e-5


def test_training_follows_oracle_and_reduces_loss():
    p = inputs.mlp_init(4)
    X, T = data(512, 3)
    net = P.MLP(p, max_batch=512)
    Xd, Td = dev(X), dev(T)
    po, m, v = p.copy(), np.zeros_like(p), np.zeros_like(p)
    losses = []
    for t in range(1, 6):
        losses.append(net.train_step(Xd, Td, 1e-3))
        _, go = mlp.backward(po, X, T)
        po, m, v = mlp.adam_step(po, go, m, v, t, 1e-3)
    # after 5 Adam steps (each moves a parameter by at most ~lr) the parameters agree with the
    # oracle's on average to a small fraction of one step; where a gradient is near zero the
    # bfloat16 noise can flip a step, hence the looser bound on the largest difference
    d = np.abs(net.params() - po)
    assert np.mean(d) < 2e-4 and np.max(d) < 1.1e-2
    for _ in range(300):
        losses.append(net.train_step(Xd, Td, 3e-3))
    assert losses[-1] < 0.1 * losses[0]


def test_forward_after_training_uses_updated_weights():
    """Inference right after train_step sees the new bfloat16 weights (the step is complete
    when it returns), and agrees with the oracle evaluated at the returned parameters."""
    import torch
    X, T = data(384, 5)
    net = P.MLP(inputs.mlp_init(6), max_batch=384)
    Xd, Td = dev(X), dev(T)
    for _ in range(20):
        net.train_step(Xd, Td, 3e-3)
    Y = torch.empty((384, mlp.NOUT), dtype=torch.float32, device="cuda")
    net.forward(Xd, Y)
    Yo = mlp.forward(net.params(), X)[0]
    assert rel_l2(Y.cpu().numpy(), Yo) < 5e-3


def test_rejects_bad_batch():
    net = P.MLP(inputs.mlp_init(0), max_batch=64)
    X, T = data(65, 0)
    with pytest.raises(P.CSError):
        net.grad(dev(X), dev(T))
