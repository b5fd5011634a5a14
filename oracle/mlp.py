"""Plain numpy restatement of the chemistry surrogate network and its training step.

TEST INFRASTRUCTURE: only tests/, the smoke check and the CPU-baseline leg of the benchmark
may import this module.  It shares no code with the CUDA path.

Network (a multilayer perceptron, no counterpart in the paper: it stands in for the Arrhenius
source and Jacobian-diagonal evaluation of Sec. 2.1 / Sec. 2.3.2 inside the implicit operator
only): 14 inputs -> 128 -> 128 -> 128 -> 22 outputs, SiLU activations (x / (1 + e^-x)) on the
hidden layers, linear output.  Precision model of the GPU path, emulated here step by step:
weights, inputs, hidden activations and back-propagated output gradients are rounded to
bfloat16 (round to nearest even) before every matrix product, products accumulate in FP32,
biases, pre-activations and the loss are FP32.  Inputs are padded from 14 to 16 columns and
outputs from 22 to 32 rows of W4 with zeros (the padded rows carry no target).

Loss: mean over samples and the 22 outputs of (y - t)^2.  Optimiser: Adam (beta1 0.9,
beta2 0.999, eps 1e-8) on FP32 master parameters.

`exact=True` switches every rounding off and computes in FP64: that variant is what the
finite-difference checks of the tests pin.
"""
import numpy as np

NIN, NH, NOUT = 14, 128, 22
KIN, NOUTP = 16, 32          # padded input width and output rows
SHAPES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)),
          ("W3", (NH, NH)), ("b3", (NH,)), ("W4", (NOUT, NH)), ("b4", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    out, k = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[k:k + n]).reshape(shp)
        k += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name]).ravel() for name, _ in SHAPES])


def bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float32."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(a.shape)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _mm(a, b, exact):
    """a @ b.T with bf16 operands and FP32 accumulation (or FP64 when exact)."""
    if exact:
        return np.asarray(a, np.float64) @ np.asarray(b, np.float64).T
    return bf16(a).astype(np.float32) @ bf16(b).astype(np.float32).T


def forward(flat, X, exact=False):
    """Outputs y [n, 22] and the cache for backward."""
    p = unpack(flat)
    dt = np.float64 if exact else np.float32
    X = np.asarray(X, dt)
    Z1 = (_mm(X, p["W1"], exact) + p["b1"]).astype(dt)
    H1 = silu(Z1).astype(dt)
    Z2 = (_mm(H1, p["W2"], exact) + p["b2"]).astype(dt)
    H2 = silu(Z2).astype(dt)
    Z3 = (_mm(H2, p["W3"], exact) + p["b3"]).astype(dt)
    H3 = silu(Z3).astype(dt)
    Y = (_mm(H3, p["W4"], exact) + p["b4"]).astype(dt)
    return Y, (X, Z1, H1, Z2, H2, Z3, H3)


def loss(Y, T):
    d = np.asarray(Y, np.float64) - np.asarray(T, np.float64)
    return float(np.mean(d * d))


def backward(flat, X, T, exact=False):
    """Loss and the gradient of the loss with respect to the flat parameter vector."""
    p = unpack(flat)
    dt = np.float64 if exact else np.float32
    Y, (X, Z1, H1, Z2, H2, Z3, H3) = forward(flat, X, exact)
    n = X.shape[0]
    dZ4 = (2.0 * (Y - np.asarray(T, dt)) / (n * NOUT)).astype(dt)
    g = {}
    g["W4"] = _mm(dZ4.T, H3.T, exact).astype(dt)          # dZ4^T H3
    g["b4"] = dZ4.sum(axis=0, dtype=dt)
    dH3 = _mm(dZ4, p["W4"].T, exact).astype(dt)           # dZ4 W4
    dZ3 = (dH3 * dsilu(Z3)).astype(dt)
    g["W3"] = _mm(dZ3.T, H2.T, exact).astype(dt)
    g["b3"] = dZ3.sum(axis=0, dtype=dt)
    dH2 = _mm(dZ3, p["W3"].T, exact).astype(dt)
    dZ2 = (dH2 * dsilu(Z2)).astype(dt)
    g["W2"] = _mm(dZ2.T, H1.T, exact).astype(dt)
    g["b2"] = dZ2.sum(axis=0, dtype=dt)
    dH1 = _mm(dZ2, p["W2"].T, exact).astype(dt)
    dZ1 = (dH1 * dsilu(Z1)).astype(dt)
    g["W1"] = _mm(dZ1.T, X.T, exact).astype(dt)
    g["b1"] = dZ1.sum(axis=0, dtype=dt)
    return loss(Y, T), pack(g)


def adam_step(flat, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t = 1 for the first); returns new parameters, m, v (FP32)."""
    m = (beta1 * m + (1.0 - beta1) * grad).astype(np.float32)
    v = (beta2 * v + (1.0 - beta2) * grad * grad).astype(np.float32)
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return (flat - lr * mh / (np.sqrt(vh) + eps)).astype(np.float32), m, v
