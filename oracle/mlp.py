"""FP64 reference of the reaction-step surrogate network -- TEST INFRASTRUCTURE.

The surrogate replaces the 0D reaction step of the Strang split step (the
Heun substeps of the HH model, eq:heun and sec:subcelullar_model) by a small
multilayer perceptron.  The thesis has no learned component on this path; the
network shape (5 -> 128 -> 128 -> 4, SiLU) is the one the build targets.

Definition (plain, written out):
    x  in R^5                       normalised inputs (u, m, h, n, stimulus)
    z1 = W1 x + b1,  a1 = SiLU(z1)  W1: 128 x 5
    z2 = W2 a1 + b2, a2 = SiLU(z2)  W2: 128 x 128
    o  = W3 a2 + b3                 W3: 4 x 128
    SiLU(z) = z / (1 + exp(-z))
    loss = mean over samples and the 4 outputs of (o - target)^2
Parameter vector theta = [W1 (row-major), b1, W2, b2, W3, b3].

With ``quantize``, the weights and the inputs to each matrix product are
rounded to bfloat16 (round to nearest, ties to even), as the tensor-core
kernels do; gradients then treat the rounding as the identity
(straight-through), which is what the GPU training kernels implement.

Only tests/ may import this module.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 5, 128, 4
SIZES = [(N_HID, N_IN), (N_HID,), (N_HID, N_HID), (N_HID,), (N_OUT, N_HID), (N_OUT,)]
N_PARAMS = sum(int(np.prod(s)) for s in SIZES)


def unpack(theta):
    out, k = [], 0
    for s in SIZES:
        n = int(np.prod(s))
        out.append(np.asarray(theta[k:k + n], dtype=np.float64).reshape(s))
        k += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 keeps the top 16 bits of an IEEE float32; rounding adds half of
    the dropped part's range plus the tie-breaking bit, then truncates."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    rounded = ((b + 0x7FFF + lsb) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if np.any(nan):
        out = np.where(nan, np.nan, out)
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, x, quantize=False):
    """Returns (o, cache) for inputs x of shape (B, 5)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    q = bf16_round if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    xq = q(x)
    W1q, W2q, W3q = q(W1), q(W2), q(W3)
    z1 = xq @ W1q.T + b1
    a1 = silu(z1)
    a1q = q(a1)
    z2 = a1q @ W2q.T + b2
    a2 = silu(z2)
    a2q = q(a2)
    o = a2q @ W3q.T + b3
    return o, dict(xq=xq, W1q=W1q, W2q=W2q, W3q=W3q, z1=z1, a1q=a1q, z2=z2, a2q=a2q)


def loss(theta, x, target, quantize=False):
    o, _ = forward(theta, x, quantize)
    return float(np.mean((o - target) ** 2))


def backward(theta, x, target, quantize=False):
    """Analytic gradient of `loss` (straight-through for the bf16 rounding)."""
    o, c = forward(theta, x, quantize)
    B = x.shape[0]
    do = 2.0 * (o - target) / (B * N_OUT)
    gW3 = do.T @ c["a2q"]
    gb3 = do.sum(axis=0)
    da2 = do @ c["W3q"]
    dz2 = da2 * silu_grad(c["z2"])
    gW2 = dz2.T @ c["a1q"]
    gb2 = dz2.sum(axis=0)
    da1 = dz2 @ c["W2q"]
    dz1 = da1 * silu_grad(c["z1"])
    gW1 = dz1.T @ c["xq"]
    gb1 = dz1.sum(axis=0)
    return pack([gW1, gb1, gW2, gb2, gW3, gb3]), float(np.mean((o - target) ** 2))


def finite_difference_grad(theta, x, target, indices, eps=1e-6):
    """Central differences of the unquantised loss at the given parameter indices."""
    g = np.zeros(len(indices))
    for i, k in enumerate(indices):
        tp = np.array(theta, dtype=np.float64)
        tm = np.array(theta, dtype=np.float64)
        tp[k] += eps
        tm[k] -= eps
        g[i] = (loss(tp, x, target) - loss(tm, x, target)) / (2 * eps)
    return g


def adam_step(theta, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) with bias correction."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def weight_average(avg, theta, decay):
    """Exponential moving average of the weights after a step (Polyak
    averaging, Polyak & Juditsky 1992, in its exponential form)."""
    return decay * avg + (1 - decay) * theta


def init_params(seed, scale=1.0):
    """He-style uniform initialisation (for tests and as the training start)."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in SIZES:
        if len(s) == 2:
            lim = scale * np.sqrt(6.0 / s[1])
            parts.append(rng.uniform(-lim, lim, size=s))
        else:
            parts.append(np.zeros(s))
    return pack(parts)
