"""Plain FP64 reference of the atom-pair MLP used by the learned SCF guess
(test infrastructure only): three dense layers with SiLU activations,
masked mean-squared-error loss, analytic gradients.  Parameter vector layout
W1[H][nin], b1[H], W2[H][H], b2[H], W3[nout][H], b3[nout]."""
from __future__ import annotations

import numpy as np


def unpack(p, nin, H, nout):
    o = 0
    out = []
    for shape in ((H, nin), (H,), (H, H), (H,), (nout, H), (nout,)):
        n = int(np.prod(shape))
        out.append(np.asarray(p[o:o + n], dtype=np.float64).reshape(shape))
        o += n
    return out


def bf16_round(x):
    """Round float32 values to bfloat16 (round to nearest even), as floats."""
    a = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (a >> 16) & 1
    r = ((a + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, X, nin, H, nout, weights_bf16=True):
    W1, b1, W2, b2, W3, b3 = unpack(p, nin, H, nout)
    if weights_bf16:
        W1, W2, W3 = (bf16_round(w).astype(np.float64) for w in (W1, W2, W3))
    z1 = X @ W1.T + b1
    a1 = silu(z1)
    z2 = a1 @ W2.T + b2
    a2 = silu(z2)
    y = a2 @ W3.T + b3
    return y, (z1, a1, z2, a2, W1, W2, W3)


def loss_and_grad(p, X, T, mask, norm, nin, H, nout, weights_bf16=True):
    X = np.asarray(X, dtype=np.float64)
    y, (z1, a1, z2, a2, W1, W2, W3) = forward(p, X, nin, H, nout, weights_bf16)
    m = np.ones_like(y) if mask is None else np.asarray(mask, dtype=np.float64)
    r = (y - T) * m
    loss = float(np.sum(r * (y - T)) / norm)
    dy = 2.0 * r / norm
    gW3 = dy.T @ a2
    gb3 = dy.sum(0)
    d2 = (dy @ W3) * dsilu(z2)
    gW2 = d2.T @ a1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * dsilu(z1)
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g
