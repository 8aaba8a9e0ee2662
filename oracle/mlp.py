"""FP64 reference of the delayed-acceptance surrogate network.

TEST INFRASTRUCTURE ONLY: the plain numpy forward and backward pass the GPU
training kernels are checked against.  Only the tests and the benchmark's
CPU-baseline leg may import it.

The network (the learned first stage of the delayed-acceptance form of the
local rule, Sec. III B 2 with Christen and Fox's two-stage test): ten raw
environment counts c (own B counts in shells 1-5, then the first-shell
neighbours' summed B counts in shells 1-5) are scaled to x = c / max_c, then

    z1 = W1 x + b1,  h1 = SiLU(z1),  z2 = W2 h1 + b2,  h2 = SiLU(z2),
    g  = w3 . h2 + b3,               SiLU(z) = z / (1 + exp(-z)),

and g predicts E(site = B) - E(site = A).  Training minimises the mean
squared error over a batch.  Parameter vector layout: W1[64][10], b1[64],
W2[64][64], b2[64], w3[64], b3.

``rnd`` (identity when None) is applied to every tensor-core operand: the
scaled inputs, W1, W2, h1 as the input of layer 2, and the deltas entering
the weight-gradient and back-propagation products.  Passing a rounding to
BF16 there models the precision the GPU kernels use; the arithmetic itself
stays FP64.
"""
from __future__ import annotations

import numpy as np

IN = 10
H = 64
NPARAM = H * IN + H + H * H + H + H + 1
DESC_MAX = np.array([8, 6, 12, 24, 8, 56, 48, 96, 192, 64], dtype=np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    assert p.shape == (NPARAM,)
    o = 0
    W1 = p[o:o + H * IN].reshape(H, IN); o += H * IN
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _id(a):
    return a


def forward(p, counts, rnd=None):
    """Predictions g for a batch of raw counts (n, 10); returns (g, cache)."""
    r = rnd or _id
    W1, b1, W2, b2, w3, b3 = unpack(p)
    x = r(np.asarray(counts, dtype=np.float64) / DESC_MAX)
    z1 = x @ r(W1).T + b1
    h1 = silu(z1)
    z2 = r(h1) @ r(W2).T + b2
    h2 = silu(z2)
    g = h2 @ w3 + b3
    return g, (x, z1, h1, z2, h2)


def loss_and_grad(p, counts, target, rnd=None):
    """Mean squared error over the batch and its gradient (same layout as p)."""
    r = rnd or _id
    W1, b1, W2, b2, w3, b3 = unpack(p)
    g, (x, z1, h1, z2, h2) = forward(p, counts, rnd)
    n = g.shape[0]
    e = g - np.asarray(target, dtype=np.float64)
    loss = float((e * e).sum() / n)
    d3 = 2.0 * e / n                              # dL/dg
    gw3 = h2.T @ d3
    gb3 = d3.sum()
    d2 = d3[:, None] * w3[None, :] * dsilu(z2)    # dL/dz2
    gW2 = r(d2).T @ r(h1)
    gb2 = d2.sum(axis=0)
    d1 = (r(d2) @ r(W2)) * dsilu(z1)              # dL/dz1
    gW1 = r(d1).T @ x
    gb1 = d1.sum(axis=0)
    return loss, pack(gW1, gb1, gW2, gb2, gw3, gb3)


def round_bf16(a):
    """Round FP64 values to the nearest BF16 value (ties to even), via FP32."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
