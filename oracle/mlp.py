"""FP64 reference of the learned proposal network (test infrastructure only).

Plain numpy restatement of the network and losses the CUDA kernels train:
inputs normalised by (x - mean) / scale, layers n_in -> 64 -> 64 -> 3 with
SiLU, outputs (log h0, log sigma, log cost) de-normalised by
y * scale + mean; loss = mean over rows of
(p0 - t0)^2 + pinball_0.9(t1 - p1) + (p2 - t2)^2 on normalised targets,
where a NaN target contributes no term (rows logged at spectral-radius
points carry a sigma target only).
The parameter vector layout: W1 [64][n_in], b1 [64], W2 [64][64], b2 [64],
W3 [3][64], b3 [3]; the normalisation block x_mean, x_scale, x_min, x_max
[33 each], y_mean, y_scale [3 each].
"""
from __future__ import annotations

import numpy as np

H, MAX_IN, OUT, TAU = 64, 33, 3, 0.9
NORM_SIZE = 4 * MAX_IN + 2 * OUT


def num_params(n_in):
    return H * n_in + H + H * H + H + OUT * H + OUT


def unpack(params, n_in):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * n_in].reshape(H, n_in); o += H * n_in
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + OUT * H].reshape(OUT, H); o += OUT * H
    b3 = p[o:o + OUT]; o += OUT
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def unpack_norm(norm, n_in):
    q = np.asarray(norm, dtype=np.float64)
    xm, xs = q[0:n_in], q[MAX_IN:MAX_IN + n_in]
    ym, ys = q[4 * MAX_IN:4 * MAX_IN + OUT], q[4 * MAX_IN + OUT:4 * MAX_IN + 2 * OUT]
    return xm, xs, ym, ys


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, norm, X, bf16_operands: bool = False):
    """De-normalised outputs (log h0, log sigma, log cost) for raw feature rows X.

    bf16_operands: round the normalised inputs and both layers' activations
    to BF16 before each product, as a tensor-core evaluation with BF16
    operands does (the weights are rounded by the caller)."""
    n_in = X.shape[1]
    W1, b1, W2, b2, W3, b3 = unpack(params, n_in)
    xm, xs, ym, ys = unpack_norm(norm, n_in)
    rnd = bf16_round if bf16_operands else (lambda v: v)
    x = rnd((np.asarray(X, np.float64) - xm) / xs)
    a1 = rnd(silu(x @ W1.T + b1))
    a2 = rnd(silu(a1 @ W2.T + b2))
    return (a2 @ W3.T + b3) * ys + ym


def loss_and_grad(params, norm, X, Y):
    """Mean loss over the rows and its gradient (same layout as params)."""
    n_in = X.shape[1]
    W1, b1, W2, b2, W3, b3 = unpack(params, n_in)
    xm, xs, ym, ys = unpack_norm(norm, n_in)
    x = (np.asarray(X, np.float64) - xm) / xs
    t = (np.asarray(Y, np.float64) - ym) / ys
    z1 = x @ W1.T + b1
    a1 = silu(z1)
    z2 = a1 @ W2.T + b2
    a2 = silu(z2)
    p = a2 @ W3.T + b3
    n = x.shape[0]
    have = np.isfinite(t)  # a NaN target is no target
    t = np.where(have, t, 0.0)
    r0 = p[:, 0] - t[:, 0]
    r1 = t[:, 1] - p[:, 1]
    r2 = p[:, 2] - t[:, 2]
    terms = np.stack([r0 ** 2, np.where(r1 > 0, TAU * r1, (TAU - 1.0) * r1), r2 ** 2], axis=1)
    loss = np.sum(np.where(have, terms, 0.0)) / n
    g = np.stack([2.0 * r0, np.where(r1 > 0, -TAU, 1.0 - TAU), 2.0 * r2], axis=1)
    g = np.where(have, g, 0.0) / n
    gW3 = g.T @ a2
    gb3 = g.sum(axis=0)
    d2 = (g @ W3) * silu_grad(z2)
    gW2 = d2.T @ a1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * silu_grad(z1)
    gW1 = d1.T @ x
    gb1 = d1.sum(axis=0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, grad


def bf16_round(x):
    """Round float32 values to bfloat16 (nearest, ties to even), as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
