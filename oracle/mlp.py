"""FP64 reference of the learned warm start's network (test infrastructure, see ``oracle``).

Not part of the paper: the network is a systems pattern that predicts an initial guess for the
coarse Poisson solve of Eq. 21. It maps the coarse right-hand side b (n entries) to the pressure:

    s = ||b||_2,  x = b / s
    z1 = W1 x + b1,   h1 = gelu(z1)          (hidden H)
    z2 = W2 h1 + b2,  h2 = gelu(z2)          (hidden H)
    y  = W3 h2 + b3                           (n outputs)
    p  = s * y,  with pressure-held entries set to 0

(a linear solve is homogeneous of degree one in b, so the network works on the unit-norm
right-hand side). gelu is the tanh form of Hendrycks & Gimpel (2016):
gelu(z) = z/2 (1 + tanh(c (z + a z^3))), c = sqrt(2/pi), a = 0.044715.
Training minimises L = 1/(B n) sum_b sum_j m_j (y_bj - t_bj)^2 with t = p_true / s and m the
mask of unconstrained entries, by Adam (Kingma & Ba 2015) on FP32-style master weights.

``bf16=True`` rounds to bfloat16 (round to nearest even) at the points where the GPU stores
bfloat16: x, the weights used by the products, h1, h2 and the back-propagated dz; everything else
is FP64. Weights are stored row-major as W[out, in].
"""
from __future__ import annotations

import math

import numpy as np

GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounding = np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))
    r = ((u + rounding) >> np.uint64(16)) << np.uint64(16)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))


def gelu_grad(z):
    u = GELU_C * (z + GELU_A * z ** 3)
    t = np.tanh(u)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * z * z)


def _r(x, on):
    return bf16_round(x) if on else x


def forward(params, b, mask=None, bf16=False):
    """Batch forward. ``b``: [B, n] right-hand sides. Returns (p [B, n], cache)."""
    W1, b1, W2, b2, W3, b3 = params
    s = np.linalg.norm(b, axis=1, keepdims=True)
    s = np.where(s > 0.0, s, 1.0)
    x = _r(b / s, bf16)
    z1 = x @ _r(W1, bf16).T + b1
    h1 = _r(gelu(z1), bf16)
    z2 = h1 @ _r(W2, bf16).T + b2
    h2 = _r(gelu(z2), bf16)
    y = h2 @ _r(W3, bf16).T + b3
    p = s * y
    if mask is not None:
        p = p * mask
    return p, dict(s=s, x=x, z1=z1, h1=h1, z2=z2, h2=h2, y=y)


def loss_and_grads(params, b, p_true, mask, bf16=False):
    """Loss L and gradients (dW1, db1, dW2, db2, dW3, db3) for one batch."""
    W1, b1, W2, b2, W3, b3 = params
    _, c = forward(params, b, None, bf16)
    Bn = b.shape[0] * float(mask.sum())
    t = p_true / c["s"]
    diff = (c["y"] - t) * mask
    L = float((diff ** 2).sum() / Bn)
    dy = 2.0 * diff / Bn
    db3 = dy.sum(axis=0)
    dyr = _r(dy, bf16)
    dW3 = dyr.T @ c["h2"]
    dh2 = dyr @ _r(W3, bf16)
    dz2 = dh2 * gelu_grad(c["z2"])
    db2 = dz2.sum(axis=0)
    dz2r = _r(dz2, bf16)
    dW2 = dz2r.T @ c["h1"]
    dh1 = dz2r @ _r(W2, bf16)
    dz1 = dh1 * gelu_grad(c["z1"])
    db1 = dz1.sum(axis=0)
    dW1 = _r(dz1, bf16).T @ c["x"]
    return L, (dW1, db1, dW2, db2, dW3, db3)


def adam_step(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), returning new params, m, v."""
    out_p, out_m, out_v = [], [], []
    bc1 = 1.0 - beta1 ** step
    bc2 = 1.0 - beta2 ** step
    for P, G, M, V in zip(params, grads, m, v):
        M = beta1 * M + (1.0 - beta1) * G
        V = beta2 * V + (1.0 - beta2) * G * G
        P = P - lr * (M / bc1) / (np.sqrt(V / bc2) + eps)
        out_p.append(P)
        out_m.append(M)
        out_v.append(V)
    return out_p, out_m, out_v
