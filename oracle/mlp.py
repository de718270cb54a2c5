"""Rank-proposer MLP -- TEST INFRASTRUCTURE ONLY (oracle).

Not from the paper: the learned rank proposer of the adaptive (ps2) runs. A
plain FP64 restatement of what the GPU kernels compute, written from the
textbook definitions:

    h1 = relu(W1 x + b1)          (24 -> 64)
    h2 = relu(W2 h1 + b2)         (64 -> 64)
    z  = W3 h2 + b3               (64 -> 13 logits, rank change -4..+8)
    L  = mean_b [ logsumexp(z_b) - z_b[y_b] ]      (softmax cross-entropy)

Backward by the chain rule (dL/dz = (softmax(z) - onehot(y)) / B, relu'(a) =
[a > 0]); Adam (Kingma & Ba 2015) with bias correction. Parameters are packed
in one vector in the order W1, b1, W2, b2, W3, b3, matrices row-major
(output index first).

Pinned by tests/test_oracle_mlp.py: central finite differences of L against
every parameter block, and the softmax cross-entropy gradient identity.
"""
from __future__ import annotations

from typing import Dict, Tuple

import numpy as np

N_IN, N_H, N_OUT = 24, 64, 13
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> Dict[str, np.ndarray]:
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def init_params(seed: int) -> np.ndarray:
    """He-style initial weights (normal, std sqrt(2/fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in SHAPES:
        if name.startswith("W"):
            parts.append(rng.normal(0.0, np.sqrt(2.0 / shape[1]), size=shape).reshape(-1))
        else:
            parts.append(np.zeros(shape).reshape(-1))
    return np.concatenate(parts)


def forward(theta: np.ndarray, x: np.ndarray):
    p = unpack(theta)
    a1 = x @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["W3"].T + p["b3"]
    return z, (a1, h1, a2, h2)


def loss(theta: np.ndarray, x: np.ndarray, y: np.ndarray) -> float:
    z, _ = forward(theta, x)
    zmax = z.max(axis=1, keepdims=True)
    lse = zmax[:, 0] + np.log(np.exp(z - zmax).sum(axis=1))
    return float(np.mean(lse - z[np.arange(len(y)), y]))


def grad(theta: np.ndarray, x: np.ndarray, y: np.ndarray) -> Tuple[float, np.ndarray]:
    """Loss and dL/dtheta by backpropagation."""
    p = unpack(theta)
    z, (a1, h1, a2, h2) = forward(theta, x)
    B = len(y)
    zmax = z.max(axis=1, keepdims=True)
    e = np.exp(z - zmax)
    sm = e / e.sum(axis=1, keepdims=True)
    L = float(np.mean(np.log(e.sum(axis=1)) + zmax[:, 0] - z[np.arange(B), y]))
    dz = sm.copy()
    dz[np.arange(B), y] -= 1.0
    dz /= B
    g = {"W3": dz.T @ h2, "b3": dz.sum(axis=0)}
    dh2 = dz @ p["W3"]
    da2 = dh2 * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * (a1 > 0)
    g["W1"] = da1.T @ x
    g["b1"] = da1.sum(axis=0)
    return L, np.concatenate([g[name].reshape(-1) for name, _ in SHAPES])


def adam_step(theta, m, v, g, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (t counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
