"""CPU oracle of the rotation-proposal network (test infrastructure only).

Plain NumPy, FP64: the forward pass, the weighted mean-squared loss, the
gradient by hand-written backpropagation (chain rule layer by layer) and one
Adam step (Kingma & Ba, arXiv 1412.6980, Algorithm 1).  The network is the one
of include/tnqe_mlp.h: n_in -> n_h -> n_h -> n_out, exact GELU
gelu(z) = z (1 + erf(z / sqrt 2)) / 2 (Hendrycks & Gimpel, arXiv 1606.08415).

Pinned in tests/test_mlp_oracle.py against central finite differences of the
loss (an independent check of the backpropagation), closed forms of GELU and
a hand-computed Adam step.  Only tests/, __graft_entry__.smoke() and bench.py
may import this module.
"""
from __future__ import annotations

from typing import Dict, Tuple

import numpy as np
from scipy.special import erf

NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def shapes(n_in: int, n_h: int, n_out: int):
    return {"W1": (n_h, n_in), "b1": (n_h,), "W2": (n_h, n_h), "b2": (n_h,), "W3": (n_out, n_h), "b3": (n_out,)}


def unpack(flat: np.ndarray, n_in: int, n_h: int, n_out: int) -> Dict[str, np.ndarray]:
    out, o = {}, 0
    for k, shp in shapes(n_in, n_h, n_out).items():
        n = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    assert o == len(flat)
    return out


def pack(p: Dict[str, np.ndarray]) -> np.ndarray:
    return np.concatenate([np.ravel(p[k]) for k in NAMES])


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(p, X):
    Z1 = X @ p["W1"].T + p["b1"]
    A1 = gelu(Z1)
    Z2 = A1 @ p["W2"].T + p["b2"]
    A2 = gelu(Z2)
    Y = A2 @ p["W3"].T + p["b3"]
    return Y, (Z1, A1, Z2, A2)


def loss(p, X, T, w=None) -> float:
    Y, _ = forward(p, X)
    w = np.ones(len(X)) if w is None else np.asarray(w, dtype=np.float64)
    return float(np.sum(w[:, None] * (Y - T) ** 2) / (Y.shape[1] * np.sum(w)))


def gradient(p, X, T, w=None) -> Tuple[float, Dict[str, np.ndarray]]:
    """Loss and dLoss/dparam by backpropagation through the three layers."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    w = np.ones(len(X)) if w is None else np.asarray(w, dtype=np.float64)
    Y, (Z1, A1, Z2, A2) = forward(p, X)
    scale = 1.0 / (Y.shape[1] * np.sum(w))
    R = Y - T
    L = float(np.sum(w[:, None] * R ** 2) * scale)
    dY = 2.0 * w[:, None] * R * scale
    g = {"W3": dY.T @ A2, "b3": dY.sum(axis=0)}
    dZ2 = (dY @ p["W3"]) * gelu_grad(Z2)
    g["W2"] = dZ2.T @ A1
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ p["W2"]) * gelu_grad(Z1)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0)
    return L, g


def adam_step(flat, grad_flat, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update; t is the 1-based step number.  Returns (params, m, v)."""
    m = b1 * m + (1.0 - b1) * grad_flat
    v = b2 * v + (1.0 - b2) * grad_flat ** 2
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return flat - lr * mhat / (np.sqrt(vhat) + eps), m, v
