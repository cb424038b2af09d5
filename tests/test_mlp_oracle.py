"""Pins of the proposal-network oracle (CPU): GELU closed forms, backpropagation
against central finite differences, and a hand-computed Adam step."""
import math

import numpy as np
import pytest

from oracle import mlp as om
from paper_2404_10223_gb300 import inputs


def test_gelu_closed_forms():
    # gelu(z) = z Phi(z); Phi(1) = 0.8413447460685429 (standard normal CDF)
    assert om.gelu(np.array(0.0)) == 0.0
    assert abs(om.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    assert abs(om.gelu(np.array(-1.0)) - (-1.0) * (1 - 0.8413447460685429)) < 1e-15
    assert abs(om.gelu(np.array(30.0)) - 30.0) < 1e-12 and abs(om.gelu(np.array(-30.0))) < 1e-12
    z = np.linspace(-5, 5, 41)
    h = 1e-6
    fd = (om.gelu(z + h) - om.gelu(z - h)) / (2 * h)
    assert np.abs(om.gelu_grad(z) - fd).max() < 1e-8
    assert abs(om.gelu_grad(np.array(0.0)) - 0.5) < 1e-15


@pytest.mark.parametrize("weighted", [False, True])
def test_backprop_matches_finite_differences(weighted):
    rng = np.random.default_rng(3)
    n_in, n_h, n_out, B = 4, 6, 3, 5
    flat = inputs.draw_mlp_params(rng, n_in, n_h, n_out, out_scale=1.0).astype(np.float64)
    flat += rng.normal(0, 0.1, flat.shape)           # non-zero biases too
    X = rng.normal(size=(B, n_in))
    T = rng.normal(size=(B, n_out))
    w = rng.uniform(0.1, 2.0, B) if weighted else None
    p = om.unpack(flat, n_in, n_h, n_out)
    L, g = om.gradient(p, X, T, w)
    assert abs(L - om.loss(p, X, T, w)) < 1e-15
    gflat = om.pack(g)
    h = 1e-6
    fd = np.zeros_like(flat)
    for i in range(len(flat)):
        e = np.zeros_like(flat)
        e[i] = h
        fd[i] = (om.loss(om.unpack(flat + e, n_in, n_h, n_out), X, T, w) -
                 om.loss(om.unpack(flat - e, n_in, n_h, n_out), X, T, w)) / (2 * h)
    assert np.abs(gflat - fd).max() <= 1e-7 * max(1.0, np.abs(fd).max())


def test_loss_weights_are_scale_free_and_zero_at_target():
    rng = np.random.default_rng(4)
    flat = inputs.draw_mlp_params(rng, 3, 4, 2).astype(np.float64)
    p = om.unpack(flat, 3, 4, 2)
    X = rng.normal(size=(6, 3))
    T = rng.normal(size=(6, 2))
    w = rng.uniform(0.5, 1.5, 6)
    assert abs(om.loss(p, X, T, w) - om.loss(p, X, T, 7.0 * w)) < 1e-14
    Y, _ = om.forward(p, X)
    assert om.loss(p, X, Y, w) == 0.0


def test_adam_first_step_is_signed_learning_rate():
    # t = 1: mhat = g, vhat = g^2, so the step is lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p0 = np.array([1.0, 1.0, 1.0, 1.0])
    p1, m, v = om.adam_step(p0, g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=1e-8)
    expect = p0 - 0.01 * g / (np.abs(g) + 1e-8)
    assert np.abs(p1 - expect).max() < 1e-15
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
