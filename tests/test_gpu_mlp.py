"""Proposal-network kernels (GPU) against the NumPy FP64 oracle: forward,
backpropagated gradient (relative 1e-4 in FP32), Adam step, and training."""
import numpy as np
import pytest

from oracle import mlp as om
from paper_2404_10223_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2404_10223_gb300 import build as B
    import os
    if not os.path.exists(B.LIB):
        B.build()


def setup(n_in=74, n_h=256, n_out=66, B=512, seed=0, weighted=True):
    from paper_2404_10223_gb300 import mlp
    rng = np.random.default_rng(seed)
    flat = inputs.draw_mlp_params(rng, n_in, n_h, n_out, out_scale=1.0)
    X = rng.normal(size=(B, n_in)).astype(np.float32)
    T = rng.normal(size=(B, n_out)).astype(np.float32)
    w = rng.uniform(0.0, 2.0, B).astype(np.float32) if weighted else None
    net = mlp.Mlp(n_in, n_h, n_out, max_batch=max(B, 1024))
    net.set_params(flat)
    return net, flat, X, T, w


@pytest.mark.parametrize("weighted", [False, True])
def test_forward_and_gradient_match_oracle(weighted):
    net, flat, X, T, w = setup(weighted=weighted)
    with net:
        p = om.unpack(flat.astype(np.float64), net.n_in, net.n_h, net.n_out)
        Y = net.forward(X)
        Yo, _ = om.forward(p, X.astype(np.float64))
        assert np.abs(Y - Yo).max() <= 1e-5 * max(1.0, np.abs(Yo).max())
        L, g = net.gradient(X, T, w)
        Lo, go = om.gradient(p, X.astype(np.float64), T.astype(np.float64), None if w is None else w.astype(np.float64))
        gof = om.pack(go)
        assert abs(L - Lo) <= 1e-5 * abs(Lo)
        for name in om.NAMES:   # per tensor, relative to that tensor's largest entry
            a = om.unpack(g.astype(np.float64), net.n_in, net.n_h, net.n_out)[name]
            b = go[name]
            assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max(), name
        assert net.last_launches() > 0
        assert np.isfinite(gof).all()


def test_adam_step_matches_oracle():
    net, flat, X, T, w = setup(n_in=8, n_h=16, n_out=4, B=64, seed=2)
    with net:
        p = om.unpack(flat.astype(np.float64), 8, 16, 4)
        _, go = om.gradient(p, X.astype(np.float64), T.astype(np.float64), w.astype(np.float64))
        g = om.pack(go)
        lr = 1e-2
        net.adam_step(X, T, w, lr=lr)
        p1 = net.get_params().astype(np.float64)
        ref, _, _ = om.adam_step(flat.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, lr)
        keep = np.abs(g) > 1e-5            # near-zero gradients: g / (|g| + eps) is ill-conditioned in FP32
        assert np.abs(p1 - ref)[keep].max() <= 1e-3 * lr + 1e-7
        assert np.abs(p1 - ref).max() <= 2 * lr


def test_training_reduces_loss():
    rng = np.random.default_rng(5)
    from paper_2404_10223_gb300 import mlp
    n_in, n_h, n_out, B = 10, 64, 3, 256
    X = rng.normal(size=(B, n_in)).astype(np.float32)
    A = rng.normal(size=(n_in, n_out)) / np.sqrt(n_in)
    T = np.tanh(X @ A).astype(np.float32)           # a smooth target
    with mlp.Mlp(n_in, n_h, n_out, max_batch=B) as net:
        net.set_params(inputs.draw_mlp_params(rng, n_in, n_h, n_out))
        l0 = net.gradient(X, T)[0]
        for _ in range(300):
            net.adam_step(X, T, lr=3e-3)
        l1 = net.gradient(X, T)[0]
    assert l1 < 0.05 * l0
