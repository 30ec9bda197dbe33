"""Pins for the MLP oracle (oracle/mlp.py): finite differences, closed forms,
Adam's first step."""
import numpy as np
import pytest

from oracle import mlp

import cosma_inputs as ci


def _params(scale=0.3, seed=4, nin=7, nh=16, nout=5):
    n = mlp.nparams(nin, nh, nout)
    return scale * ci.entries(np.arange(n), np.zeros(n), 1, "uniform", "f64", seed, 3)


def _batch(B=9, nin=7, nout=5, seed=6):
    X = ci.matrix(B, nin, "uniform", "f64", seed, 0)
    cand = (ci.entries(np.arange(B), np.zeros(B), 1, "integer", "f64", seed, 1) + 8).astype(int) % nout
    t = ci.entries(np.arange(B), np.zeros(B), 1, "uniform", "f64", seed, 2)
    return X, cand, t


def test_gradient_matches_central_differences():
    kw = dict(nin=7, nh=16, nout=5)
    p = _params()
    X, cand, t = _batch()
    g = mlp.grad(p, X, cand, t, **kw)
    h = 1e-6
    num = np.zeros_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        num[i] = (mlp.loss(p + e, X, cand, t, **kw) - mlp.loss(p - e, X, cand, t, **kw)) / (2 * h)
    assert np.allclose(g, num, rtol=1e-5, atol=1e-8)


def test_zero_weights_give_output_bias():
    kw = dict(nin=7, nh=16, nout=5)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(np.zeros(mlp.nparams(**kw)), **kw)
    b3 = np.arange(5, dtype=float)
    p = mlp.pack([W1, b1, W2, b2, W3, b3])
    X, _, _ = _batch()
    y, _ = mlp.forward(p, X, **kw)
    assert np.array_equal(y, np.tile(b3, (X.shape[0], 1)))


def test_last_layer_gradient_closed_form():
    # with every hidden unit active the last layer is linear in h2:
    # dL/dW3[c] = (2/B) sum_b (y_b[c] - t_b) h2_b over rows with c_b = c
    kw = dict(nin=7, nh=16, nout=5)
    p = _params(scale=0.1)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, **kw)
    b1 = b1 + 10.0
    b2 = b2 + 10.0
    p = mlp.pack([W1, b1, W2, b2, W3, b3])
    X, cand, t = _batch()
    y, (_, z1, h1, z2, h2) = mlp.forward(p, X, **kw)
    assert (z1 > 0).all() and (z2 > 0).all()
    g = mlp.unpack(mlp.grad(p, X, cand, t, **kw), **kw)
    B = X.shape[0]
    for c in range(5):
        rows = cand == c
        want = 2.0 / B * ((y[rows, c] - t[rows])[:, None] * h2[rows]).sum(axis=0)
        assert np.allclose(g[4][c], want, rtol=1e-12, atol=1e-15)


def test_adam_first_step_is_lr_sign():
    p = _params()
    g = _params(seed=9) + 0.01
    p1, m, v = mlp.adam_step(p, g, np.zeros_like(p), np.zeros_like(p), 1, lr=1e-3, eps=0.0)
    assert np.allclose(p - p1, 1e-3 * np.sign(g), rtol=1e-12)


def test_layout_roundtrip_and_count():
    assert mlp.nparams() == 7 * 64 + 64 + 64 * 64 + 64 + 16 * 64 + 16
    p = np.arange(mlp.nparams(), dtype=float)
    assert np.array_equal(mlp.pack(mlp.unpack(p)), p)


def test_features():
    x = mlp.features(256, 65536, 1024, 2)
    assert np.allclose(x[:3], [0.5, 1.0, 10 / 16]) and x[5] == 1 and x[3:].sum() == 1
