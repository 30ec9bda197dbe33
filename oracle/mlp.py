"""Oracle for the selector's cost model: a 3-layer MLP in FP64 (test
infrastructure only).  Not part of the paper; it follows the plain
definitions of a fully connected network with ReLU, the mean-squared loss
and Adam (Kingma and Ba, ICLR 2015, Algorithm 1).

Network (sizes IN -> H -> H -> OUT):
    z1 = W1 x + b1,  h1 = relu(z1)
    z2 = W2 h1 + b2, h2 = relu(z2)
    y  = W3 h2 + b3
Parameter vector layout: W1 (H x IN, row-major), b1 (H), W2 (H x H), b2 (H),
W3 (OUT x H), b3 (OUT).

Loss over a batch of B rows, each with one observed output c_b and target t_b
(the measured log-time of candidate c_b):
    L = (1/B) sum_b (y_b[c_b] - t_b)^2

grad() is the analytic backward pass (chain rule, written out); adam_step()
one Adam update with bias correction.

Pins (tests/test_oracle_mlp.py): central finite differences of loss(),
closed forms (zero weights give y = b3; a single active row reproduces the
hand-derived gradient of a linear layer), and Adam's first step moving every
parameter by exactly lr * sign(g).
"""

import numpy as np

IN, H, OUT = 7, 64, 16


def sizes(nin=IN, nh=H, nout=OUT):
    return [(nh, nin), (nh,), (nh, nh), (nh,), (nout, nh), (nout,)]


def nparams(nin=IN, nh=H, nout=OUT):
    return sum(int(np.prod(s)) for s in sizes(nin, nh, nout))


def unpack(p, nin=IN, nh=H, nout=OUT):
    p = np.asarray(p, dtype=np.float64)
    out, o = [], 0
    for s in sizes(nin, nh, nout):
        n = int(np.prod(s))
        out.append(p[o:o + n].reshape(s))
        o += n
    assert o == p.size
    return out


def pack(parts):
    return np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in parts])


def forward(p, X, nin=IN, nh=H, nout=OUT):
    W1, b1, W2, b2, W3, b3 = unpack(p, nin, nh, nout)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + b3
    return y, (X, z1, h1, z2, h2)


def loss(p, X, cand, target, **kw):
    y, _ = forward(p, X, **kw)
    B = y.shape[0]
    r = y[np.arange(B), cand] - target
    return float(np.sum(r * r) / B)


def grad(p, X, cand, target, nin=IN, nh=H, nout=OUT):
    """Analytic gradient of loss() with respect to the parameter vector."""
    W1, b1, W2, b2, W3, b3 = unpack(p, nin, nh, nout)
    y, (X, z1, h1, z2, h2) = forward(p, X, nin, nh, nout)
    B = y.shape[0]
    dy = np.zeros_like(y)
    dy[np.arange(B), cand] = 2.0 * (y[np.arange(B), cand] - target) / B
    dW3 = dy.T @ h2
    db3 = dy.sum(axis=0)
    dz2 = (dy @ W3) * (z2 > 0)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    dW1 = dz1.T @ X
    db1 = dz1.sum(axis=0)
    return pack([dW1, db1, dW2, db2, dW3, db3])


def adam_step(p, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def features(m, n, k, dtype_index):
    """Input row of the selector for an m x n x k product of a dtype
    (0 f64, 1 f32, 2 bf16, 3 emulated f64): log2 sizes / 16 and a one-hot."""
    x = np.zeros(IN)
    x[0], x[1], x[2] = np.log2(m) / 16.0, np.log2(n) / 16.0, np.log2(k) / 16.0
    x[3 + dtype_index] = 1.0
    return x
