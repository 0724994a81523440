"""Pin of the FP64 network oracle: back-propagated gradient against central
finite differences, and the forward pass against a direct numpy evaluation."""
import numpy as np

import oracle


def _params(rng):
    p = rng.normal(0, 0.3, size=oracle.MLP_PARAMS)
    return p


def _numpy_forward(p, X):
    W1 = p[:768].reshape(64, 12)
    b1 = p[768:832]
    W2 = p[832:832 + 4096].reshape(64, 64)
    b2 = p[4928:4992]
    W3 = p[4992:5248].reshape(4, 64)
    b3 = p[5248:5252]
    h1 = np.maximum(X @ W1.T + b1, 0)
    h2 = np.maximum(h1 @ W2.T + b2, 0)
    return h2 @ W3.T + b3


def test_forward_matches_numpy():
    rng = np.random.default_rng(0)
    p = _params(rng)
    X = rng.normal(size=(17, 12))
    T = rng.normal(size=(17, 4))
    loss, _, Y = oracle.mlp_loss_grad(p, X, T, want_grad=False)
    Yn = _numpy_forward(p, X)
    assert np.allclose(Y, Yn, rtol=1e-12, atol=1e-12)
    assert abs(loss - ((Yn - T) ** 2).mean()) < 1e-12


def test_gradient_against_finite_differences():
    rng = np.random.default_rng(1)
    p = _params(rng)
    X = rng.normal(size=(9, 12))
    T = rng.normal(size=(9, 4))
    _, g, _ = oracle.mlp_loss_grad(p, X, T)
    idx = np.concatenate([rng.choice(768, 40, replace=False), 768 + rng.choice(64, 10, replace=False),
                          832 + rng.choice(4096, 60, replace=False), 4928 + rng.choice(64, 10, replace=False),
                          4992 + rng.choice(256, 30, replace=False), 5248 + np.arange(4)])
    h = 1e-6
    for k in idx:
        pp = p.copy()
        pp[k] += h
        lp, _, _ = oracle.mlp_loss_grad(pp, X, T, want_grad=False)
        pp[k] -= 2 * h
        lm, _, _ = oracle.mlp_loss_grad(pp, X, T, want_grad=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])) + 1e-9, k
