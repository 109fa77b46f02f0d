"""The fp64 MLP reference pinned by central finite differences and closed
forms (CPU only)."""

import numpy as np

from oracle import mlp


def _params(rng, scale=0.2):
    W1 = rng.standard_normal((256, 256)) * scale / 16
    b1 = rng.standard_normal(256) * 0.1
    w2 = rng.standard_normal(256) * scale
    b2 = 0.3
    return W1, b1, w2, b2


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    W1, b1, w2, b2 = _params(rng)
    X = rng.standard_normal((24, 256))
    t = rng.standard_normal(24)
    dW1, db1, dw2, db2 = mlp.backward(W1, b1, w2, b2, X, t)
    h = 1e-6
    for (i, j) in [(0, 0), (3, 200), (255, 17), (128, 128), (77, 5)]:
        P, M = W1.copy(), W1.copy()
        P[i, j] += h
        M[i, j] -= h
        fd = (mlp.loss(P, b1, w2, b2, X, t) - mlp.loss(M, b1, w2, b2, X, t)) / (2 * h)
        assert abs(fd - dW1[i, j]) <= 1e-6 * max(1.0, abs(fd)), (i, j, fd, dW1[i, j])
    for k in (0, 100, 255):
        P, M = b1.copy(), b1.copy()
        P[k] += h
        M[k] -= h
        fd = (mlp.loss(W1, P, w2, b2, X, t) - mlp.loss(W1, M, w2, b2, X, t)) / (2 * h)
        assert abs(fd - db1[k]) <= 1e-6 * max(1.0, abs(fd))
        P, M = w2.copy(), w2.copy()
        P[k] += h
        M[k] -= h
        fd = (mlp.loss(W1, b1, P, b2, X, t) - mlp.loss(W1, b1, M, b2, X, t)) / (2 * h)
        assert abs(fd - dw2[k]) <= 1e-6 * max(1.0, abs(fd))
    fd = (mlp.loss(W1, b1, w2, b2 + h, X, t) - mlp.loss(W1, b1, w2, b2 - h, X, t)) / (2 * h)
    assert abs(fd - db2) <= 1e-6 * max(1.0, abs(fd))


def test_closed_forms():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((10, 256))
    # zero first layer: every hidden unit equals relu(b1); output is constant
    W1 = np.zeros((256, 256))
    b1 = np.linspace(-1, 1, 256)
    w2 = np.ones(256)
    _, _, y = mlp.forward(W1, b1, w2, 0.5, X)
    assert np.allclose(y, np.maximum(b1, 0).sum() + 0.5)
    # identity-like first layer with positive inputs: y = sum of inputs (w2 = 1)
    Xp = np.abs(X)
    _, _, y = mlp.forward(np.eye(256), np.zeros(256), np.ones(256), 0.0, Xp)
    assert np.allclose(y, Xp.sum(axis=1))
    # loss is zero at the target and the gradient vanishes there
    W1, b1, w2, b2 = _params(rng)
    _, _, y = mlp.forward(W1, b1, w2, b2, X)
    g = mlp.backward(W1, b1, w2, b2, X, y)
    assert mlp.loss(W1, b1, w2, b2, X, y) == 0.0
    assert all(np.all(np.asarray(a) == 0) for a in g)
