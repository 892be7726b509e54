"""Pins of the FP64 reference network: finite differences and a closed form."""
import numpy as np

from oracle import mlp


def test_parameter_count():
    assert mlp.NPARAM == 16 * 64 + 64 + 64 * 64 + 64 + 64 * 4 + 4 + 32


def test_zero_network_gives_uniform_softmax():
    p = np.zeros(mlp.NPARAM)
    p[-16:] = 1.0  # sd
    X = np.random.default_rng(0).standard_normal((7, 16))
    y = np.array([0, 1, 2, 3, 0, 1, 2])
    assert abs(mlp.loss(p, X, y) - np.log(4.0)) < 1e-15
    g = mlp.grad(p, X, y)
    # only b3 can move: d loss / d b3_k = mean(1/4 - [y == k])
    gb3 = g[mlp.NPARAM - 32 - 4:mlp.NPARAM - 32]
    want = np.array([0.25 - np.mean(y == k) for k in range(4)])
    assert np.abs(gb3 - want).max() < 1e-15


def test_gelu_matches_erf_definition():
    x = np.array([-3.0, -0.5, 0.0, 0.7, 2.5])
    from math import erf, sqrt
    assert np.allclose(mlp.gelu(x), [0.5 * v * (1 + erf(v / sqrt(2))) for v in x], rtol=0, atol=1e-16)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.abs(fd - mlp.gelu_prime(x)).max() < 1e-8


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((9, 16)) * 3 - 2
    y = rng.integers(0, 4, 9)
    p = mlp.init(3, mu=X.mean(axis=0), sd=X.std(axis=0))
    g = mlp.grad(p, X, y)
    idx = np.concatenate([rng.choice(mlp.NTRAIN, 60, replace=False), [mlp.NTRAIN - 1, 0]])
    h = 1e-5
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, X, y) - mlp.loss(p - e, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(fd), (i, fd, g[i])
