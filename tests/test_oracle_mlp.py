"""Oracle pin for the learned-guess network: analytic gradient against central differences."""
import numpy as np

from oracle import mlp


def test_parameter_count():
    assert mlp.NPARAM == 8 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 4801


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    theta = mlp.init_params(7) + 0.05 * rng.standard_normal(mlp.NPARAM)
    X = rng.standard_normal((37, 8))
    Y = rng.standard_normal(37)
    _, g = mlp.loss_and_grad(theta, X, Y)
    idx = rng.choice(mlp.NPARAM, size=60, replace=False)
    idx = np.concatenate([idx, [mlp.NPARAM - 1, 0, 512, 576]])
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        h = 1e-6
        e[i] = h
        fd = (mlp.loss_and_grad(theta + e, X, Y)[0] - mlp.loss_and_grad(theta - e, X, Y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_features_definition():
    rng = np.random.default_rng(0)
    yh = rng.standard_normal((9, 5, 2))
    X, Y, s = mlp.features(yh)
    assert X.shape == (10, 8) and Y.shape == (10,)
    assert np.allclose(s, np.sqrt(np.mean(yh[7] ** 2, axis=0)))
    assert np.allclose(X.reshape(5, 2, 8)[3, 1, 0], yh[7, 3, 1] / s[1])
    assert np.allclose(X.reshape(5, 2, 8)[3, 1, 7], yh[0, 3, 1] / s[1])
    assert np.allclose(Y.reshape(5, 2)[4, 0], (yh[8, 4, 0] - yh[7, 4, 0]) / s[0])


def test_extrapolation_is_exact_for_cubics():
    """The cubic extrapolation reproduces any cubic in the step index exactly (and its features
    target is then zero)."""
    n = np.arange(9.0)
    cub = (0.3 + 1.1 * n - 0.2 * n ** 2 + 0.05 * n ** 3)[:, None, None] * np.ones((9, 4, 2))
    assert np.allclose(mlp.extrapolate(cub), cub[-1], rtol=0, atol=1e-12)
    quart = (n ** 4)[:, None, None] * np.ones((9, 1, 1))
    assert abs(mlp.extrapolate(quart)[0, 0] - quart[-1, 0, 0]) == 24.0     # 4th difference of n^4
    _, Y, _ = mlp.features(cub + 1.0, base="extrap")
    assert np.max(np.abs(Y)) < 1e-12
