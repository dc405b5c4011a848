"""Pins of the FP64 reference network used to check the GPU training
kernels: the analytic gradient against central finite differences, and one
Adam step from zero state against its closed form (-lr * g / (|g| + eps))."""
import numpy as np

from oracle import mlp


def _params(seed):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.3, mlp.NP)
    p[mlp.P_IS:mlp.P_W1] = np.abs(p[mlp.P_IS:mlp.P_W1]) + 0.5
    return p


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = _params(2)
    X = rng.normal(0, 2, (37, mlp.NF))
    T = rng.normal(0, 1, 37)
    loss, g = mlp.loss_grad(p, X, T)
    assert np.all(g[:mlp.P_W1] == 0)
    idx = np.r_[rng.choice(np.arange(mlp.P_W1, mlp.NP), 60, replace=False), mlp.P_B4, mlp.P_W4, mlp.P_B1]
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_grad(pp, X, T)[0] - mlp.loss_grad(pm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    p = _params(4)
    g = rng.normal(0, 1e-2, mlp.NP)
    p1, m, v = mlp.adam(p, g, np.zeros(mlp.NP), np.zeros(mlp.NP), 1e-3, 1)
    sl = slice(mlp.P_W1, mlp.NP)
    np.testing.assert_allclose(p1[sl] - p[sl], -1e-3 * g[sl] / (np.abs(g[sl]) + 1e-8), rtol=1e-9, atol=1e-15)
    assert np.array_equal(p1[:mlp.P_W1], p[:mlp.P_W1])


def test_gelu_derivative():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_d(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), atol=1e-8)
