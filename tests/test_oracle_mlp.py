"""Pins of oracle.mlp (the surrogate network reference): GELU against known
values of the normal CDF, the backward pass against finite differences of the
forward pass, a network without hidden layers against the least-squares
gradient, and the first Adam step against its closed form."""
import numpy as np
import pytest

from oracle import mlp


def test_gelu_known_values_and_symmetry():
    # Phi(0) = 1/2, Phi(1) = 0.841344746068543, Phi(1.959963984540054) = 0.975
    # (standard normal table values), so GELU(x) = x Phi(x) there.
    np.testing.assert_allclose(mlp.gelu(0.0), 0.0, atol=0)
    np.testing.assert_allclose(mlp.gelu(1.0), 0.841344746068543, rtol=1e-14)
    np.testing.assert_allclose(mlp.gelu(1.959963984540054), 1.959963984540054 * 0.975, rtol=1e-14)
    x = np.linspace(-6, 6, 49)
    np.testing.assert_allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-15)
    np.testing.assert_allclose(mlp.gelu_grad(0.0), 0.5, atol=0)
    e = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(x), (mlp.gelu(x + e) - mlp.gelu(x - e)) / (2 * e), atol=1e-9)


def _random_net(rng, n_in, width, depth, n_out):
    lay, P = mlp.layout(n_in, width, depth, n_out)
    p = np.zeros(P)
    for w, b, fi, fo in lay:
        p[w:w + fi * fo] = rng.normal(0, 1 / np.sqrt(fi), fi * fo)
        p[b:b + fo] = rng.normal(0, 0.1, fo)
    return p


@pytest.mark.parametrize("shape", [(3, 5, 2, 4), (12, 8, 4, 14)])
def test_backward_matches_finite_differences(shape):
    n_in, width, depth, n_out = shape
    rng = np.random.default_rng(1)
    p = _random_net(rng, *shape)
    X = rng.normal(size=(6, n_in))
    T = rng.normal(size=(6, n_out))
    _, g = mlp.loss_and_grad(p, X, T, *shape)
    e = 1e-6
    for k in rng.choice(p.size, 40, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[k] += e
        pm[k] -= e
        fd = (mlp.loss_and_grad(pp, X, T, *shape)[0] - mlp.loss_and_grad(pm, X, T, *shape)[0]) / (2 * e)
        assert abs(fd - g[k]) < 1e-8 * max(1.0, abs(fd))


def test_linear_network_is_least_squares():
    """depth 0: Y = X W^T + b, dL/dW = 2 (Y - T)^T X / (B O)."""
    rng = np.random.default_rng(2)
    n_in, n_out, B = 4, 3, 7
    W = rng.normal(size=(n_out, n_in))
    b = rng.normal(size=n_out)
    p = np.concatenate([W.ravel(), b])
    X, T = rng.normal(size=(B, n_in)), rng.normal(size=(B, n_out))
    R = X @ W.T + b - T
    loss, g = mlp.loss_and_grad(p, X, T, n_in, 1, 0, n_out)
    np.testing.assert_allclose(loss, (R ** 2).sum() / (B * n_out), rtol=1e-14)
    np.testing.assert_allclose(g[:W.size], (2 * R.T @ X / (B * n_out)).ravel(), rtol=1e-13)
    np.testing.assert_allclose(g[W.size:], 2 * R.sum(0) / (B * n_out), rtol=1e-13)


def test_first_adam_step_closed_form():
    """At t = 1 the bias corrections cancel: w - lr g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    w, g = rng.normal(size=9), rng.normal(size=9)
    w1, m1, v1 = mlp.adam_step(w, np.zeros(9), np.zeros(9), g, 1, 1e-3)
    np.testing.assert_allclose(w1, w - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12)


def test_ensemble_bound_is_zero_for_identical_members():
    rng = np.random.default_rng(4)
    shape = (5, 6, 2, 3)
    p = _random_net(rng, *shape)
    X = rng.normal(size=(4, 5))
    xs = (np.zeros(5), np.ones(5))
    ys = (np.full(3, 2.0), np.full(3, 0.5))
    y, bound = mlp.predict([p, p, p], X, xs, ys, 3.0, *shape)
    np.testing.assert_allclose(y, 2.0 + 0.5 * mlp.forward(p, X, *shape)[0], rtol=1e-14)
    np.testing.assert_allclose(bound, 0.0, atol=0)
