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


def test_adam_second_and_third_steps_by_hand():
    """t = 2, 3 with scalar gradients, every quantity written out: the bias
    corrections no longer cancel, so a wrong moment recursion, a wrong power
    of beta or a missing square root fails here."""
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-8
    g1, g2, g3 = 0.5, -2.0, 1.5
    w0 = 1.0
    w1, m1, v1 = mlp.adam_step(np.array([w0]), np.zeros(1), np.zeros(1), np.array([g1]), 1, lr)
    w2, m2, v2 = mlp.adam_step(w1, m1, v1, np.array([g2]), 2, lr)
    w3, m3, v3 = mlp.adam_step(w2, m2, v2, np.array([g3]), 3, lr)
    # m_2 = 0.9 * 0.05 + 0.1 * (-2) = -0.155;  v_2 = 0.999 * 0.00025 + 0.001 * 4
    m2_hand = 0.045 - 0.2
    v2_hand = 0.999 * 0.00025 + 0.004
    step2 = lr * (m2_hand / (1 - 0.81)) / (np.sqrt(v2_hand / (1 - 0.998001)) + eps)
    assert abs(m2[0] - m2_hand) < 1e-15 and abs(v2[0] - v2_hand) < 1e-17
    assert abs(w2[0] - (w1[0] - step2)) < 1e-15
    # m_3 = 0.9 m_2 + 0.15;  v_3 = 0.999 v_2 + 0.001 * 2.25; corrections 1 - 0.9^3, 1 - 0.999^3
    m3_hand = 0.9 * m2_hand + 0.1 * g3
    v3_hand = 0.999 * v2_hand + 0.001 * g3 * g3
    step3 = lr * (m3_hand / (1 - 0.729)) / (np.sqrt(v3_hand / (1 - 0.997002999)) + eps)
    assert abs(m3[0] - m3_hand) < 1e-15 and abs(v3[0] - v3_hand) < 1e-17
    assert abs(w3[0] - (w2[0] - step3)) < 1e-14
    # and the values themselves: w1 = 1 - 0.01 * 0.5 / (0.5 + 1e-8)
    assert abs(w1[0] - (1.0 - 0.01 * 0.5 / (0.5 + 1e-8))) < 1e-15


def test_ensemble_bound_two_members_by_hand():
    """Two members whose outputs differ only through the output bias: member
    outputs y +- delta, so the mean is y, the per-output population standard
    deviation is |delta| (not |delta| sqrt 2, the sample one), and the bound
    is kappa ||delta||_2 / ||y||_2."""
    rng = np.random.default_rng(5)
    shape = (4, 5, 1, 3)
    p = _random_net(rng, *shape)
    lay, _ = mlp.layout(*shape)
    _, b_off, _, fo = lay[-1]
    delta = np.array([0.3, -0.1, 0.2])
    pa, pb = p.copy(), p.copy()
    pa[b_off:b_off + fo] += delta
    pb[b_off:b_off + fo] -= delta
    X = rng.normal(size=(2, 4))
    xs = (np.zeros(4), np.ones(4))
    ys = (np.zeros(3), np.ones(3))
    kappa = 2.5
    y, bound = mlp.predict([pa, pb], X, xs, ys, kappa, *shape)
    base = mlp.forward(p, X, *shape)[0]
    np.testing.assert_allclose(y, base, rtol=1e-13, atol=1e-15)
    want = kappa * np.sqrt(0.09 + 0.01 + 0.04) / np.linalg.norm(base, axis=1)
    np.testing.assert_allclose(bound, want, rtol=1e-12)


def test_column_stats_constant_two_valued_and_affine_columns():
    """Column 0 constant (sd reported as 1), column 1 takes -1 and 3 equally
    often (mean 1, population sd 2), column 2 is 2 x column 1 + 5 (mean 7,
    sd 4)."""
    c1 = np.array([-1.0, 3.0, -1.0, 3.0])
    A = np.stack([np.full(4, 7.25), c1, 2 * c1 + 5], axis=1)
    mu, sd = mlp.column_stats(A)
    np.testing.assert_allclose(mu, [7.25, 1.0, 7.0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(sd, [1.0, 2.0, 4.0], rtol=1e-15)
