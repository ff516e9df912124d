"""Pins of oracle.reference: the closed form reduces to Phi0 at t = 0 and
its moments solve the linear ODE; Monte Carlo with the nonlinear term off
reproduces the closed form (two independent routes to the same number)."""
import numpy as np

from oracle import model, reference
import synthetic


def test_closed_form_at_t0_is_initial_gaussian():
    d = 5
    m0, C0 = model.cell_moments(d, (0.1,), (1.0,), 0.4, 0.8)
    pts = np.random.default_rng(0).normal(0, 1.0, (7, d))
    expect = np.exp(1j * pts @ m0 - 0.5 * np.einsum("pj,jk,pk->p", pts, C0, pts))
    np.testing.assert_allclose(reference.closed_form(pts, m0, C0, 0.3, 0.0), expect, atol=1e-15)


def test_closed_form_moments_solve_linear_ode():
    """d/dt m = nu D2 m, d/dt C = nu (D2 C + C D2^T) by central differences in t."""
    d, nu, t, e = 6, 0.2, 0.3, 1e-5
    m0, C0 = model.cell_moments(d, (0.5,), (1.0,), 0.4, 0.8)
    _, D2 = model.fd_matrices(d)
    mp, Cp = reference.closed_form_moments(m0, C0, nu, t + e)
    mm, Cm = reference.closed_form_moments(m0, C0, nu, t - e)
    m, C = reference.closed_form_moments(m0, C0, nu, t)
    np.testing.assert_allclose((mp - mm) / (2 * e), nu * D2 @ m, atol=1e-7)
    np.testing.assert_allclose((Cp - Cm) / (2 * e), nu * (D2 @ C + C @ D2.T), atol=1e-7)


def test_monte_carlo_linear_matches_closed_form():
    d, nu, T = 4, 0.3, 0.25
    m0, C0 = model.cell_moments(d, (0.0,), (1.0,), 0.3, 1.0)
    pts = np.array([[0.5, -0.3, 0.2, 0.0], [1.0, 1.0, 1.0, 1.0], [2.0, -1.0, 0.0, 0.5]])
    z = synthetic.mc_gaussian_samples(d, 100000, seed=5)

    # the Burgers ODE with the flux term removed is du/dt = nu D2 u
    D1, D2 = model.fd_matrices(d)
    Lc = np.linalg.cholesky(C0)
    u = m0[None, :] + z @ Lc.T
    dt = 1e-3
    for _ in range(int(round(T / dt))):
        f = lambda v: nu * v @ D2.T
        k1 = f(u); k2 = f(u + dt / 2 * k1); k3 = f(u + dt / 2 * k2); k4 = f(u + dt * k3)
        u = u + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    ph = np.exp(1j * u @ pts.T)
    est = ph.mean(axis=0)
    se = np.maximum(ph.real.std(axis=0), ph.imag.std(axis=0)) / np.sqrt(len(z))
    exact = reference.closed_form(pts, m0, C0, nu, T)
    assert np.all(np.abs(est - exact) <= 5 * se)


def test_monte_carlo_nonlinear_conserves_mean_sum():
    """The Burgers flux form conserves sum_k u_k sample by sample."""
    d = 5
    m0, C0 = model.cell_moments(d, (0.0,), (1.0,), 0.3, 1.0)
    z = synthetic.mc_gaussian_samples(d, 2000, seed=6)
    Lc = np.linalg.cholesky(C0)
    u0 = m0[None, :] + z @ Lc.T
    uT = reference.burgers_rk4(u0, 0.2, 1e-3, 0.05)
    np.testing.assert_allclose(uT.sum(axis=1), u0.sum(axis=1), atol=1e-12)
