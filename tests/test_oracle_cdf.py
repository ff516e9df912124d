"""Pins of oracle.cdf (the CDF equation, Sec. 5 Eq. cdf-burgers) and of the
truncated Euler and midpoint schemes of oracle.tt (Eqs. adaptive-euler-method
and adaptive-midpoint-method).

What fixes each part without the oracle itself:
* the tensor-train operator against the equation written term by term on the
  full grid;
* the corner value F(U, .., U): every term carries dF/du_i, which the
  outflow condition sets to zero on the face u_i = U, so it is conserved
  exactly;
* with the D1 terms off the dynamics are linear, u' = gamma D2 u: the normal
  CDF with covariance sigma^2 E E^T, E = exp(t gamma D2) (scipy's
  multivariate normal CDF), reached at second order in du;
* the full equation against Monte Carlo of the Burgers ODE with the velocity
  of Eq. (pdf-burgers), v = -u o (D1 u) + gamma D2 u, from shifted means so
  that the D1 terms move the CDF well beyond the sampling error (a sign or
  index error in them fails);
* local truncation errors of the explicit Euler and midpoint steps by
  Richardson extrapolation (the paper's order study, Sec. 5.1): orders 1
  and 2, i.e. errors falling by 4 and 8 per halving of dt; and the
  truncated TT schemes equal the full-grid ones when nothing is discarded."""
import numpy as np
import pytest
from scipy.linalg import expm
from scipy.stats import multivariate_normal

from oracle import cdf, model, tt
import synthetic


@pytest.mark.parametrize("d,n,nonlinear", [(3, 8, True), (4, 7, True), (3, 9, False)])
def test_mpo_matches_the_equation_term_by_term(d, n, nonlinear):
    gamma = 0.07
    x = synthetic.random_tt_cores(d, n, [1] + [3] * (d - 1) + [1], seed=40 + d)
    W = cdf.mpo_blocks(d, n, gamma, nonlinear=nonlinear)
    y = tt.apply_mpo(x, W, model.mpo_bond_dims(d))
    want = cdf.apply_G(tt.full(x), d, n, gamma, nonlinear=nonlinear)
    assert np.linalg.norm(tt.full(y) - want) <= 1e-12 * np.linalg.norm(want)


def test_operator_pieces():
    """J integrates exactly the functions the trapezoidal rule integrates
    exactly (linear ones), D differentiates quadratics exactly in the
    interior and vanishes on the boundary rows."""
    n = 11
    A, D, J = cdf.mode_operators(n)
    u, du = cdf.u_grid(n)
    assert abs(u[0] + 1.3) < 1e-15 and abs(u[-1] - 1.3) < 1e-15
    np.testing.assert_allclose(J @ (2 * u + 1), (u ** 2 + u) - (u[0] ** 2 + u[0]), atol=1e-14)
    np.testing.assert_allclose((D @ u ** 2)[1:-1], 2 * u[1:-1], atol=1e-13)
    assert np.all(D[0] == 0) and np.all(D[-1] == 0)


def test_corner_value_is_conserved():
    d, n, gamma = 3, 9, 0.1
    F = cdf.initial_grid(d, n, mu=[0.2, -0.1, 0.05])
    G = lambda X: cdf.apply_G(X, d, n, gamma)
    out = cdf.apply_G(F, d, n, gamma)
    assert out[-1, -1, -1] == 0.0
    F2 = cdf.rk4_step(F, 0.05, G)
    assert F2[-1, -1, -1] == F[-1, -1, -1]


def _linear_solution(d, gamma, T, pts):
    _, D2 = model.fd_matrices(d)
    E = expm(T * gamma * D2)
    C = cdf.SIGMA0 ** 2 * E @ E.T
    return np.array([multivariate_normal.cdf(p, mean=np.zeros(d), cov=C, abseps=1e-12, releps=1e-12) for p in pts])


def test_linear_dynamics_closed_form_second_order():
    """D1 terms off: F(t) = normal CDF of N(0, sigma^2 E E^T); the full-grid
    RK4 solve reaches it with error falling by ~4 when du halves."""
    d, gamma, T, dt = 3, 0.4, 0.5, 0.0125
    pts = np.array([[0.0, 0.0, 0.0], [0.1625, -0.1625, 0.0], [-0.325, 0.1625, 0.325], [0.325, 0.325, -0.1625]])
    exact = _linear_solution(d, gamma, T, pts)
    errs = []
    for n in (33, 65):
        u, du = cdf.u_grid(n)
        idx = np.rint((pts + 1.3) / du).astype(int)
        assert np.allclose(u[idx], pts, atol=1e-12)
        G = lambda X: cdf.apply_G(X, d, n, gamma, nonlinear=False)
        F = cdf.initial_grid(d, n)
        for _ in range(int(round(T / dt))):
            F = cdf.rk4_step(F, dt, G)
        errs.append(np.abs(F[tuple(idx.T)] - exact).max())
    # the change over [0, T] is far above the error (the test has power)
    F0 = np.prod(cdf.gaussian_cdf(pts), axis=1)
    assert np.abs(exact - F0).max() > 50 * errs[0]
    assert 3.3 < errs[0] / errs[1] < 4.8 and errs[1] < 2e-4


def test_full_equation_against_monte_carlo():
    """Forty points around the mean after T = 2: the grid solve (n = 65,
    RK4) against 2e5 samples of the Burgers ODE.  The D1 terms move the
    sampled CDF by tens of standard errors (the linear dynamics alone are
    far off), and the equation reproduces the samples within 4 of them."""
    d, n, gamma, T, dt = 3, 65, 0.01, 2.0, 0.02
    mu = np.array([0.3, -0.3, 0.0])
    u, du = cdf.u_grid(n)
    rng = np.random.default_rng(1)
    idx = np.rint((mu[None, :] + rng.choice([-0.25, -0.1, 0.0, 0.1, 0.25], (40, d)) + 1.3) / du).astype(int)
    pts = u[idx]
    G = lambda X: cdf.apply_G(X, d, n, gamma)
    F = cdf.initial_grid(d, n, mu=mu)
    for _ in range(int(round(T / dt))):
        F = cdf.rk4_step(F, dt, G)
    got = F[tuple(idx.T)]
    z = synthetic.mc_gaussian_samples(d, 200000, seed=9)
    u0 = mu[None, :] + cdf.SIGMA0 * z
    mc, se = cdf.mc_cdf(pts, u0, gamma, T, 0.01)
    lin, _ = cdf.mc_cdf(pts, u0, gamma, T, 0.01, nonlinear=False)
    assert np.max(np.abs(mc - lin) / se) > 30
    assert np.all(np.abs(got - mc) <= 4 * se)


@pytest.mark.parametrize("scheme,ratio", [("euler", 4.0), ("midpoint", 8.0)])
def test_richardson_local_error_orders(scheme, ratio):
    """One step of size dt against the extrapolation of two steps of dt/2
    (order p: (2^p f2 - f1) / (2^p - 1)): errors ~ dt^(p+1)."""
    d, n, gamma = 3, 17, 0.05
    F0 = cdf.initial_grid(d, n, mu=[0.2, -0.1, 0.0])
    G = lambda X: cdf.apply_G(X, d, n, gamma)
    step = cdf.euler_step if scheme == "euler" else cdf.midpoint_step
    p = 1 if scheme == "euler" else 2
    errs = []
    for dt in (0.04, 0.02, 0.01):
        f1 = step(F0, dt, G)
        f2 = step(step(F0, dt / 2, G), dt / 2, G)
        fr = (2 ** p * f2 - f1) / (2 ** p - 1)
        errs.append(np.linalg.norm(f1 - fr))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert abs(r1 / ratio - 1) < 0.15 and abs(r2 / ratio - 1) < 0.15


@pytest.mark.parametrize("scheme", ["euler", "midpoint"])
def test_truncated_tt_schemes_equal_full_grid_without_truncation(scheme):
    d, n, gamma, dt = 3, 9, 0.05, 0.02
    W = cdf.mpo_blocks(d, n, gamma)
    bond = model.mpo_bond_dims(d)
    G_tt = lambda x: tt.apply_mpo(x, W, bond)
    G_full = lambda X: cdf.apply_G(X, d, n, gamma)
    x = cdf.initial_tt(d, n, mu=[0.2, -0.1, 0.0])
    F = tt.full(x)
    step_tt = tt.euler_step if scheme == "euler" else tt.midpoint_step
    step_full = cdf.euler_step if scheme == "euler" else cdf.midpoint_step
    log = []
    for _ in range(3):
        x, discs = step_tt(x, dt, G_tt, 0.0, 10 ** 6, record=log)
        F = step_full(F, dt, G_full)
    assert len(log) == 3 * (2 if scheme == "euler" else 3)
    assert np.linalg.norm(tt.full(x) - F) <= 1e-12 * np.linalg.norm(F)
