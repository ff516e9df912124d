"""Pins of the full-grid oracle: plane-wave symbol and its small-da limit (the
Burgers right-hand side written here with np.roll, independent of the
oracle's matrices), exact invariants of the discrete scheme, the linear
closed form with its convergence orders, RK4's local order by Richardson
(the paper's LTE technique, Sec. 5.1), the Gaussian closed form of the
finite-difference moments, and a Monte-Carlo estimate from the Burgers ODE."""
import numpy as np
import pytest

from oracle import fullgrid, model, reference
import synthetic


def _burgers_rhs_roll(u, nu):
    d = len(u)
    h = 2 * np.pi / d
    up, um = np.roll(u, -1), np.roll(u, 1)
    return -(up ** 2 - um ** 2) / (4 * h) + nu * (up - 2 * u + um) / h ** 2


def _plane_wave(m, n, L):
    d = len(m)
    a, _ = model.a_grid(n, L)
    X = np.stack(np.meshgrid(*([a] * d), indexing="ij"), axis=-1)
    return np.exp(1j * (X @ m)), X


def test_planewave_symbol_exact():
    """G exp(i a.m) at interior points = sum_k a_k [ (i/2) (D1 s_S)_k
    + nu (D2 s_D)_k ] exp(i a.m), s_S(w) = -4 sin^2(w da/2)/da^2,
    s_D(w) = i sin(w da)/da; written with np.roll stencils."""
    d, n, L, nu = 3, 14, 2.0, 0.13
    rng = np.random.default_rng(3)
    m = rng.normal(0, 1.0, d)
    F, X = _plane_wave(m, n, L)
    G = fullgrid.apply_G(F, d, n, L, nu)
    _, da = model.a_grid(n, L)
    h = 2 * np.pi / d
    sS = -4 * np.sin(m * da / 2) ** 2 / da ** 2
    sD = 1j * np.sin(m * da) / da
    coef = 0.5j * (np.roll(sS, -1) - np.roll(sS, 1)) / (2 * h) \
        + nu * (np.roll(sD, -1) - 2 * sD + np.roll(sD, 1)) / h ** 2
    expect = (X @ coef) * F
    inner = (slice(2, n - 1),) * d
    np.testing.assert_allclose(G[inner], expect[inner], atol=1e-11 * np.abs(expect).max())


def test_planewave_limit_is_burgers():
    """(G Phi)/Phi -> i a . (du/dt)(m) as da -> 0, second order."""
    d, nu, L = 4, 0.07, 1.0
    m = np.array([0.3, -0.2, 0.5, 0.1])
    errs = []
    for n in (16, 32, 64):
        F, X = _plane_wave(m, n, L)
        G = fullgrid.apply_G(F, d, n, L, nu)
        pt = (n // 2 + n // 8, n // 2 - n // 16, n // 2 + n // 4, n // 2)
        a = X[pt]
        exact = 1j * a @ _burgers_rhs_roll(m, nu)
        errs.append(abs(G[pt] / F[pt] - exact))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def _c1_like(n=12, d=4):
    w = synthetic.C1
    m0, C0 = model.cell_moments(d, w.alpha, w.beta, w.sigma, w.ell)
    L = model.default_L(C0)
    return m0, C0, L


def _mirror(F):
    n = F.shape[0]
    perm = np.array([0] + [n - i for i in range(1, n)])
    return F[np.ix_(*([perm] * F.ndim))]


def test_invariants_through_rk4():
    """Phi(0,t) = 1 (every term carries a factor a_k); Phi(c1,t) = Phi0(c1)
    (D1, D2 have zero column sums); Phi(-a) = conj Phi(a) on the mirrored
    grid; |Phi| <= 1 up to discretisation error."""
    d, n = 4, 12
    m0, C0, L = _c1_like(n, d)
    F0 = fullgrid.phi0_grid(m0, C0, n, L)
    F = fullgrid.solve(F0, 1e-3, 40, d, n, L, 0.05)
    c = n // 2
    assert abs(F[(c,) * d] - 1.0) < 1e-13
    for i in range(1, n):
        assert abs(F[(i,) * d] - F0[(i,) * d]) < 1e-13
    np.testing.assert_allclose(_mirror(F), F.conj(), atol=1e-13)
    assert np.abs(F).max() < 1.0 + 1e-3


@pytest.mark.parametrize("nonlinear", [True, False])
def test_phi_stays_zero_on_boundary_slot(nonlinear):
    d, n = 3, 10
    m0, C0, L = _c1_like(n, d)
    F = fullgrid.solve(fullgrid.phi0_grid(m0, C0, n, L), 1e-3, 5, d, n, L, 0.05, nonlinear)
    assert np.abs(F[0]).max() == 0 and np.abs(F[:, 0]).max() == 0 and np.abs(F[:, :, 0]).max() == 0


def test_linear_closed_form_second_order_in_da():
    """Nonlinear term off: full grid -> closed form, error ~ da^2."""
    d, nu, T, dt = 3, 0.3, 0.2, 0.01
    m0, C0 = model.cell_moments(d, (0.0,), (1.0,), 0.3, 1.0)
    L = model.default_L(C0)
    errs = []
    for n in (32, 64):
        a, _ = model.a_grid(n, L)
        F = fullgrid.solve(fullgrid.phi0_grid(m0, C0, n, L), dt, int(round(T / dt)), d, n, L, nu, nonlinear=False)
        idx = np.array([[n // 2 + n // 16, n // 2 - n // 8, n // 2 + n // 8]])
        errs.append(abs(F[tuple(idx.T)][0] - reference.closed_form(a[idx], m0, C0, nu, T)[0]))
    # pre-asymptotic at n = 16; from n = 32 on the ratio approaches 4
    assert errs[0] / errs[1] > 3.4 and errs[1] < 3e-3


def test_zero_viscosity_linear_is_stationary():
    """nu = 0 and nonlinear off: G = 0, Phi constant in time."""
    d, n = 3, 10
    m0, C0, L = _c1_like(n, d)
    F0 = fullgrid.phi0_grid(m0, C0, n, L)
    F = fullgrid.solve(F0, 0.1, 3, d, n, L, 0.0, nonlinear=False)
    assert np.abs(F - F0).max() == 0.0


def test_rk4_local_order_by_richardson():
    """LTE of one RK4 step against two half steps scales like dt^5."""
    d, n = 3, 16
    m0, C0, L = _c1_like(n, d)
    F0 = fullgrid.phi0_grid(m0, C0, n, L)
    errs = []
    for dt in (0.08, 0.04, 0.02):
        one = fullgrid.rk4_step(F0, dt, d, n, L, 0.05)
        two = fullgrid.rk4_step(fullgrid.rk4_step(F0, dt / 2, d, n, L, 0.05), dt / 2, d, n, L, 0.05)
        errs.append(np.abs(one - two).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 25 < r1 < 40 and 25 < r2 < 40


def test_fd_moments_of_gaussian_closed_form():
    """For Phi0 = exp(i a.m - a^T C a/2) the difference formulas have closed
    forms: mean_k = e^{-C_kk da^2/2} sin(m_k da)/da, second moments from the
    Gaussian values at (+-da, +-da); both tend to (m, C + m m^T)."""
    d, n = 3, 16
    m0, C0 = model.cell_moments(d, (0.2,), (1.0,), 0.3, 1.0)
    L = model.default_L(C0)
    _, da = model.a_grid(n, L)
    mean, cov = fullgrid.moments(fullgrid.phi0_grid(m0, C0, n, L), n, L)
    ph = lambda v: np.exp(1j * v @ m0 - 0.5 * v @ C0 @ v)
    e = np.eye(d) * da
    exp_mean = np.exp(-np.diag(C0) * da ** 2 / 2) * np.sin(m0 * da) / da
    np.testing.assert_allclose(mean, exp_mean, atol=1e-13)
    sec = np.zeros((d, d))
    for j in range(d):
        for k in range(d):
            if j == k:
                sec[j, k] = (-(ph(e[k]) - 2 + ph(-e[k])) / da ** 2).real
            else:
                sec[j, k] = (-(ph(e[j] + e[k]) - ph(e[j] - e[k]) - ph(-e[j] + e[k]) + ph(-e[j] - e[k])) / (4 * da ** 2)).real
    np.testing.assert_allclose(cov, sec - np.outer(exp_mean, exp_mean), atol=1e-12)
    # the O(da^2) bias shrinks as da halves (n = 32 -> 64; da ~ 1.4 -> 0.7)
    b = []
    for nn in (32, 64):
        mm, cc = fullgrid.moments(fullgrid.phi0_grid(m0, C0, nn, L), nn, L)
        b.append((np.abs(mm - m0).max(), np.abs(cc - C0).max()))
    assert b[0][0] / b[1][0] > 2.5 and b[0][1] / b[1][1] > 2.5


def test_monte_carlo_agrees_with_full_grid():
    """Nonlinear Burgers, d = 3: the full-grid Phi at a few points agrees with
    a 1e5-sample Monte-Carlo estimate of E[exp(i a.u(T))] within 4 standard
    errors plus the discretisation error (estimated from n -> 2n)."""
    d, nu, T, dt = 3, 0.05, 0.2, 0.005
    m0, C0 = model.cell_moments(d, (0.0,), (1.0,), 0.3, 1.0)
    L = model.default_L(C0)
    sols = {}
    for n in (32, 64):
        sols[n] = fullgrid.solve(fullgrid.phi0_grid(m0, C0, n, L), dt, int(round(T / dt)), d, n, L, nu)
    a32, _ = model.a_grid(32, L)
    idx32 = np.array([[17, 15, 16], [18, 18, 18], [16, 19, 14], [20, 13, 17]])
    idx64 = 2 * idx32  # same physical points on the finer grid: i64 - 32 = 2 (i32 - 16)
    pts = a32[idx32]
    z = synthetic.mc_gaussian_samples(d, 100000, seed=11)
    est, se_re, se_im, _, _ = reference.mc_charfun(pts, m0, C0, nu, T, dt / 4, z)
    fine = sols[64][tuple(idx64.T)]
    disc = np.abs(fine - sols[32][tuple(idx32.T)])
    assert np.all(np.abs(fine.real - est.real) <= 4 * se_re + disc + 1e-4)
    assert np.all(np.abs(fine.imag - est.imag) <= 4 * se_im + disc + 1e-4)
