"""Pins of oracle.model against facts fixed outside the oracle: Fourier
symbols of the difference stencils, exact antiderivatives, scipy quadrature,
and a brute-force expansion of the MPO into operator terms."""
import itertools

import numpy as np
import pytest
from scipy import integrate

from oracle import model


@pytest.mark.parametrize("d", [3, 4, 7, 16])
def test_fd_symbols_on_fourier_modes(d):
    """On f_j = exp(i q j h) the periodic stencils act as multiplication by
    i sin(qh)/h (D1) and -4 sin^2(qh/2)/h^2 (D2)."""
    D1, D2 = model.fd_matrices(d)
    h = 2 * np.pi / d
    j = np.arange(d)
    for q in range(d):
        f = np.exp(1j * q * j * h)
        np.testing.assert_allclose(D1 @ f, 1j * np.sin(q * h) / h * f, atol=1e-12)
        np.testing.assert_allclose(D2 @ f, -4 * np.sin(q * h / 2) ** 2 / h ** 2 * f, atol=1e-10)


def test_fd_needs_three_cells():
    with pytest.raises(ValueError):
        model.fd_matrices(2)


def test_mode_operators_on_plane_waves():
    """Interior rows of D and S act on exp(i w a) by their symbols; the
    boundary slot 0 has zero row and column; A is diag(a) with a_{n/2} = 0."""
    n, L = 20, 3.0
    A, D, S = model.mode_operators(n, L)
    a, da = model.a_grid(n, L)
    assert a[n // 2] == 0.0 and np.isclose(a[0], -L) and np.isclose(da, 2 * L / n)
    w = 0.7
    f = np.exp(1j * w * a)
    inner = slice(2, n - 1)
    np.testing.assert_allclose((D @ f)[inner], (1j * np.sin(w * da) / da * f)[inner], atol=1e-12)
    np.testing.assert_allclose((S @ f)[inner], (-4 * np.sin(w * da / 2) ** 2 / da ** 2 * f)[inner], atol=1e-12)
    for M in (A, D, S):
        assert not M[0, :].any() and not M[:, 0].any()
    np.testing.assert_allclose(np.diag(A)[1:], a[1:])


def test_mirror_symmetry_of_mode_operators():
    """The mirror J: i -> n - i (slot 0 fixed) maps a -> -a, so
    J A J = -A, J D J = -D, J S J = S."""
    n, L = 16, 2.5
    A, D, S = model.mode_operators(n, L)
    J = np.zeros((n, n))
    J[0, 0] = 1
    for i in range(1, n):
        J[i, n - i] = 1
    np.testing.assert_allclose(J @ A @ J, -A, atol=1e-14)
    np.testing.assert_allclose(J @ D @ J, -D, atol=1e-14)
    np.testing.assert_allclose(J @ S @ J, S, atol=1e-14)


def test_cell_mean_matches_exact_antiderivative():
    d = 9
    alpha, beta = (0.3, -0.5, 0.2), (1.0, 0.25, -0.7)
    m0, _ = model.cell_moments(d, alpha, beta, 0.3, 1.0)
    h = 2 * np.pi / d
    x0, x1 = np.arange(d) * h, (np.arange(d) + 1) * h
    exact = np.zeros(d)
    for m, (al, be) in enumerate(zip(alpha, beta), start=1):
        exact += al * (np.sin(m * x1) - np.sin(m * x0)) / m
        exact += be * (np.cos(m * x0) - np.cos(m * x1)) / m
    np.testing.assert_allclose(m0, exact / h, atol=1e-13)


@pytest.mark.parametrize("jk", [(0, 0), (0, 1), (2, 5), (1, 6)])
def test_cell_covariance_matches_dblquad(jk):
    d, sigma, ell = 7, 0.4, 0.7
    _, C0 = model.cell_moments(d, (0.0,), (1.0,), sigma, ell)
    h = 2 * np.pi / d
    j, k = jk
    K = lambda y, x: sigma ** 2 * np.exp(-2 * np.sin((x - y) / 2) ** 2 / ell ** 2)
    val, _ = integrate.dblquad(K, j * h, (j + 1) * h, k * h, (k + 1) * h, epsabs=1e-13, epsrel=1e-12)
    assert abs(C0[j, k] - val / h ** 2) < 1e-11


def test_covariance_is_psd_and_limits():
    _, C0 = model.cell_moments(12, (0.0,), (1.0,), 0.5, 0.5)
    assert np.allclose(C0, C0.T)
    assert np.linalg.eigvalsh(C0).min() > -1e-12
    # very long correlation length: every cell sees the same value sigma^2
    _, Cl = model.cell_moments(6, (0.0,), (1.0,), 0.3, 1e4)
    np.testing.assert_allclose(Cl, 0.09 * np.ones((6, 6)), rtol=1e-6)


def _dense_from_terms(d, n, L, nu, nonlinear):
    """The generator as a dense n^d x n^d matrix, from its term list."""
    A, D, S = model.mode_operators(n, L)
    I = np.eye(n)
    out = np.zeros((n ** d, n ** d), dtype=complex)
    for k, j, cS, cD in model.generator_terms(d, nu, nonlinear):
        ops = [I] * d
        inner = cS * S + cD * D
        if j == k:
            ops[k] = A @ inner
        else:
            ops[k], ops[j] = A, inner
        M = np.ones((1, 1))
        for o in ops:  # first mode slowest (C order of the full tensor)
            M = np.kron(M, o)
        out += M
    return out


def _dense_from_mpo(d, n, L, nu, nonlinear):
    """Brute-force expansion of the MPO: sum over every bond-state path."""
    W = model.mpo_blocks(d, n, L, nu, nonlinear)
    bond = model.mpo_bond_dims(d)
    out = np.zeros((n ** d, n ** d), dtype=complex)
    for path in itertools.product(*[range(b) for b in bond[1:-1]]):
        states = (0,) + path + (0,)
        ops = []
        for k in range(d):
            key = (states[k], states[k + 1])
            if key not in W[k]:
                break
            ops.append(W[k][key])
        else:
            M = np.ones((1, 1))
            for o in ops:
                M = np.kron(M, o)
            out += M
    return out


@pytest.mark.parametrize("d,nonlinear", [(3, True), (4, True), (4, False), (5, True)])
def test_mpo_expands_to_generator_terms(d, nonlinear):
    n, L, nu = 4, 1.7, 0.3
    Gt = _dense_from_terms(d, n, L, nu, nonlinear)
    Gm = _dense_from_mpo(d, n, L, nu, nonlinear)
    np.testing.assert_allclose(Gm, Gt, atol=1e-12 * np.abs(Gt).max())
