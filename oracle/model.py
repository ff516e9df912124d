"""The discretised Burgers-Hopf PDE (oracle; test infrastructure only).

Physics (Sec. 5, Eq. burgers-rxn with reaction alpha = 0, and Eq. BHfde): the
characteristic function Phi(a,t) = E[exp(i a . u_bar(t))] of the cell averages
u_bar of the periodic Burgers solution.  The test function theta is projected
on d cell-indicator functions (Eq. sense), x-derivatives become second-order
periodic finite differences (the choice stated under Eq. pdf-burgers), and the
FDE becomes the linear PDE of the form of Eq. (hyper1)

    dPhi/dt = sum_k a_k sum_j [ (i/2) D1[k,j] d^2Phi/da_j^2 + nu D2[k,j] dPhi/da_j ].

Each a_j is discretised on a uniform grid (Eq. tt / Eq. ode); the tensor
product structure lets the generator act mode by mode.

Readings where the paper is silent: the a-grid is
a_i = (i - n/2) da, da = 2L/n, i = 0..n-1, with slot 0 (a = -L) held at zero
and a = +L an implicit zero ghost; the covariance kernel is the periodic
squared exponential sigma^2 exp(-2 sin^2((x-y)/2)/ell^2).
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- x grid ----

def cell_width(d: int) -> float:
    """h = 2 pi / d: d cells I_k = [k h, (k+1) h) on the periodic [0, 2 pi)."""
    return 2.0 * np.pi / d


def fd_matrices(d: int):
    """Periodic second-order difference matrices in x (Eq. pdf-burgers text:
    'second-order finite difference matrix on a periodic domain').

    D1[k, k+1] = +1/(2h), D1[k, k-1] = -1/(2h);
    D2[k, k] = -2/h^2, D2[k, k+-1] = 1/h^2; indices mod d.  Needs d >= 3.
    Pinned by tests/test_oracle_model.py (action on trigonometric grid
    functions)."""
    if d < 3:
        raise ValueError("the central x-stencil needs d >= 3 cells")
    h = cell_width(d)
    D1 = np.zeros((d, d))
    D2 = np.zeros((d, d))
    for k in range(d):
        D1[k, (k + 1) % d] += 1.0 / (2 * h)
        D1[k, (k - 1) % d] -= 1.0 / (2 * h)
        D2[k, k] += -2.0 / h ** 2
        D2[k, (k + 1) % d] += 1.0 / h ** 2
        D2[k, (k - 1) % d] += 1.0 / h ** 2
    return D1, D2


def burgers_rhs(u, D1, D2, nu):
    """Discrete conservative Burgers on cell averages:
    du/dt = -1/2 D1 (u o u) + nu D2 u (Eq. burgers-rxn with alpha = 0 in the
    flux form that Eq. BHfde's (i/2) d/dx delta^2/delta theta^2 term encodes).
    Works on arrays of shape (..., d)."""
    return -0.5 * (u * u) @ D1.T + nu * (u @ D2.T)


# ---------------------------------------------------------------- a grid ----

def a_grid(n: int, L: float):
    """a_i = (i - n/2) da, da = 2L/n, i = 0..n-1; a = 0 is index n/2."""
    da = 2.0 * L / n
    return (np.arange(n) - n // 2) * da, da


def mode_operators(n: int, L: float):
    """Per-mode n x n operators on the a-grid of one variable:
    A = diag(a_i); D = central first difference (+-1/(2 da) off the
    diagonal); S = second difference (1, -2, 1)/da^2.  Row and column of the
    boundary slot 0 are zero, index n is an implicit zero ghost (Phi = 0 at
    the boundary of [-L, L])."""
    a, da = a_grid(n, L)
    A = np.diag(a).astype(float)
    D = np.zeros((n, n))
    S = np.zeros((n, n))
    for i in range(n):
        S[i, i] = -2.0 / da ** 2
        if i + 1 < n:
            D[i, i + 1] = 1.0 / (2 * da)
            S[i, i + 1] = 1.0 / da ** 2
        if i - 1 >= 0:
            D[i, i - 1] = -1.0 / (2 * da)
            S[i, i - 1] = 1.0 / da ** 2
    for M in (A, D, S):
        M[0, :] = 0.0
        M[:, 0] = 0.0
    return A, D, S


def default_L(C0) -> float:
    """L = sqrt(36.8 / min_k C0_kk): Phi0 ~ exp(-18.4) ~ 1e-8 at the edge of
    the box along the narrowest marginal."""
    return float(np.sqrt(36.8 / np.min(np.diag(C0))))


# ------------------------------------------------------------- generator ----

def generator_terms(d: int, nu: float, nonlinear: bool = True):
    """The generator as a list of (k, j, c_S, c_D): the term
    a_k (c_S d^2/da_j^2 + c_D d/da_j), from Eq. (hyper1) specialised to 1-D
    Burgers: c_S = (i/2) D1[k,j], c_D = nu D2[k,j]."""
    D1, D2 = fd_matrices(d)
    terms = []
    for k in range(d):
        for j in range(d):
            cS = 0.5j * D1[k, j] if nonlinear else 0.0
            cD = nu * D2[k, j]
            if cS != 0.0 or cD != 0.0:
                terms.append((k, j, cS, cD))
    return terms


def mpo_blocks(d: int, n: int, L: float, nu: float, nonlinear: bool = True):
    """Matrix-product-operator form of the generator: W[k] is a dict
    {(alpha, beta): n x n complex matrix} of the non-zero blocks of site k.

    Bond states: 0 idle, 1 'A placed, P pending', 2 'Q placed, A pending',
    3 done, 4 wrap 'P at site 1, A pending at site d', 5 wrap 'A at site 1,
    Q pending at site d'.  With c = i/(4h) (0 when the nonlinear term is off)
    and e = nu/h^2: P = cS + eD, Q = -cS + eD, Z = -2e A D.  Each cyclic
    neighbour pair (m, m+1) contributes A_m (x) P_{m+1} + Q_m (x) A_{m+1},
    each site k contributes Z_k.  Site 1 is a row (alpha = 0), site d a
    column (beta = 0).  Pinned against the full-grid definition
    (tests/test_oracle_tt.py::test_apply_matches_fullgrid)."""
    A, D, S = mode_operators(n, L)
    h = cell_width(d)
    c = 1j / (4 * h) if nonlinear else 0.0
    e = nu / h ** 2
    I = np.eye(n)
    I[0, 0] = 1.0  # identity keeps the (zero) boundary slot unchanged
    P = c * S + e * D
    Q = -c * S + e * D
    Z = -2.0 * e * (A @ D)
    W = []
    for k in range(d):
        if k == 0:
            blocks = {(0, 0): I, (0, 1): A, (0, 2): Q, (0, 3): Z,
                      (0, 4): P, (0, 5): A}
        elif k == d - 1:
            blocks = {(0, 0): Z, (1, 0): P, (2, 0): A, (3, 0): I,
                      (4, 0): A, (5, 0): Q}
        else:
            blocks = {(0, 0): I, (0, 1): A, (0, 2): Q, (0, 3): Z,
                      (1, 3): P, (2, 3): A, (3, 3): I, (4, 4): I, (5, 5): I}
        W.append({key: np.asarray(val, dtype=complex) for key, val in blocks.items()})
    return W


def mpo_bond_dims(d: int):
    """(1, 6, 6, ..., 6, 1): left/right MPO bond dimension of each site."""
    return [1] + [6] * (d - 1) + [1]


# ------------------------------------------------------- initial state ----

def gauss_legendre(q: int):
    """Nodes and weights on [0, 1] (numpy's Legendre quadrature)."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def mean_function(x, alpha, beta):
    """u0 mean: sum_m alpha_m cos(m x) + beta_m sin(m x), m = 1, 2, ..."""
    x = np.asarray(x, dtype=float)
    out = np.zeros_like(x)
    for m, (al, be) in enumerate(zip(alpha, beta), start=1):
        out = out + al * np.cos(m * x) + be * np.sin(m * x)
    return out


def periodic_se_kernel(x, y, sigma, ell):
    """sigma^2 exp(-2 sin^2((x - y)/2) / ell^2) (periodic squared
    exponential covariance of u0)."""
    return sigma ** 2 * np.exp(-2.0 * np.sin(0.5 * (x - y)) ** 2 / ell ** 2)


def cell_moments(d: int, alpha, beta, sigma: float, ell: float, q: int = 12):
    """Projection of the Gaussian initial state on the cell-indicator basis
    phi_k = 1_{I_k}/h (Eq. sense): m0_k = (1/h) int_{I_k} mu,
    C0_jk = (1/h^2) int_{I_j} int_{I_k} K, by q-point tensor Gauss-Legendre
    per cell.  Pinned by tests/test_oracle_model.py (exact antiderivatives
    for m0, scipy dblquad for C0)."""
    h = cell_width(d)
    t, w = gauss_legendre(q)
    xs = (np.arange(d)[:, None] + t[None, :]) * h  # (d, q) nodes per cell
    m0 = (mean_function(xs, alpha, beta) * w[None, :]).sum(axis=1)
    K = periodic_se_kernel(xs[:, None, :, None], xs[None, :, None, :], sigma, ell)
    C0 = np.einsum("jkab,a,b->jk", K, w, w)
    C0 = 0.5 * (C0 + C0.T)
    return m0, C0
