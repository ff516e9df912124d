"""The CDF equation of the stochastic Burgers equation (oracle; test
infrastructure only).

The paper's own experiment (Sec. 5, Eq. cdf-burgers) solves for the joint CDF
F(u_1..u_N, t) of the grid values of the Burgers solution instead of the
characteristic function.  With the reaction term off (alpha = 0, the
workload of Sec. 5.1) the equation reads

  dF/dt = sum_{i,j} (u_i D1_ij u_j - gamma D2_ij u_j) dF/du_i
          - sum_{i != j} (D1_ij u_i - gamma D2_ij) int_{-inf}^{u_j} dF/du_i du_j,

D1, D2 the periodic second-order difference matrices in x (model.fd_matrices,
N = d grid points on [0, 2 pi)).  Discretisation as stated under the
equation: each u_j on an evenly spaced grid of n points over the box
[-U, U] (U = 1.3), centred second-order differences for d/du with the
outflow condition dF/du = 0 on the boundary, the trapezoidal rule for the
integrals (taken from the box's lower edge, where F vanishes), and the
initial state a product of zero-mean Gaussian CDFs g(u) = (1 + erf(u /
(sigma sqrt 2))) / 2 with sigma = 0.25.

``apply_G`` states the operator term by term as printed (the plain
definition on the full grid, d <= 4); ``mpo_blocks`` is its tensor-train
operator, pinned against ``apply_G``.  Readings (the paper is silent): the
grid includes both box edges (u_k = -U + k du, du = 2U/(n-1)); the
trapezoidal integral at node k runs over nodes 0..k; the numerical diffusion
the paper adds to stabilise explicit schemes is left out (its coefficient is
not given).

Pinned by tests/test_oracle_cdf.py: the MPO against apply_G; the corner
value F(U, .., U) conserved exactly; with the D1 terms off the dynamics are
linear, u' = gamma D2 u, so F(t) is the normal CDF with covariance
sigma^2 E E^T, E = exp(t gamma D2), reached at second order in du; the full
equation against Monte Carlo of the Burgers ODE u' = -u o (D1 u) +
gamma D2 u (the velocity field of Eq. pdf-burgers); local truncation errors
of orders 2 and 3 for the truncated Euler and midpoint schemes by Richardson
extrapolation (Sec. 5.1's order study).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from . import model

BOX = 1.3
SIGMA0 = 0.25


def u_grid(n: int, U: float = BOX):
    """u_k = -U + k du, du = 2U / (n - 1), k = 0..n-1 (both edges on the grid)."""
    du = 2.0 * U / (n - 1)
    return -U + np.arange(n) * du, du


def mode_operators(n: int, U: float = BOX):
    """Per-variable n x n operators: A = diag(u_k); D = centred first
    difference, rows 0 and n-1 zero (outflow: dF/du = 0 on the boundary);
    J = trapezoidal integral from the lower edge, (J g)_k =
    du (g_0 / 2 + g_1 + ... + g_{k-1} + g_k / 2), (J g)_0 = 0."""
    u, du = u_grid(n, U)
    A = np.diag(u)
    D = np.zeros((n, n))
    for k in range(1, n - 1):
        D[k, k + 1] = 1.0 / (2 * du)
        D[k, k - 1] = -1.0 / (2 * du)
    J = np.zeros((n, n))
    for k in range(1, n):
        J[k, 0] = du / 2
        J[k, 1:k] = du
        J[k, k] = du / 2
    return A, D, J


def apply_on_axis(M, F, axis):
    return np.moveaxis(np.tensordot(M, F, axes=([1], [axis])), 0, axis)


def apply_G(F, d: int, n: int, gamma: float, U: float = BOX, nonlinear: bool = True):
    """The right-hand side of Eq. (cdf-burgers), alpha = 0, on the full grid,
    term by term: for every i, dF/du_i by D on axis i; then
    sum_j (u_i D1_ij u_j - gamma D2_ij u_j) dF/du_i and, for j != i,
    -(D1_ij u_i - gamma D2_ij) J_j dF/du_i.  nonlinear=False drops every D1
    term (the linear dynamics u' = gamma D2 u)."""
    A, D, J = mode_operators(n, U)
    D1, D2 = model.fd_matrices(d)
    if not nonlinear:
        D1 = np.zeros_like(D1)
    out = np.zeros(F.shape, dtype=np.result_type(F, float))
    for i in range(d):
        dF = apply_on_axis(D, F, i)
        for j in range(d):
            if D1[i, j] == 0.0 and D2[i, j] == 0.0:
                continue
            # (u_i D1_ij u_j - gamma D2_ij u_j) dF/du_i
            t = apply_on_axis(A, dF, j)          # u_j dF/du_i
            out += D1[i, j] * apply_on_axis(A, t, i) - gamma * D2[i, j] * t
            if j != i:
                # -(D1_ij u_i - gamma D2_ij) int^{u_j} dF/du_i du_j
                s = apply_on_axis(J, dF, j)
                out -= D1[i, j] * apply_on_axis(A, s, i) - gamma * D2[i, j] * s
    return out


def mpo_blocks(d: int, n: int, gamma: float, U: float = BOX, nonlinear: bool = True):
    """Tensor-train operator of apply_G.  Collecting the terms of each
    ordered neighbour pair (i, j) gives [D1_ij (A D) - gamma D2_ij D]_i
    (x) (A - J)_j, and the diagonal j = i gives (2 gamma / h^2) (A D)_i.
    With K = A - J, P+ = (A D)/(2h) - (gamma/h^2) D and
    P- = -(A D)/(2h) - (gamma/h^2) D, each cyclic pair (m, m+1)
    contributes P+_m (x) K_{m+1} + K_m (x) P-_{m+1}: the bond states of the
    characteristic-function operator (model.mpo_blocks) with A, P, Q, A
    replaced by P+, K, K, P-."""
    A, D, J = mode_operators(n, U)
    h = model.cell_width(d)
    c = 1.0 / (2 * h) if nonlinear else 0.0
    e = gamma / h ** 2
    I = np.eye(n)
    K = A - J
    AD = A @ D
    Pp = c * AD - e * D
    Pm = -c * AD - e * D
    Z = 2.0 * e * AD
    W = []
    for k in range(d):
        if k == 0:
            blocks = {(0, 0): I, (0, 1): Pp, (0, 2): K, (0, 3): Z, (0, 4): K, (0, 5): Pm}
        elif k == d - 1:
            blocks = {(0, 0): Z, (1, 0): K, (2, 0): Pm, (3, 0): I, (4, 0): Pp, (5, 0): K}
        else:
            blocks = {(0, 0): I, (0, 1): Pp, (0, 2): K, (0, 3): Z,
                      (1, 3): K, (2, 3): Pm, (3, 3): I, (4, 4): I, (5, 5): I}
        W.append({key: np.asarray(val, dtype=complex) for key, val in blocks.items()})
    return W


def gaussian_cdf(u, sigma: float = SIGMA0):
    """g(u) = (1 + erf(u / (sigma sqrt 2))) / 2."""
    return 0.5 * (1.0 + erf(np.asarray(u, dtype=float) / (sigma * np.sqrt(2.0))))


def initial_tt(d: int, n: int, sigma: float = SIGMA0, U: float = BOX, mu=None):
    """F(u, 0) = prod_k g(u_k - mu_k) (mu = 0: the paper's initial state): a
    rank-1 TT (complex cores, zero imaginary part)."""
    u, _ = u_grid(n, U)
    mu = np.zeros(d) if mu is None else np.asarray(mu, dtype=float)
    return [np.asfortranarray(gaussian_cdf(u - mu[k], sigma).astype(complex).reshape(1, n, 1)) for k in range(d)]


def initial_grid(d: int, n: int, sigma: float = SIGMA0, U: float = BOX, mu=None):
    u, _ = u_grid(n, U)
    mu = np.zeros(d) if mu is None else np.asarray(mu, dtype=float)
    F = gaussian_cdf(u - mu[0], sigma)
    for k in range(1, d):
        F = np.multiply.outer(F, gaussian_cdf(u - mu[k], sigma))
    return F


# ---- full-grid time steps (no truncation) -----------------------------------

def euler_step(F, dt, G):
    """f + dt G(f)."""
    return F + dt * G(F)


def midpoint_step(F, dt, G):
    """f + dt G(f + dt/2 G(f)) (explicit midpoint)."""
    return F + dt * G(F + 0.5 * dt * G(F))


def rk4_step(F, dt, G):
    k1 = G(F)
    k2 = G(F + 0.5 * dt * k1)
    k3 = G(F + 0.5 * dt * k2)
    k4 = G(F + dt * k3)
    return F + (dt / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)


def burgers_velocity(u, gamma: float, nonlinear: bool = True):
    """v_i = -u_i (D1 u)_i + gamma (D2 u)_i for an ensemble u (nsamples x
    d): the velocity field of Eq. (pdf-burgers) with R = 0."""
    d = u.shape[1]
    D1, D2 = model.fd_matrices(d)
    v = gamma * u @ D2.T
    if nonlinear:
        v = v - u * (u @ D1.T)
    return v


def mc_cdf(points, u0, gamma: float, T: float, dt: float, nonlinear: bool = True):
    """Empirical CDF at the given points (npts x d) of the samples u0
    (nsamples x d) pushed to time T by RK4 on u' = burgers_velocity(u),
    with its standard error."""
    u = np.array(u0, dtype=float)
    f = lambda x: burgers_velocity(x, gamma, nonlinear)
    # a sample far out in the tail may blow up in finite time (the
    # non-conservative flux is quadratic); it leaves the box and never
    # counts as <= a point of it
    with np.errstate(over="ignore", invalid="ignore"):
        for _ in range(int(round(T / dt))):
            k1 = f(u)
            k2 = f(u + 0.5 * dt * k1)
            k3 = f(u + 0.5 * dt * k2)
            k4 = f(u + dt * k3)
            u = u + (dt / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    u = np.where(np.isfinite(u), u, np.inf)
    ind = np.all(u[:, None, :] <= np.asarray(points)[None, :, :], axis=2).astype(float)
    p = ind.mean(axis=0)
    return p, np.sqrt(np.maximum(p * (1 - p), 1e-300) / u.shape[0])
