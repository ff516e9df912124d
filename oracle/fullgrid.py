"""Full-grid solver (oracle; test infrastructure only).

The plain definition of the semi-discrete system Eq. (ode), df/dt = G(f), on
the whole n^d grid, for small d: the generator is applied as the sum over its
terms a_k (c_S S_j + c_D D_j) (see ``model.generator_terms``), each a matrix
acting on one or two axes of the array, and time integration is classical RK4
with no truncation (the increment function Psi of Eq. discrete-flow-intro).
"""
from __future__ import annotations

import numpy as np

from . import model


def apply_on_axis(M, F, axis):
    """(M acting on the given axis of F): out[..., i, ...] = sum_j M[i, j] F[..., j, ...]."""
    return np.moveaxis(np.tensordot(M, F, axes=([1], [axis])), 0, axis)


def apply_G(F, d, n, L, nu, nonlinear=True):
    """G F = sum over terms a_k (c_S d^2/da_j^2 + c_D d/da_j) F on the full
    grid (Eq. hyper1 for 1-D Burgers).  Pinned by the plane-wave symbol test,
    the mass and Phi(0)=1 invariants and the closed form."""
    A, D, S = model.mode_operators(n, L)
    terms = model.generator_terms(d, nu, nonlinear)
    SF = {j: apply_on_axis(S, F, j) for j in {t[1] for t in terms if t[2] != 0.0}}
    DF = {j: apply_on_axis(D, F, j) for j in {t[1] for t in terms if t[3] != 0.0}}
    out = np.zeros_like(F, dtype=complex)
    for k in range(d):
        inner = np.zeros_like(F, dtype=complex)
        for kk, j, cS, cD in terms:
            if kk != k:
                continue
            if cS != 0.0:
                inner += cS * SF[j]
            if cD != 0.0:
                inner += cD * DF[j]
        out += apply_on_axis(A, inner, k)
    return out


def rk4_step(F, dt, d, n, L, nu, nonlinear=True):
    """Classical RK4 increment for the linear, autonomous G."""
    g = lambda X: apply_G(X, d, n, L, nu, nonlinear)
    k1 = g(F)
    k2 = g(F + 0.5 * dt * k1)
    k3 = g(F + 0.5 * dt * k2)
    k4 = g(F + dt * k3)
    return F + (dt / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)


def solve(F0, dt, nsteps, d, n, L, nu, nonlinear=True):
    F = F0.copy()
    for _ in range(nsteps):
        F = rk4_step(F, dt, d, n, L, nu, nonlinear)
    return F


def phi0_grid(m0, C0, n, L):
    """Phi0(a) = exp(i a.m0 - a^T C0 a / 2) on the n^d grid, zero on every
    boundary slot (index 0 of any mode)."""
    d = len(m0)
    a, _ = model.a_grid(n, L)
    grids = np.meshgrid(*([a] * d), indexing="ij")
    X = np.stack(grids, axis=-1)  # (n,)*d + (d,)
    phase = X @ m0
    quad = np.einsum("...j,jk,...k->...", X, C0, X)
    F = np.exp(1j * phase - 0.5 * quad)
    for ax in range(d):
        idx = [slice(None)] * d
        idx[ax] = 0
        F[tuple(idx)] = 0.0
    return F


def moments(F, n, L):
    """Mean and covariance of u_bar from central differences of Phi at a = 0
    (Sec. 1: E[u] = (1/i) dPhi/dtheta at 0, E[u u] = (1/i^2) d^2Phi at 0).
    mean_k = Re[-i (Phi(+da e_k) - Phi(-da e_k)) / (2 da)];
    E[u_j u_k] = -mixed central difference (j != k), -second difference
    (j == k); cov = E[u u^T] - mean mean^T."""
    d = F.ndim
    _, da = model.a_grid(n, L)
    c = n // 2

    def at(offsets):
        idx = [c] * d
        for ax, o in offsets:
            idx[ax] += o
        return F[tuple(idx)]

    mean = np.zeros(d)
    second = np.zeros((d, d))
    for k in range(d):
        mean[k] = (-1j * (at([(k, 1)]) - at([(k, -1)])) / (2 * da)).real
    for j in range(d):
        for k in range(d):
            if j == k:
                v = -(at([(k, 1)]) - 2 * at([]) + at([(k, -1)])) / da ** 2
            else:
                v = -(at([(j, 1), (k, 1)]) - at([(j, 1), (k, -1)])
                      - at([(j, -1), (k, 1)]) + at([(j, -1), (k, -1)])) / (4 * da ** 2)
            second[j, k] = v.real
    return mean, second - np.outer(mean, mean)
