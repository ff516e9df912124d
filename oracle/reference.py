"""Exact and statistical references (oracle; test infrastructure only).

* ``closed_form``: with the nonlinear term switched off the u-dynamics are
  linear, du/dt = nu D2 u, so a Gaussian initial state stays Gaussian:
  m(t) = e^{t nu D2} m0, C(t) = e^{t nu D2} C0 e^{t nu D2^T} and
  Phi(a,t) = exp(i a.m(t) - a^T C(t) a / 2)  (continuous in a).
* ``mc_charfun``: Monte-Carlo estimate of E[exp(i a . u_bar(T))] from samples
  u_bar(0) ~ N(m0, C0) pushed through the discrete Burgers ODE with RK4 (the
  paper validates against Monte Carlo of the underlying Burgers equation,
  Sec. 5.1 "Numerical results").
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm

from . import model


def closed_form_moments(m0, C0, nu, t):
    d = len(m0)
    _, D2 = model.fd_matrices(d)
    E = expm(t * nu * D2)
    return E @ m0, E @ C0 @ E.T


def closed_form(points, m0, C0, nu, t):
    """Phi(a, t) at real points a (npts x d) for the linear dynamics."""
    m, C = closed_form_moments(m0, C0, nu, t)
    a = np.asarray(points, dtype=float)
    return np.exp(1j * (a @ m) - 0.5 * np.einsum("pj,jk,pk->p", a, C, a))


def burgers_rk4(u, T, dt, nu):
    """Integrate the discrete Burgers ODE du/dt = -1/2 D1(u o u) + nu D2 u for
    an ensemble u (nsamples x d) with classical RK4."""
    d = u.shape[1]
    D1, D2 = model.fd_matrices(d)
    f = lambda v: model.burgers_rhs(v, D1, D2, nu)
    nsteps = int(round(T / dt))
    for _ in range(nsteps):
        k1 = f(u)
        k2 = f(u + 0.5 * dt * k1)
        k3 = f(u + 0.5 * dt * k2)
        k4 = f(u + dt * k3)
        u = u + (dt / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return u


def mc_charfun(points, m0, C0, nu, T, dt, z):
    """E[exp(i a . u_bar(T))] at the given points from standard-normal draws
    z (nsamples x d), coloured with the Cholesky factor of C0.  Returns
    (estimate, standard error of the real part, of the imaginary part) and
    the sample mean and covariance of u_bar(T)."""
    Lc = np.linalg.cholesky(C0 + 1e-14 * np.eye(len(m0)))
    u0 = m0[None, :] + z @ Lc.T
    uT = burgers_rk4(u0, T, dt, nu)
    a = np.asarray(points, dtype=float)
    ph = np.exp(1j * (uT @ a.T))  # (nsamples, npts)
    est = ph.mean(axis=0)
    ns = ph.shape[0]
    se_re = ph.real.std(axis=0) / np.sqrt(ns)
    se_im = ph.imag.std(axis=0) / np.sqrt(ns)
    return est, se_re, se_im, uT.mean(axis=0), np.cov(uT.T)
