"""Surrogate network reference (oracle; test infrastructure only).

A plain float64 numpy statement of the small multilayer perceptron that maps
the parameters of a Gaussian initial state (nu, sigma, ell, Fourier
coefficients of the mean, horizon T) to the mean and covariance of the cell
averages at time T.  The paper has no such network: it is the learned
surrogate added on top of the solver, so the passages followed here are the
textbook definitions named in each function (GELU of Hendrycks & Gimpel, 2016;
Adam of Kingma & Ba, 2015; mean-squared error and the chain rule).

Parameter layout of one member (shared with nothing; the CUDA library states
the same layout in its header): for each linear layer l = 0..depth with
widths dims = [n_in, width x depth, n_out], the weight W_l (out x in,
row-major) followed by the bias b_l (out).  An ensemble is an array
[members][P].

Pinned by (tests/test_oracle_mlp.py): GELU at points where the normal CDF is
known, its odd part GELU(x) - GELU(-x) = x and its slope 1/2 at 0; the
backward pass against central finite differences of the forward pass; a
network without hidden layers against the closed-form least-squares gradient;
the first Adam step against its closed form -lr g / (|g| + eps) and the
second and third steps against the recursions written out by hand with their
bias corrections; the ensemble bound of a two-member ensemble against the
spread |y_1 - y_2| / 2 worked by hand; the column statistics on constant,
two-valued and affine columns.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf as _erf


def layer_dims(n_in: int, width: int, depth: int, n_out: int):
    return [n_in] + [width] * depth + [n_out]


def layout(n_in: int, width: int, depth: int, n_out: int):
    """[(w_off, b_off, fan_in, fan_out)] per layer and the member size P."""
    dims = layer_dims(n_in, width, depth, n_out)
    out, off = [], 0
    for fi, fo in zip(dims[:-1], dims[1:]):
        out.append((off, off + fi * fo, fi, fo))
        off += fi * fo + fo
    return out, off


def unpack(params, n_in, width, depth, n_out):
    lay, _ = layout(n_in, width, depth, n_out)
    return [(params[w:w + fi * fo].reshape(fo, fi), params[b:b + fo]) for w, b, fi, fo in lay]


_SQRT1_2 = 1.0 / math.sqrt(2.0)


def gelu(z):
    """GELU(z) = z Phi(z), Phi the standard normal CDF written with erf."""
    z = np.asarray(z, dtype=float)
    return 0.5 * z * (1.0 + _erf(z * _SQRT1_2))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    z = np.asarray(z, dtype=float)
    return 0.5 * (1.0 + _erf(z * _SQRT1_2)) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, X, n_in, width, depth, n_out):
    """Returns (Y, cache): hidden layers z = W h + b, h = GELU(z); the last
    layer is linear.  X: batch x n_in (already normalised)."""
    layers = unpack(np.asarray(params, dtype=float), n_in, width, depth, n_out)
    h = np.asarray(X, dtype=float)
    cache = []
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        cache.append((h, z))
        h = gelu(z) if l < len(layers) - 1 else z
    return h, cache


def loss_and_grad(params, X, T, n_in, width, depth, n_out):
    """Mean-squared error over batch and outputs, and its gradient with
    respect to the packed parameters (chain rule, layer by layer)."""
    params = np.asarray(params, dtype=float)
    Y, cache = forward(params, X, n_in, width, depth, n_out)
    T = np.asarray(T, dtype=float)
    B, O = Y.shape
    loss = float(np.mean((Y - T) ** 2))
    g = 2.0 * (Y - T) / (B * O)
    layers = unpack(params, n_in, width, depth, n_out)
    lay, P = layout(n_in, width, depth, n_out)
    grad = np.zeros(P)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        h, z = cache[l]
        if l < len(layers) - 1:
            g = g * gelu_grad(z)
        w_off, b_off, fi, fo = lay[l]
        grad[w_off:w_off + fi * fo] = (g.T @ h).ravel()
        grad[b_off:b_off + fo] = g.sum(axis=0)
        g = g @ W
    return loss, grad


def adam_step(w, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) at step t >= 1; returns the
    new (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def column_stats(A):
    """Per-column mean and population standard deviation (1 where a column
    is constant), used to normalise inputs and targets."""
    A = np.asarray(A, dtype=float)
    mu = A.mean(axis=0)
    sd = np.sqrt(((A - mu) ** 2).mean(axis=0))
    return mu, np.where(sd > 0, sd, 1.0)


def predict(ensemble, X, xstats, ystats, kappa, n_in, width, depth, n_out, base=None, scale=None):
    """Ensemble prediction in physical units and its error bound.

    Member m answers y_m = base + scale (mu_y + s_y net_m((x - mu_x) / s_x))
    (base 0 and scale 1 when absent); the answer is the member mean ybar and
    the bound is kappa ||spread||_2 / ||ybar||_2 with spread the per-output
    standard deviation over members."""
    Xn = (np.asarray(X, dtype=float) - xstats[0]) / xstats[1]
    b0 = 0.0 if base is None else np.asarray(base, dtype=float)
    sc = 1.0 if scale is None else np.asarray(scale, dtype=float)[:, None]
    Ys = np.stack([b0 + sc * (ystats[0] + ystats[1] * forward(p, Xn, n_in, width, depth, n_out)[0])
                   for p in ensemble])
    ybar = Ys.mean(axis=0)
    spread = np.sqrt(((Ys - ybar) ** 2).mean(axis=0))
    bound = kappa * np.linalg.norm(spread, axis=1) / np.linalg.norm(ybar, axis=1)
    return ybar, bound
