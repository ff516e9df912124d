"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This module holds workload parameters and random-number generation only.  It
contains none of the method's arithmetic (no operator, no rounding, no
quadrature): both the CPU oracle and the CUDA path receive what is made here
as plain inputs.

Workloads (all synthetic; the paper's own runs start from Gaussian random
initial states of the Burgers equation, Sec. 5 "Burgers-Hopf FDE"):

* ``C1`` d=4, n=24, nu=0.05, mean sin x, sigma=0.3, ell=1.0, dt=1e-3, T=0.5,
  rank cap 16, tol 1e-10.
* ``C2`` d=16, n=64, nu=0.02, mean sin x + 0.5 cos 2x, sigma=0.4, ell=0.7,
  dt=5e-4, T=1.0, rank cap 32, tol 1e-9.
* ``C3`` d=32, n=128, nu=0.01, mean sin x + 0.5 cos 2x, sigma=0.5, ell=0.5,
  rank cap 64, tol 1e-7.
* ``C4`` ensemble generator: d in {8..48}, n in {64,96,128}, nu~U[0.01,0.1],
  sigma~U[0.1,0.5], ell~U[0.3,2.0], mean = 4 random Fourier modes with
  amplitudes ~ N(0, 0.5^2).
* ``surrogate_member`` the C4 parameter draw on the C1 grid (d=4, n=24,
  rank cap 16, tol 1e-10) with dt=1e-2: the training and held-out solves of
  the learned surrogate, plus the network's random initial parameters and
  batch indices.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    """Parameters of one solve.  ``alpha[m-1]``/``beta[m-1]`` are the cos/sin
    amplitudes of Fourier mode m of the initial mean u0(x)."""

    name: str
    d: int
    n: int
    nu: float
    sigma: float
    ell: float
    alpha: tuple = field(default_factory=tuple)
    beta: tuple = field(default_factory=tuple)
    dt: float = 1e-3
    T: float = 0.0
    cap: int = 16
    tol: float = 1e-10
    nonlinear: bool = True

    @property
    def steps(self) -> int:
        return int(round(self.T / self.dt)) if self.T > 0 else 0

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


C1 = Workload("C1", d=4, n=24, nu=0.05, sigma=0.3, ell=1.0,
              alpha=(0.0,), beta=(1.0,), dt=1e-3, T=0.5, cap=16, tol=1e-10)
C2 = Workload("C2", d=16, n=64, nu=0.02, sigma=0.4, ell=0.7,
              alpha=(0.0, 0.5), beta=(1.0, 0.0), dt=5e-4, T=1.0, cap=32,
              tol=1e-9)
# C3 gives no horizon; dt is chosen for explicit-RK4 stability at this size.
C3 = Workload("C3", d=32, n=128, nu=0.01, sigma=0.5, ell=0.5,
              alpha=(0.0, 0.5), beta=(1.0, 0.0), dt=1.2e-5, T=0.0, cap=64,
              tol=1e-7)

WORKLOADS = {"C1": C1, "C2": C2, "C3": C3}


def ensemble_member(seed: int) -> Workload:
    """One draw of the C4 ensemble generator (seeded)."""
    rng = np.random.default_rng(seed)
    d = int(rng.integers(8, 49))
    n = int(rng.choice([64, 96, 128]))
    nu = float(rng.uniform(0.01, 0.1))
    sigma = float(rng.uniform(0.1, 0.5))
    ell = float(rng.uniform(0.3, 2.0))
    alpha = tuple(float(x) for x in rng.normal(0.0, 0.5, 4))
    beta = tuple(float(x) for x in rng.normal(0.0, 0.5, 4))
    return Workload(f"C4[{seed}]", d=d, n=n, nu=nu, sigma=sigma, ell=ell,
                    alpha=alpha, beta=beta, dt=1e-5, cap=64, tol=1e-7)


def random_tt_cores(d: int, n: int, ranks, seed: int, scale: float = 1.0):
    """Complex Gaussian TT cores C_k of shape (r_{k-1}, n, r_k), returned as
    numpy arrays in the paper's column-major core layout
    C[i,j,k] = v[i + a*j + a*b*k] (Fortran order)."""
    rng = np.random.default_rng(seed)
    ranks = list(ranks)
    assert len(ranks) == d + 1 and ranks[0] == 1 and ranks[-1] == 1
    cores = []
    for k in range(d):
        shape = (ranks[k], n, ranks[k + 1])
        c = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
        c *= scale / np.sqrt(2.0 * ranks[k] * n)
        cores.append(np.asfortranarray(c))
    return cores


def saturated_tt_cores(d: int, n: int, r: int, seed: int = 0):
    """Deterministic synthetic TT with every interior rank equal to
    min(r, n^k, n^(d-k)) and random cores whose vertical flattenings have
    orthonormal columns (cores 1..d-1), last core random.  This is the timed
    'saturated' state: it sits exactly at the rank cap."""
    rng = np.random.default_rng(seed)
    ranks = [1]
    for k in range(1, d):
        ranks.append(int(min(r, n ** min(k, d - k))))
    ranks.append(1)
    cores = []
    for k in range(d):
        a, c = ranks[k], ranks[k + 1]
        g = rng.standard_normal((a * n, c)) + 1j * rng.standard_normal((a * n, c))
        if k < d - 1:
            q, _ = np.linalg.qr(g)
            g = q
        else:
            g = g / np.linalg.norm(g)
        cores.append(np.asfortranarray(g.reshape((a, n, c), order="F")))
    return cores, ranks


def random_probe_indices(d: int, n: int, npts: int, seed: int):
    """Random multi-indices (npts x d) into the n^d grid."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, n, size=(npts, d)).astype(np.int32)


def mc_gaussian_samples(d: int, nsamples: int, seed: int):
    """Standard-normal draws (nsamples x d) for Monte-Carlo initial states;
    the caller colours them with its own covariance factor."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nsamples, d))


def surrogate_member(seed: int) -> Workload:
    """One solve of the surrogate's data set: C4's parameter distribution
    (nu, sigma, ell, 4 Fourier modes of the mean) on the C1 grid, with the
    step 1e-2 (dt |lambda|_max <= 0.2 over the parameter box, far inside
    RK4's stability region)."""
    rng = np.random.default_rng(seed)
    nu = float(rng.uniform(0.01, 0.1))
    sigma = float(rng.uniform(0.1, 0.5))
    ell = float(rng.uniform(0.3, 2.0))
    alpha = tuple(float(x) for x in rng.normal(0.0, 0.5, 4))
    beta = tuple(float(x) for x in rng.normal(0.0, 0.5, 4))
    return Workload(f"S[{seed}]", d=4, n=24, nu=nu, sigma=sigma, ell=ell,
                    alpha=alpha, beta=beta, dt=1e-2, cap=16, tol=1e-10)


def mlp_init(seed: int, dims, members: int):
    """Initial parameters of `members` networks with layer widths `dims`,
    packed per member as W_l (fan_out x fan_in, row-major) then b_l: weights
    ~ N(0, 2 / fan_in) (He et al. 2015), biases 0.  float32 [members][P]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(members):
        parts = []
        for fi, fo in zip(dims[:-1], dims[1:]):
            parts.append(rng.normal(0.0, np.sqrt(2.0 / fi), fi * fo))
            parts.append(np.zeros(fo))
        out.append(np.concatenate(parts))
    return np.asarray(out, dtype=np.float32)


def batch_indices(seed: int, iters: int, members: int, batch: int, nsamples: int):
    """Sample indices [iters][members][batch]: each member walks its own
    random permutations of the data set (epochs), drawn from one seed."""
    rng = np.random.default_rng(seed)
    need = iters * batch
    out = np.empty((members, need), dtype=np.int32)
    for e in range(members):
        reps = -(-need // nsamples)
        out[e] = np.concatenate([rng.permutation(nsamples) for _ in range(reps)])[:need]
    return np.ascontiguousarray(out.reshape(members, iters, batch).transpose(1, 0, 2))
