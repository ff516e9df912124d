"""Learned surrogate of the solver: parameters of a Gaussian initial state
-> mean and covariance of the cell averages at time T.

Orchestration only: the solves run through the library's hopf_* calls, the
network's training and inference through its hopf_mlp_* calls (every
arithmetic step a CUDA kernel); this module moves arrays between them.

Inputs (12): nu, sigma, ell, the cos/sin amplitudes of Fourier modes 1..4
of the initial mean, and T.  Outputs (d + d(d+1)/2): the d means and the
upper triangle (row by row, j <= k) of the covariance, as the solver's
hopf_eval_moments returns them after T / dt RK4 steps.

The solver is the fallback and the judge: a query is answered by the
network only when the ensemble's error bound is at most `tol`; every other
query is solved.  The bound's scale kappa is calibrated on held-out solves
so that it covers every calibration error.
"""
from __future__ import annotations

import time

import numpy as np

from . import binding as B

N_IN = 12


def features(w, T):
    """The 12 network inputs of workload `w` at horizon T."""
    a = list(w.alpha) + [0.0] * (4 - len(w.alpha))
    b = list(w.beta) + [0.0] * (4 - len(w.beta))
    return np.array([w.nu, w.sigma, w.ell, *a[:4], *b[:4], T], dtype=np.float64)


def n_out(d):
    return d + d * (d + 1) // 2


def pack_moments(mean, cov):
    d = len(mean)
    iu = np.triu_indices(d)
    return np.concatenate([mean, np.asarray(cov).reshape(d, d)[iu]])


def solve(members, snapshots, concurrency=16):
    """Solves every workload in `members` (same d, n, dt) and returns the
    packed moments at each snapshot step count: array
    [len(members)][len(snapshots)][n_out].  Up to `concurrency` solves run
    at once (hopf_step_ensemble), each on its own stream and on an equal
    share of the SMs."""
    import torch  # device streams

    if not members:
        return np.zeros((0, len(snapshots), 0))
    d, n = members[0].d, members[0].n
    out = np.zeros((len(members), len(snapshots), n_out(d)))
    concurrency = max(1, min(concurrency, len(members)))
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    share = max(1, sms // concurrency)
    streams = [torch.cuda.Stream() for _ in range(concurrency)]
    helper = B.Context(d=d, n=n, nu=0.05, tol=1e-10, rank_cap=4, L=1.0, stream=streams[0].cuda_stream)
    try:
        for w0 in range(0, len(members), concurrency):
            wave = members[w0:w0 + concurrency]
            ctxs, tts = [], []
            try:
                for i, w in enumerate(wave):
                    m0, C0 = helper.hopf_cell_moments(w.alpha, w.beta, w.sigma, w.ell)
                    ctx = B.Context(d=d, n=n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=0.0,
                                    stream=streams[i].cuda_stream)
                    if len(wave) > 1:
                        ctx.hopf_set_max_ctas(share)
                    ctxs.append(ctx)
                    tts.append(ctx.hopf_init_gaussian(m0, C0))
                done = 0
                for j, s in enumerate(snapshots):
                    if s > done:
                        B.hopf_step_ensemble(list(zip(ctxs, tts)), [w.dt for w in wave], s - done)
                        done = s
                    for i, (ctx, t) in enumerate(zip(ctxs, tts)):
                        mean, cov, _ = ctx.hopf_eval_moments(t)
                        out[w0 + i, j] = pack_moments(mean, cov)
            finally:
                for ctx, t in zip(ctxs, tts):
                    ctx.tt_free(t)
                for ctx in ctxs:
                    ctx.close()
    finally:
        helper.close()
    return out


def dataset(members, snapshots, dt, **kw):
    """(X, Y) pairs for every (member, snapshot) of a solve batch."""
    Y = solve(members, snapshots, **kw)
    X = np.array([features(w, s * dt) for w in members for s in snapshots])
    return X, Y.reshape(len(members) * len(snapshots), -1)


def rel_err(pred, ref):
    return np.linalg.norm(pred - ref, axis=-1) / np.linalg.norm(ref, axis=-1)


class Surrogate:
    """An ensemble of `members` networks N_IN -> width x depth -> n_out."""

    def __init__(self, ctx, d, init, width=256, depth=4, members=4, max_batch=4096):
        self.d = d
        self.net = B.Mlp(ctx, N_IN, width, depth, n_out(d), members, max_batch, init)
        self.kappa = None

    def fit(self, X, Y, idx, lr):
        self.net.set_data(X, Y)
        return self.net.train(idx, lr)

    def calibrate(self, X, Y):
        """kappa = the smallest scale for which the bound covers every
        calibration error: max_i err_i / raw_bound_i."""
        y, raw = self.net.predict(X, 1.0)
        err = rel_err(y, Y)
        self.kappa = float(np.max(err / np.maximum(raw, 1e-300)))
        return self.kappa, err, raw

    def predict(self, X):
        return self.net.predict(X, self.kappa)

    def answer(self, members, T_steps, tol, solver_kw=None):
        """Answers the queries (member i at T_steps[i] steps): the network
        where its bound <= tol, the solver elsewhere.  Returns (Y, accepted,
        seconds in the network, seconds in the solver)."""
        dt = members[0].dt
        X = np.array([features(w, s * dt) for w, s in zip(members, T_steps)])
        t0 = time.perf_counter()
        Y, bound = self.predict(X)
        t1 = time.perf_counter()
        acc = bound <= tol
        rej = np.flatnonzero(~acc)
        if rej.size:
            for s in sorted(set(int(T_steps[i]) for i in rej)):
                sel = [i for i in rej if int(T_steps[i]) == s]
                Y[sel] = solve([members[i] for i in sel], [s], **(solver_kw or {}))[:, 0]
        t2 = time.perf_counter()
        return Y, acc, t1 - t0, t2 - t1

    def close(self):
        self.net.close()
