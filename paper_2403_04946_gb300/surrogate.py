"""Learned surrogate of the solver: parameters of a Gaussian initial state
-> mean and covariance of the cell averages at time T.

Orchestration only: the solves run through the library's hopf_* calls, the
network's training and inference through its hopf_mlp_* calls (every
arithmetic step a CUDA kernel); this module moves arrays between them.

Parameters (12): nu, sigma, ell, the cos/sin amplitudes of Fourier modes
1..4 of the initial mean, and T.  Moments y (d + d(d+1)/2): the d means and
the upper triangle (row by row, j <= k) of the covariance, as the solver's
hopf_eval_moments returns them after T / dt RK4 steps.

Residual form.  The solver's own moments at T = 0, y0 (hopf_init_gaussian
then hopf_eval_moments, no time step), and their initial rate ydot0 (the
moments of G Phi0: one operator apply, hopf_apply_op, no rounding and no
time step; the moments are linear in Phi) are cheap and exact.  The network
gets the 12 parameters, y0 and ydot0 as inputs and learns the remaining mean
rate (y(T) - y0 - T ydot0) / T, so that y = y0 + T ydot0 + T net(params, y0,
ydot0).  The method without the network is the first-order extrapolation
y0 + T ydot0.

The solver is the fallback and the judge: a query is answered by the
network only when the ensemble's error bound is at most `tol`; every other
query is solved.  The bound's scale kappa is calibrated on held-out solves
so that it covers every calibration error.
"""
from __future__ import annotations

import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import binding as B

N_PARAMS = 12


def params(w, T):
    """The 12 parameters of workload `w` at horizon T."""
    a = list(w.alpha) + [0.0] * (4 - len(w.alpha))
    b = list(w.beta) + [0.0] * (4 - len(w.beta))
    return np.array([w.nu, w.sigma, w.ell, *a[:4], *b[:4], T], dtype=np.float64)


def n_in(d):
    return N_PARAMS + 2 * n_out(d)


def n_out(d):
    return d + d * (d + 1) // 2


def pack_moments(mean, cov):
    d = len(mean)
    iu = np.triu_indices(d)
    return np.concatenate([mean, np.asarray(cov).reshape(d, d)[iu]])


def solve(members, snapshots, concurrency=16, rate0=False):
    """Solves every workload in `members` (same d, n, tol, rank cap) and
    returns the packed moments at each snapshot step count: array
    [len(members)][len(snapshots)][n_out] (with rate0, also the moments of
    G Phi0, the initial rate, [len(members)][n_out]).  Up to `concurrency`
    solves run at once (hopf_step_ensemble), each on its own stream and on
    an equal share of the SMs; one context per slot is reused from solve to
    solve (nu and L are reset per solve, the workspaces stay)."""
    import torch  # device streams

    if not members:
        z = np.zeros((0, len(snapshots), 0))
        return (z, np.zeros((0, 0))) if rate0 else z
    w0_ = members[0]
    d, n = w0_.d, w0_.n
    out = np.zeros((len(members), len(snapshots), n_out(d)))
    rates = np.zeros((len(members), n_out(d)))
    gphi = []
    concurrency = max(1, min(concurrency, len(members)))
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    share = max(1, sms // concurrency)
    streams = [torch.cuda.Stream() for _ in range(concurrency)]
    ctxs = []
    pool = ThreadPoolExecutor(max_workers=concurrency)
    try:
        for st in streams:
            ctxs.append(B.Context(d=d, n=n, nu=w0_.nu, tol=w0_.tol, rank_cap=w0_.cap, L=0.0,
                                  stream=st.cuda_stream))
            if concurrency > 1:
                ctxs[-1].hopf_set_max_ctas(share)
            if rate0:
                gphi.append(ctxs[-1].tt_create(6 * w0_.cap))
        for w0 in range(0, len(members), concurrency):
            wave = members[w0:w0 + concurrency]
            tts = [None] * len(wave)
            try:
                # Initial states of the wave, one host thread per context
                # (the foreign calls release the interpreter lock).
                def init(i):
                    ctx, w = ctxs[i], wave[i]
                    m0, C0 = ctx.hopf_cell_moments(w.alpha, w.beta, w.sigma, w.ell)
                    ctx.hopf_set_L(0.0)
                    ctx.hopf_set_nu(w.nu)
                    tts[i] = ctx.hopf_init_gaussian(m0, C0)
                    if rate0:  # moments of G Phi0 (linear in Phi)
                        ctx.hopf_apply_op(tts[i], gphi[i])
                        mean, cov, _ = ctx.hopf_eval_moments(gphi[i])
                        rates[w0 + i] = pack_moments(mean, cov)

                list(pool.map(init, range(len(wave))))
                live = list(zip(ctxs, tts))
                done = 0
                for j, s in enumerate(snapshots):
                    if s > done:
                        B.hopf_step_ensemble(live, [w.dt for w in wave], s - done)
                        done = s
                    for i, (ctx, t) in enumerate(live):
                        mean, cov, _ = ctx.hopf_eval_moments(t)
                        out[w0 + i, j] = pack_moments(mean, cov)
            finally:
                for ctx, t in zip(ctxs, tts):
                    if t is not None:
                        ctx.tt_free(t)
    finally:
        pool.shutdown()
        for ctx, g in zip(ctxs, gphi):
            ctx.tt_free(g)
        for ctx in ctxs:
            ctx.close()
    return (out, rates) if rate0 else out


def features(w, t, y0, ydot0):
    """Network input of one query: [params(T), y0, ydot0]."""
    return np.concatenate([params(w, t), y0, ydot0])


def dataset(members, snapshots, **kw):
    """Training pairs from one batch of solves: inputs [params(T), y0, ydot0]
    and targets (y(T) - y0 - T ydot0) / T for every member and every snapshot
    > 0, plus the first-order base y0 + T ydot0 per pair and y(T) for
    evaluation."""
    steps = sorted(set([0] + [int(s) for s in snapshots]))
    Y, Yd = solve(members, steps, rate0=True, **kw)
    X, R, BASE, YT, T = [], [], [], [], []
    for i, w in enumerate(members):
        y0, yd = Y[i, 0], Yd[i]
        for j, s in enumerate(steps):
            if s == 0:
                continue
            t = s * w.dt
            base = y0 + t * yd
            X.append(features(w, t, y0, yd))
            R.append((Y[i, j] - base) / t)
            BASE.append(base)
            YT.append(Y[i, j])
            T.append(t)
    return np.array(X), np.array(R), np.array(BASE), np.array(YT), np.array(T)


def rel_err(pred, ref):
    return np.linalg.norm(pred - ref, axis=-1) / np.linalg.norm(ref, axis=-1)


class Surrogate:
    """An ensemble of `members` networks (12 + 2 n_out) -> width x depth ->
    n_out on the remaining rate (y(T) - y0 - T ydot0) / T."""

    def __init__(self, ctx, d, init, width=256, depth=4, members=4, max_batch=4096):
        self.d = d
        self.net = B.Mlp(ctx, n_in(d), width, depth, n_out(d), members, max_batch, init)
        self.kappa = None

    def fit(self, X, R, idx, lr):
        self.net.set_data(X, R)
        return self.net.train(idx, lr)

    def predict(self, X, BASE, T, kappa=None):
        """y = (y0 + T ydot0) + T net(x) and its error bound."""
        k = self.kappa if kappa is None else kappa
        return self.net.predict(X, k, base=BASE, scale=T)

    def calibrate(self, X, BASE, T, YT):
        """kappa = the smallest scale for which the bound covers every
        calibration error: max_i err_i / raw_bound_i."""
        y, raw = self.predict(X, BASE, T, kappa=1.0)
        err = rel_err(y, YT)
        self.kappa = float(np.max(err / np.maximum(raw, 1e-300)))
        return self.kappa, err, raw

    def answer(self, members, steps, tol, concurrency=8):
        """Answers the queries (member i after steps[i] RK4 steps): the
        network where its bound <= tol, the solver elsewhere.  Returns a
        dict: y (the answers), accepted, y_net and bound (the network's own
        answers and bounds), and the seconds spent on y0, in the network and
        in the fallback solves."""
        t0 = time.perf_counter()
        Y0, Yd = solve(members, [0], concurrency=concurrency, rate0=True)
        y0 = Y0[:, 0]
        t1 = time.perf_counter()
        T = np.array([s * w.dt for w, s in zip(members, steps)])
        X = np.array([features(w, t, y, yd) for w, t, y, yd in zip(members, T, y0, Yd)])
        y_net, bound = self.predict(X, y0 + T[:, None] * Yd, T)
        t2 = time.perf_counter()
        y = y_net.copy()
        acc = bound <= tol
        rej = np.flatnonzero(~acc)
        for s in sorted(set(int(steps[i]) for i in rej)):
            sel = [i for i in rej if int(steps[i]) == s]
            y[sel] = solve([members[i] for i in sel], [s], concurrency=concurrency)[:, 0]
        t3 = time.perf_counter()
        return {"y": y, "accepted": acc, "y_net": y_net, "bound": bound,
                "t_y0": t1 - t0, "t_net": t2 - t1, "t_fallback": t3 - t2}

    def close(self):
        self.net.close()
