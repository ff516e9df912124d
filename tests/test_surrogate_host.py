"""Host-side logic of the surrogate (no GPU): feature and target packing,
the seeded batch schedule, and the network-shape validation of the C ABI."""
import ctypes as C

import numpy as np

import synthetic
from oracle import mlp as O


def test_features_and_packing():
    from paper_2403_04946_gb300 import surrogate as S
    w = synthetic.surrogate_member(3)
    x = S.params(w, 0.05)
    assert x.shape == (S.N_PARAMS,)
    np.testing.assert_array_equal(x[:3], [w.nu, w.sigma, w.ell])
    np.testing.assert_array_equal(x[3:7], w.alpha)
    np.testing.assert_array_equal(x[7:11], w.beta)
    assert x[11] == 0.05
    cov = np.arange(16.0).reshape(4, 4)
    cov = cov + cov.T
    y = S.pack_moments(np.arange(4.0), cov)
    assert y.shape == (S.n_out(4),) == (14,)
    np.testing.assert_array_equal(y[4:8], cov[0])  # first row of the upper triangle
    np.testing.assert_array_equal(y[-1], cov[3, 3])


def test_batch_schedule_walks_permutations():
    idx = synthetic.batch_indices(0, iters=10, members=3, batch=7, nsamples=35)
    assert idx.shape == (10, 3, 7)
    for e in range(3):
        seq = idx[:, e, :].reshape(-1)
        for k in range(0, 70, 35):  # every epoch visits each sample once
            assert sorted(seq[k:k + 35]) == list(range(35))
    assert not np.array_equal(idx[:, 0], idx[:, 1])


def test_param_count_matches_layout(lib):
    from paper_2403_04946_gb300 import binding as B
    for shape, M in [((12, 256, 4, 14), 4), ((3, 5, 0, 2), 1), ((7, 9, 2, 4), 2)]:
        p = B.HopfMlpParams(shape[0], shape[1], shape[2], shape[3], M, 16)
        assert B.Mlp.param_count(lib, p) == O.layout(*shape)[1]
    bad = B.HopfMlpParams(0, 8, 1, 2, 1, 16)
    P = C.c_longlong()
    assert lib.hopf_mlp_param_count(C.byref(bad), C.byref(P)) == B.HOPF_EINVAL


def test_dataset_pairs_rates_with_initial_moments(monkeypatch):
    """dataset(): one pair per (solve, snapshot > 0), input [params(T), y0,
    ydot0], target (y(T) - y0 - T ydot0) / T, base y0 + T ydot0; the solver
    is replaced by known tables."""
    from paper_2403_04946_gb300 import surrogate as S
    members = [synthetic.surrogate_member(s) for s in (1, 2)]
    table = np.arange(2 * 3 * 14, dtype=float).reshape(2, 3, 14) ** 1.5
    rates = -np.arange(2 * 14, dtype=float).reshape(2, 14) ** 0.5

    def fake_solve(ms, steps, rate0=False, **kw):
        assert steps == [0, 2, 5] and rate0
        return table[: len(ms)], rates[: len(ms)]

    monkeypatch.setattr(S, "solve", fake_solve)
    X, R, BASE, YT, T = S.dataset(members, [5, 2])
    assert X.shape == (4, S.n_in(4)) == (4, 12 + 28) and R.shape == (4, 14)
    dt = members[0].dt
    np.testing.assert_allclose(T, [2 * dt, 5 * dt, 2 * dt, 5 * dt])
    np.testing.assert_array_equal(X[1, :S.N_PARAMS], S.params(members[0], 5 * dt))
    np.testing.assert_array_equal(X[3, S.N_PARAMS:S.N_PARAMS + 14], table[1, 0])
    np.testing.assert_array_equal(X[3, S.N_PARAMS + 14:], rates[1])
    np.testing.assert_allclose(R[2], (table[1, 1] - table[1, 0] - 2 * dt * rates[1]) / (2 * dt))
    np.testing.assert_array_equal(YT[3], table[1, 2])
    np.testing.assert_allclose(BASE[0], table[0, 0] + 2 * dt * rates[0])


def test_answer_routes_rejected_queries_to_the_solver(monkeypatch):
    """answer(): the network's answer where its bound <= tol, the solver's
    elsewhere, with the solves grouped by step count."""
    from paper_2403_04946_gb300 import surrogate as S
    members = [synthetic.surrogate_member(s) for s in (3, 4, 5, 6)]
    steps = [4, 7, 4, 7]
    calls = []

    def fake_solve(ms, st, rate0=False, **kw):
        calls.append((len(ms), tuple(st)))
        if st == [0]:
            assert rate0
            return np.zeros((len(ms), 1, 14)), np.zeros((len(ms), 14))
        return np.full((len(ms), 1, 14), 100.0 + st[0])

    class FakeNet:
        def predict(self, X, kappa, base=None, scale=None):
            return np.ones((len(X), 14)), np.array([1e-4, 5e-3, 2e-3, 1e-5])

    monkeypatch.setattr(S, "solve", fake_solve)
    sur = S.Surrogate.__new__(S.Surrogate)
    sur.net, sur.kappa, sur.d = FakeNet(), 1.0, 4
    out = sur.answer(members, steps, 1e-3)
    np.testing.assert_array_equal(out["accepted"], [True, False, False, True])
    np.testing.assert_array_equal(out["y"][0], np.ones(14))
    np.testing.assert_array_equal(out["y"][1], np.full(14, 107.0))
    np.testing.assert_array_equal(out["y"][2], np.full(14, 104.0))
    np.testing.assert_array_equal(out["y_net"][1], np.ones(14))
    assert calls == [(4, (0,)), (1, (4,)), (1, (7,))]
