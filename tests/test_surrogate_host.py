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
