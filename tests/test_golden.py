"""The oracle still reproduces its stored full-grid values
(tests/golden/c1_fullgrid_20steps.txt, written by tests/golden/make_golden.py
from oracle.fullgrid alone), and the stored values obey what the paper's
model fixes: |Phi| <= 1, a symmetric positive covariance, and the
reflection symmetry of the sin x initial state."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden  # noqa: E402


def test_oracle_reproduces_stored_values():
    L, idx, vals, mean, cov, ranks, tvals = make_golden.read_c1()
    L2, idx2, vals2, mean2, cov2 = make_golden.c1_fullgrid()
    assert abs(L2 - L) <= 1e-13 * L  # quadrature rounding differs across hosts
    np.testing.assert_array_equal(idx2, idx)
    np.testing.assert_allclose(vals2, vals, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(mean2, mean, rtol=1e-12)
    np.testing.assert_allclose(cov2, cov, rtol=1e-10, atol=1e-14)
    ranks2, tvals2 = make_golden.c1_tt(L, idx)
    np.testing.assert_array_equal(ranks2, ranks)
    np.testing.assert_allclose(tvals2, tvals, rtol=0, atol=1e-12)


def test_stored_values_obey_model_invariants():
    _, _, vals, mean, cov, ranks, _ = make_golden.read_c1()
    assert ranks.shape == (8 * make_golden.NSTEPS, 5) and np.all(ranks[:, [0, -1]] == 1)
    assert np.all(np.abs(vals) <= 1.0)
    # Burgers keeps u(x) -> -u(-x); sin x and the stationary covariance are
    # invariant under it, and x -> -x maps cell k to cell 3 - k (d = 4), so
    # m_k = -m_{3-k} and C_jk = C_{3-j,3-k} for all time
    np.testing.assert_allclose(mean, -mean[::-1], rtol=1e-12)
    np.testing.assert_allclose(cov, cov[::-1, ::-1], rtol=1e-10)
    np.testing.assert_allclose(cov, cov.T, atol=1e-15)
    assert np.all(np.linalg.eigvalsh(cov) > 0)
