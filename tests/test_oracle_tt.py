"""Pins of the TT oracle against the plain definition (full contraction of
the iterated matrix product, App. A), the full-grid generator, and the
invariants the paper states for orthogonalisation and truncation
(orthogonality conditions; ||g - f|| <= eps for Alg. 2)."""
import numpy as np
import pytest

from oracle import fullgrid, model, tt
import synthetic


def _rand(d, n, ranks, seed):
    return synthetic.random_tt_cores(d, n, ranks, seed)


def test_flattening_layout_matches_paper_vectorisation():
    """C[i,j,k] = v[i + a j + a b k]; H[i, j + b k]; V[i + a j, k]."""
    a, b, c = 3, 4, 5
    v = np.arange(a * b * c) + 0j
    C = tt.unV(v, a, b, c)
    Hm, Vm = tt.H(C), tt.V(C)
    for i in range(a):
        for j in range(b):
            for k in range(c):
                assert C[i, j, k] == v[i + a * j + a * b * k]
                assert Hm[i, j + b * k] == C[i, j, k]
                assert Vm[i + a * j, k] == C[i, j, k]


def test_full_equals_pointwise_product():
    cores = _rand(4, 5, [1, 2, 3, 2, 1], 0)
    F = tt.full(cores)
    idx = synthetic.random_probe_indices(4, 5, 30, 1)
    np.testing.assert_allclose(F[tuple(idx.T)], tt.evaluate(cores, idx), atol=1e-14)


def test_sum_and_scale():
    x = _rand(4, 3, [1, 2, 3, 2, 1], 2)
    y = _rand(4, 3, [1, 3, 1, 4, 1], 3)
    z = tt.tt_sum([(0.7, x), (-1.3j, y)])
    assert tt.ranks(z) == [1, 5, 4, 6, 1]
    np.testing.assert_allclose(tt.full(z), 0.7 * tt.full(x) - 1.3j * tt.full(y), atol=1e-14)
    np.testing.assert_allclose(tt.full(tt.scale(x, 2 - 1j)), (2 - 1j) * tt.full(x), atol=1e-14)


@pytest.mark.parametrize("d,n,nonlinear", [(3, 8, True), (4, 6, True), (4, 6, False), (5, 4, True)])
def test_apply_matches_fullgrid(d, n, nonlinear):
    """The MPO apply equals the generator applied on the full grid."""
    L, nu = 3.1, 0.04
    ranks = [1] + [3] * (d - 1) + [1]
    x = _rand(d, n, ranks, 4)
    W = model.mpo_blocks(d, n, L, nu, nonlinear)
    y = tt.apply_mpo(x, W, model.mpo_bond_dims(d))
    assert tt.ranks(y) == [1] + [18] * (d - 1) + [1]
    G = fullgrid.apply_G(tt.full(x), d, n, L, nu, nonlinear)
    np.testing.assert_allclose(tt.full(y), G, atol=1e-13 * np.abs(G).max())


def test_right_orthogonality_after_sweep():
    """H(C_c) H(C_c)^H = I for c >= 2 and the tensor is unchanged."""
    x = _rand(5, 4, [1, 3, 5, 6, 2, 1], 5)
    y = tt.orthogonalize_rl(x)
    for C in y[1:]:
        Hm = tt.H(C)
        np.testing.assert_allclose(Hm @ Hm.conj().T, np.eye(Hm.shape[0]), atol=1e-13)
    np.testing.assert_allclose(tt.full(y), tt.full(x), atol=1e-13)
    assert abs(tt.norm(x) - np.linalg.norm(tt.full(x))) < 1e-13


def test_round_error_bound_and_left_orthogonality():
    x = _rand(5, 5, [1, 4, 6, 6, 4, 1], 6)
    y = _rand(5, 5, [1, 3, 3, 3, 3, 1], 7)
    f = tt.tt_sum([(1.0, x), (0.3, y), (0.01, x)])
    F = tt.full(f)
    for tol in (1e-1, 1e-3, 1e-8):
        g, r, disc = tt.round_tt(f, tol, 1000)
        err = np.linalg.norm(tt.full(g) - F)
        assert err <= tol * np.linalg.norm(F) * (1 + 1e-10)
        assert err <= disc * (1 + 1e-8) + 1e-13
        for C in g[:-1]:
            Vm = tt.V(C)
            np.testing.assert_allclose(Vm.conj().T @ Vm, np.eye(Vm.shape[1]), atol=1e-12)


def test_round_recovers_planted_ranks():
    x = _rand(5, 4, [1, 3, 4, 4, 2, 1], 8)
    f = tt.tt_sum([(1.0, x), (0.5, x), (-0.25j, x)])
    g, r, disc = tt.round_tt(f, 1e-12, 1000)
    assert r == [1, 3, 4, 4, 2, 1]
    np.testing.assert_allclose(tt.full(g), (1.5 - 0.25j) * tt.full(x), atol=1e-12)


def test_round_separable_to_rank_one():
    rng = np.random.default_rng(9)
    vecs = [rng.normal(size=6) + 1j * rng.normal(size=6) for _ in range(4)]
    F = np.einsum("a,b,c,d->abcd", *vecs)
    f = tt.tt_sum([(1.0, tt.tt_svd(F, 0.0, 100)), (1.0, tt.tt_svd(F, 0.0, 100))])
    g, r, _ = tt.round_tt(f, 1e-12, 100)
    assert r == [1, 1, 1, 1, 1]
    np.testing.assert_allclose(tt.full(g), 2 * F, atol=1e-12)


def test_round_tol_zero_is_exact_and_cap_binds():
    x = _rand(4, 6, [1, 5, 7, 5, 1], 10)
    g, r, disc = tt.round_tt(x, 0.0, 1000)
    np.testing.assert_allclose(tt.full(g), tt.full(x), atol=1e-13)
    g2, r2, disc2 = tt.round_tt(x, 0.0, 3)
    assert max(r2) == 3 and disc2 > 0
    assert np.linalg.norm(tt.full(g2) - tt.full(x)) <= disc2 * (1 + 1e-10)


def test_forced_ranks_replay():
    x = _rand(4, 5, [1, 4, 6, 4, 1], 11)
    f = tt.tt_sum([(1.0, x), (1e-3, _rand(4, 5, [1, 2, 2, 2, 1], 12))])
    g, r, _ = tt.round_tt(f, 1e-6, 1000)
    g2, r2, _ = tt.round_tt(f, 0.5, 1000, forced_ranks=r)
    assert r2 == r
    np.testing.assert_allclose(tt.full(g2), tt.full(g), atol=1e-13)


def test_tt_svd_accuracy():
    d, n = 4, 10
    m0, C0 = model.cell_moments(d, (0.0,), (1.0,), 0.3, 1.0)
    L = model.default_L(C0)
    F = fullgrid.phi0_grid(m0, C0, n, L)
    for tol in (1e-4, 1e-10):
        cores = tt.tt_svd(F, tol, 1000)
        assert np.linalg.norm(tt.full(cores) - F) <= tol * np.linalg.norm(F) * (1 + 1e-9)


def test_diagonal_covariance_gives_rank_one():
    """ell -> 0: uncorrelated cells, Phi0 is a product, TT rank 1."""
    d, n = 4, 8
    m0 = np.array([0.1, -0.2, 0.3, 0.0])
    C0 = np.diag([0.05, 0.06, 0.07, 0.08])
    F = fullgrid.phi0_grid(m0, C0, n, model.default_L(C0))
    assert tt.ranks(tt.tt_svd(F, 1e-12, 100)) == [1, 1, 1, 1, 1]


def test_tt_rk4_tracks_fullgrid():
    """Step-truncation RK4 stays within the accumulated truncation budget of
    the untruncated full-grid RK4 (d = 4, C1 parameters, n = 12)."""
    w = synthetic.C1
    d, n = 4, 12
    m0, C0 = model.cell_moments(d, w.alpha, w.beta, w.sigma, w.ell)
    L = model.default_L(C0)
    F = fullgrid.phi0_grid(m0, C0, n, L)
    cores = tt.tt_svd(F, 1e-12, 1000)
    W = model.mpo_blocks(d, n, L, w.nu)
    bond = model.mpo_bond_dims(d)
    budget = np.linalg.norm(tt.full(cores) - F)
    for _ in range(5):
        cores, discs = tt.rk4_step(cores, w.dt, W, bond, 1e-12, 1000)
        F = fullgrid.rk4_step(F, w.dt, d, n, L, w.nu)
        budget += sum(discs) * 2.0  # stage errors enter with O(1) weights
    err = np.linalg.norm(tt.full(cores) - F)
    assert err <= budget + 1e-12
    assert err / np.linalg.norm(F) < 1e-10


def test_tt_moments_match_fullgrid():
    d, n = 4, 12
    m0, C0 = model.cell_moments(d, (0.3,), (1.0,), 0.3, 1.0)
    L = model.default_L(C0)
    F = fullgrid.phi0_grid(m0, C0, n, L)
    cores = tt.tt_svd(F, 1e-13, 1000)
    _, da = model.a_grid(n, L)
    mt, ct = tt.moments(cores, n, L, da)
    mf, cf = fullgrid.moments(F, n, L)
    np.testing.assert_allclose(mt, mf, atol=1e-10)
    np.testing.assert_allclose(ct, cf, atol=1e-10)
