"""Parity of the CUDA path (called through the C ABI) with the CPU oracle.

Gauge: TT cores are unique only up to invertible factors on the bonds, so
results of roundings are compared as tensors (full contraction for small d,
or sampled entries), while the operator apply and sums, which are gauge-free,
are compared core by core.  Rank decisions are replayed from the oracle
("forced ranks") where element-wise parity is asserted.

Tolerances (relative L2 unless stated): 1e-13 for gauge-free kernels
(a few roundings of 16-byte complex products); 1e-12 for one rounding;
1e-10 for time stepping (the acceptance bound for the FP64 path)."""
import os
import sys

import numpy as np
import pytest

from oracle import fullgrid, model, tt
import synthetic

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.fixture(scope="module")
def B():
    from paper_2403_04946_gb300 import binding, build
    build.build()
    return binding


def ctx_for(B, d, n, nu=0.05, L=3.0, tol=1e-10, cap=16, nonlinear=True, svd=0):
    ctx = B.Context(d=d, n=n, nu=nu, tol=tol, rank_cap=cap, L=L, nonlinear=nonlinear)
    ctx.hopf_set_svd_method(svd)
    return ctx


SVD_METHODS = pytest.mark.parametrize("svd", [0, 1], ids=["bidiag", "jacobi"])


@pytest.mark.parametrize("d,n,r", [(3, 8, 2), (4, 12, 5), (6, 20, 11), (5, 33 - 1, 7)])
def test_apply_matches_oracle_core_by_core(B, d, n, r):
    L, nu = 2.7, 0.03
    ranks = [1] + [r] * (d - 1) + [1]
    x = synthetic.random_tt_cores(d, n, ranks, seed=d * 100 + n)
    ctx = ctx_for(B, d, n, nu=nu, L=L)
    tx = ctx.tt_from_host(x)
    ty = ctx.tt_create(6 * r)
    ctx.hopf_apply_op(tx, ty)
    got = ctx.tt_to_host(ty)
    want = tt.apply_mpo(x, model.mpo_blocks(d, n, L, nu), model.mpo_bond_dims(d))
    assert ctx.tt_get_ranks(ty) == tt.ranks(want)
    for g, w in zip(got, want):
        assert g.shape == w.shape
        assert rel(g, w) < 1e-13


def test_apply_linear_flag(B):
    d, n, L, nu = 4, 10, 2.0, 0.2
    x = synthetic.random_tt_cores(d, n, [1, 3, 3, 3, 1], seed=5)
    ctx = ctx_for(B, d, n, nu=nu, L=L, nonlinear=False)
    tx, ty = ctx.tt_from_host(x), ctx.tt_create(18)
    ctx.hopf_apply_op(tx, ty)
    want = tt.apply_mpo(x, model.mpo_blocks(d, n, L, nu, nonlinear=False), model.mpo_bond_dims(d))
    for g, w in zip(ctx.tt_to_host(ty), want):
        assert rel(g, w) < 1e-13


def test_sum_matches_oracle(B):
    d, n = 5, 10
    x = synthetic.random_tt_cores(d, n, [1, 2, 4, 3, 2, 1], 1)
    y = synthetic.random_tt_cores(d, n, [1, 3, 2, 2, 5, 1], 2)
    ctx = ctx_for(B, d, n)
    tx, ty, tz = ctx.tt_from_host(x), ctx.tt_from_host(y), ctx.tt_create(8)
    ctx.tt_sum([tx, ty], [0.3 - 0.2j, 1.5j], tz)
    want = tt.tt_sum([(0.3 - 0.2j, x), (1.5j, y)])
    for g, w in zip(ctx.tt_to_host(tz), want):
        assert np.array_equal(g.shape, w.shape) and rel(g, w) < 1e-15


@pytest.mark.parametrize("d,n,ranks,tol,cap", [
    (4, 12, [1, 6, 20, 6, 1], 1e-8, 100),      # tolerance-bound, wide first/last cores
    (6, 20, [1, 20, 45, 70, 45, 20, 1], 1e-6, 33),  # several QR panels, ragged tail, cap
    (5, 40, [1, 17, 33, 33, 17, 1], 0.0, 100),  # tol = 0: exact
])
@SVD_METHODS
def test_round_matches_oracle_with_rank_replay(B, d, n, ranks, tol, cap, svd):
    base = synthetic.random_tt_cores(d, n, [1] + [min(4, r) for r in ranks[1:-1]] + [1], seed=7)
    noise = synthetic.random_tt_cores(d, n, ranks, seed=8, scale=1e-3)
    x = tt.tt_sum([(1.0, base), (1.0, noise)])
    want, wranks, wdisc = tt.round_tt(x, tol, cap)
    ctx = ctx_for(B, d, n, tol=tol, cap=cap, svd=svd)
    tx = ctx.tt_from_host(x, max_rank=max(tt.ranks(x)))
    disc, st = ctx.tt_round(tx, tol, cap, forced_ranks=wranks)
    assert ctx.tt_get_ranks(tx) == wranks
    got = ctx.tt_to_host(tx)
    F = tt.full(x)
    assert rel(tt.full(got), tt.full(want)) < 1e-12 * max(1.0, np.linalg.norm(F) / max(np.linalg.norm(tt.full(want)), 1e-300))
    # tails far below the cut are resolved to 1e-3 of the per-SVD tolerance
    eps_hat = tol * np.linalg.norm(F) / np.sqrt(d - 1)
    assert abs(disc - wdisc) <= 1e-8 * wdisc + 1e-3 * eps_hat * np.sqrt(d) + 1e-13 * np.linalg.norm(F)
    # left-orthonormal cores (the result of the left-to-right truncation)
    for C in got[:-1]:
        V = tt.V(C)
        assert np.abs(V.conj().T @ V - np.eye(V.shape[1])).max() < 1e-12
    # free-running rank choice agrees with the oracle's
    tx2 = ctx.tt_from_host(x, max_rank=max(tt.ranks(x)))
    ctx.tt_round(tx2, tol, cap)
    assert ctx.tt_get_ranks(tx2) == wranks


@SVD_METHODS
def test_round_rank_deficient_keeps_noise_level_values(B, svd):
    """x + x/2 has numerically the ranks of x; with tol = 0 every singular
    value is kept, the ones at the rounding level included.  Their vectors
    are not determined by the data, but the rounded tensor and the
    orthonormality of the cores are."""
    d, n = 5, 12
    base = synthetic.random_tt_cores(d, n, [1, 5, 9, 9, 5, 1], seed=17)
    x = tt.tt_sum([(1.0, base), (0.5, base)])
    want, wranks, _ = tt.round_tt(x, 0.0, 100)
    assert max(wranks) > 9  # noise-level values are kept
    ctx = ctx_for(B, d, n, tol=0.0, cap=100, svd=svd)
    tx = ctx.tt_from_host(x, max_rank=max(tt.ranks(x)))
    ctx.tt_round(tx, 0.0, 100, forced_ranks=wranks)
    got = ctx.tt_to_host(tx)
    assert rel(tt.full(got), tt.full(x)) < 1e-13
    for C in got[:-1]:
        V = tt.V(C)
        assert np.abs(V.conj().T @ V - np.eye(V.shape[1])).max() < 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 33, 97, 160])
def test_square_svd_paths_agree(B, n):
    """Bidiagonal and Jacobi SVD give the oracle's rounding of a three-core
    tensor whose bond factors are n x n triangles with a graded spectrum
    (from a single element to many CTAs of the bidiagonalisation)."""
    rng = np.random.default_rng(n)
    d, m = 3, n + 2 + n % 2
    Ul = np.linalg.qr(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n)))[0]
    s = np.logspace(0, -12, n)
    Vr = np.linalg.qr(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n)))[0]
    Mid = (rng.standard_normal((n, m, n)) + 1j * rng.standard_normal((n, m, n))) / np.sqrt(m)
    cores = [np.asfortranarray((Ul * s).reshape(1, m, n)), np.asfortranarray(Mid),
             np.asfortranarray(Vr.conj().T.reshape(n, m, 1))]
    want, wranks, wdisc = tt.round_tt(cores, 1e-9, n)
    Fw = tt.full(want)
    for svd in (0, 1):
        ctx = ctx_for(B, d, m, tol=1e-9, cap=n, svd=svd)
        tx = ctx.tt_from_host(cores, max_rank=n)
        disc, _ = ctx.tt_round(tx, 1e-9, n)
        assert ctx.tt_get_ranks(tx) == wranks
        assert rel(tt.full(ctx.tt_to_host(tx)), Fw) < 1e-11
        assert abs(disc - wdisc) <= 1e-6 * wdisc + 1e-14 * np.linalg.norm(Fw)


def test_max_ctas_and_ensemble_match_solo_runs(B):
    """Three independent states advanced together by hopf_step_ensemble,
    each context limited to 40 CTAs, give the same tensors as each state
    advanced alone on the whole GPU (different CTA counts change only the
    order of floating-point sums)."""
    specs = [(5, 12, 10, 31), (6, 10, 8, 32), (4, 16, 12, 33)]
    solo, members, ctxs = [], [], []
    for d, n, r, seed in specs:
        cores, _ = synthetic.saturated_tt_cores(d, n, r, seed=seed)
        cores = [0.3 * c for c in cores]
        ctx = ctx_for(B, d, n, tol=1e-9, cap=3 * r, L=2.5)
        t = ctx.tt_from_host(cores, max_rank=3 * r)
        ctx.hopf_step(t, 1e-4, 2)
        solo.append(tt.full(ctx.tt_to_host(t)))
        ctx.close()
        ectx = ctx_for(B, d, n, tol=1e-9, cap=3 * r, L=2.5)
        ectx.hopf_set_max_ctas(40)
        members.append((ectx, ectx.tt_from_host(cores, max_rank=3 * r)))
        ctxs.append(ectx)
    st = B.hopf_step_ensemble(members, 1e-4, 2)
    assert all(x in (B.HOPF_OK, B.HOPF_ERANKCAP) for x in st)
    for (ectx, t), want in zip(members, solo):
        assert rel(tt.full(ectx.tt_to_host(t)), want) < 1e-11
    with pytest.raises(B.HopfError):
        B.hopf_step_ensemble([members[0], members[0]], 1e-4, 1)  # a context twice
    for c in ctxs:
        c.close()


def test_round_error_bound_and_cap_status(B):
    d, n = 5, 16
    x = synthetic.random_tt_cores(d, n, [1, 10, 20, 20, 10, 1], 9)
    ctx = ctx_for(B, d, n)
    tx = ctx.tt_from_host(x)
    disc, st = ctx.tt_round(tx, 1e-12, 4)
    assert st == B.HOPF_ERANKCAP and max(ctx.tt_get_ranks(tx)) == 4
    err = np.linalg.norm(tt.full(ctx.tt_to_host(tx)) - tt.full(x))
    assert err <= disc * (1 + 1e-9)


def test_norm_eval_points(B):
    d, n = 6, 12
    x = synthetic.random_tt_cores(d, n, [1, 4, 7, 9, 7, 4, 1], 10)
    ctx = ctx_for(B, d, n)
    tx = ctx.tt_from_host(x)
    assert abs(ctx.tt_norm(tx) - tt.norm(x)) < 1e-13 * tt.norm(x)
    idx = synthetic.random_probe_indices(d, n, 200, 3)
    assert rel(ctx.hopf_eval_points(tx, idx), tt.evaluate(x, idx)) < 1e-14


def test_cell_moments_match_oracle(B):
    w = synthetic.C2
    ctx = ctx_for(B, w.d, w.n)
    m0, C0 = ctx.hopf_cell_moments(w.alpha, w.beta, w.sigma, w.ell)
    om0, oC0 = model.cell_moments(w.d, w.alpha, w.beta, w.sigma, w.ell)
    assert np.abs(m0 - om0).max() < 1e-13 and np.abs(C0 - oC0).max() < 1e-13


def _c1_state(n=None):
    w = synthetic.C1
    n = n or w.n
    m0, C0 = model.cell_moments(w.d, w.alpha, w.beta, w.sigma, w.ell)
    L = model.default_L(C0)
    return w, n, m0, C0, L


def test_init_gaussian_matches_full_grid(B):
    w, n, m0, C0, L = _c1_state()
    ctx = B.Context(d=w.d, n=n, nu=w.nu, tol=1e-10, rank_cap=200)
    t = ctx.hopf_init_gaussian(m0, C0)
    assert abs(ctx.hopf_get_L() - L) < 1e-12
    F = fullgrid.phi0_grid(m0, C0, n, L)
    G = tt.full(ctx.tt_to_host(t))
    assert np.linalg.norm(G - F) <= 1e-10 * np.linalg.norm(F) * (1 + 1e-6)
    assert ctx.tt_get_ranks(t) == tt.ranks(tt.tt_svd(F, 1e-10, 200))


def test_init_gaussian_cross_matches_full_grid(B):
    """d = 5, n = 24 (24^5 > 2^20 grid points): the TT-cross construction
    against the full-grid Gaussian (C2's correlated covariance)."""
    w = synthetic.C2
    d, n = 5, 24
    m0, C0 = model.cell_moments(d, w.alpha, w.beta, w.sigma, w.ell)
    L = model.default_L(C0)
    ctx = B.Context(d=d, n=n, nu=w.nu, tol=1e-10, rank_cap=200, L=L)
    t = ctx.hopf_init_gaussian(m0, C0)
    F = fullgrid.phi0_grid(m0, C0, n, L)
    err = rel(tt.full(ctx.tt_to_host(t)), F)
    print(f"cross d=5: ranks {ctx.tt_get_ranks(t)}, rel err {err:.2e}")
    assert err < 1e-9


def test_init_gaussian_cross_pointwise_d10(B):
    """d = 10, n = 16 (10^12 grid points, no full grid): the cross TT at
    tol = 0 reproduces exp(i a.m0 - a^T C0 a / 2) pointwise, and its error
    falls as the rank cap grows."""
    d, n = 10, 16
    m0, C0 = model.cell_moments(d, (0.0, 0.5), (1.0, 0.0), 0.4, 0.3)
    L = model.default_L(C0)
    a, _ = model.a_grid(n, L)
    rng = np.random.default_rng(2)
    idx = (n // 2 + rng.integers(-3, 4, size=(500, d))).astype(np.int32)
    pts = a[idx]
    want = np.exp(1j * pts @ m0 - 0.5 * np.einsum("pj,jk,pk->p", pts, C0, pts))
    errs = []
    for cap in (64, 128):
        ctx = B.Context(d=d, n=n, nu=0.02, tol=0.0, rank_cap=cap, L=L)
        t = ctx.hopf_init_gaussian(m0, C0)
        errs.append(np.abs(ctx.hopf_eval_points(t, idx) - want).max())
        ctx.close()
    print(f"cross d=10 max abs err: cap 64 {errs[0]:.2e}, cap 128 {errs[1]:.2e}")
    assert errs[1] < 1e-7 and errs[1] < errs[0]


def test_init_gaussian_diagonal_is_rank_one(B):
    d, n = 8, 16
    m0 = np.linspace(-0.3, 0.4, d)
    C0 = np.diag(np.linspace(0.05, 0.1, d))
    ctx = B.Context(d=d, n=n, nu=0.01, tol=1e-10, rank_cap=8)
    t = ctx.hopf_init_gaussian(m0, C0)
    assert ctx.tt_get_ranks(t) == [1] * (d + 1)
    L = model.default_L(C0)
    a, _ = model.a_grid(n, L)
    idx = synthetic.random_probe_indices(d, n, 50, 4)
    pts = a[idx]
    want = np.exp(1j * pts @ m0 - 0.5 * np.einsum("pj,jk,pk->p", pts, C0, pts)) * np.all(idx > 0, axis=1)
    assert rel(ctx.hopf_eval_points(t, idx), want) < 1e-14


def test_moments_match_oracle(B):
    w, n, m0, C0, L = _c1_state()
    F = fullgrid.phi0_grid(m0, C0, n, L)
    cores = tt.tt_svd(F, 1e-12, 200)
    ctx = B.Context(d=w.d, n=n, nu=w.nu, tol=1e-10, rank_cap=200, L=L)
    t = ctx.tt_from_host(cores)
    mean, cov, ir = ctx.hopf_eval_moments(t)
    _, da = model.a_grid(n, L)
    om, oc = tt.moments(cores, n, L, da)
    assert np.abs(mean - om).max() < 1e-11 and np.abs(cov - oc).max() < 1e-11
    assert ir < 1e-10


def _step_parity(B, w, n, nsteps, cores, L, svd=0):
    W = model.mpo_blocks(w.d, n, L, w.nu, w.nonlinear)
    bond = model.mpo_bond_dims(w.d)
    log = []
    ocores = cores
    for _ in range(nsteps):
        ocores, _ = tt.rk4_step(ocores, w.dt, W, bond, w.tol, w.cap, record=log)
    ctx = B.Context(d=w.d, n=n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=L, nonlinear=w.nonlinear)
    ctx.hopf_set_svd_method(svd)
    t = ctx.tt_from_host(cores, max_rank=w.cap)
    out = ctx.hopf_step(t, w.dt, nsteps, record=True, replay=np.array(log))
    assert np.array_equal(out["ranks"], np.array(log))
    return ctx, t, ocores


@SVD_METHODS
def test_step_parity_c1_short(B, svd):
    """C1 parameters, 20 RK4 steps with ranks replayed: <= 1e-10 rel L2."""
    w, n, m0, C0, L = _c1_state()
    cores = tt.tt_svd(fullgrid.phi0_grid(m0, C0, n, L), w.tol, w.cap)
    ctx, t, ocores = _step_parity(B, w, n, 20, cores, L, svd=svd)
    err = rel(tt.full(ctx.tt_to_host(t)), tt.full(ocores))
    print(f"C1 20 steps: rel L2 err {err:.3e}")
    assert err < 1e-10


def test_step_parity_c1_full_horizon(B):
    """The FP64 acceptance run: C1 to T = 0.5 (500 steps), ranks replayed."""
    w, n, m0, C0, L = _c1_state()
    cores = tt.tt_svd(fullgrid.phi0_grid(m0, C0, n, L), w.tol, w.cap)
    ctx, t, ocores = _step_parity(B, w, n, w.steps, cores, L)
    err = rel(tt.full(ctx.tt_to_host(t)), tt.full(ocores))
    print(f"C1 {w.steps} steps: rel L2 err {err:.3e}")
    assert err < 1e-10


def test_step_matches_stored_oracle_values(B):
    """C1, 20 RK4 steps on the GPU with the TT oracle's stored rank log
    replayed (tests/golden, written from the oracle alone): Phi at the stored
    points within 1e-10 of the oracle's, relative to the largest value."""
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import make_golden
    Ls, idx, _, _, _, ranks, tvals = make_golden.read_c1()
    w, n, m0, C0, L = _c1_state()
    assert abs(L - Ls) <= 1e-13 * Ls  # quadrature rounding differs across hosts
    cores = tt.tt_svd(fullgrid.phi0_grid(m0, C0, n, Ls), w.tol, w.cap)
    ctx = B.Context(d=w.d, n=n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=Ls)
    t = ctx.tt_from_host(cores, max_rank=w.cap)
    out = ctx.hopf_step(t, w.dt, make_golden.NSTEPS, record=True, replay=ranks)
    assert np.array_equal(out["ranks"], ranks)
    got = ctx.hopf_eval_points(t, idx)
    err = np.abs(got - tvals).max() / np.abs(tvals).max()
    print(f"stored oracle values: max err {err:.2e}")
    assert err < 1e-10


def test_step_free_running_close_to_oracle_and_invariants(B):
    """Free-running ranks (no replay) on a linear-off C1 variant; invariants
    Phi(0) = 1 and mass hold on the GPU result."""
    w, n, m0, C0, L = _c1_state(n=12)
    w = w.with_(cap=144)  # no cap binds: n^2 = 144 bounds the middle rank
    F0 = fullgrid.phi0_grid(m0, C0, n, L)
    cores = tt.tt_svd(F0, w.tol, w.cap)
    ctx = B.Context(d=w.d, n=n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=L)
    t = ctx.tt_from_host(cores, max_rank=w.cap)
    ctx.hopf_step(t, w.dt, 10)
    G = tt.full(ctx.tt_to_host(t))
    F = fullgrid.solve(F0, w.dt, 10, w.d, n, L, w.nu)
    assert rel(G, F) < 1e-8
    c = n // 2
    assert abs(G[(c,) * w.d] - 1.0) < 1e-9
    for i in range(1, n):
        assert abs(G[(i,) * w.d] - F0[(i,) * w.d]) < 1e-9


def test_step_parity_mid_size(B):
    """d = 8, n = 24, cap 12: several panels and bonds, ranks replayed."""
    w = synthetic.C1.with_(d=8, n=24, cap=12, tol=1e-8, dt=5e-4, nu=0.05)
    m0, C0 = model.cell_moments(8, w.alpha, w.beta, w.sigma, 0.05)  # short correlation
    C0 = np.diag(np.diag(C0))  # rank-1 start, ranks grow through the dynamics
    L = model.default_L(C0)
    a, _ = model.a_grid(w.n, L)
    cores = [np.asfortranarray((np.exp(1j * a * m0[k] - 0.5 * C0[k, k] * a * a) * (np.arange(w.n) > 0)).reshape(1, w.n, 1))
             for k in range(8)]
    ctx, t, ocores = _step_parity(B, w, w.n, 3, cores, L)
    idx = synthetic.random_probe_indices(8, w.n, 300, 5)
    got = ctx.hopf_eval_points(t, idx)
    want = tt.evaluate(ocores, idx)
    assert rel(got, want) < 1e-10
    assert abs(ctx.tt_norm(t) - tt.norm(ocores)) < 1e-10 * tt.norm(ocores)


# ---- mixed precision (FP32 trailing updates, FP64 panels and SVD) ----------

def test_mixed_round_close_to_fp64(B):
    """One rounding in mixed precision stays within FP32 rounding of the
    FP64 result (ranks replayed)."""
    d, n, ranks, tol, cap = 6, 20, [1, 20, 45, 70, 45, 20, 1], 1e-6, 33
    base = synthetic.random_tt_cores(d, n, [1, 4, 4, 4, 4, 4, 1], seed=7)
    noise = synthetic.random_tt_cores(d, n, ranks, seed=8, scale=1e-3)
    x = tt.tt_sum([(1.0, base), (1.0, noise)])
    want, wranks, _ = tt.round_tt(x, tol, cap)
    ctx = B.Context(d=d, n=n, nu=0.05, tol=tol, rank_cap=cap, L=3.0, precision=B.HOPF_MIXED)
    tx = ctx.tt_from_host(x, max_rank=max(tt.ranks(x)))
    ctx.tt_round(tx, tol, cap, forced_ranks=wranks)
    err = rel(tt.full(ctx.tt_to_host(tx)), tt.full(want))
    print(f"mixed rounding rel err {err:.2e}")
    assert err < 1e-5


@pytest.mark.parametrize("qr_method", [0, 1])
def test_mixed_round_with_tiny_columns(B, qr_method):
    """Columns far below the matrix's largest entry (1e-22 of it: their
    squares leave the FP32 range) next to O(1) ones, in a lossless mixed
    rounding: every reflector must stay unitary, so the result reproduces
    the input at the mixed path's precision."""
    d, n = 5, 16
    base = synthetic.random_tt_cores(d, n, [1, 4, 4, 4, 4, 1], seed=81)
    tiny = synthetic.random_tt_cores(d, n, [1, 6, 6, 6, 6, 1], seed=82)
    tiny[0] = tiny[0] * 1e-22
    x = tt.tt_sum([(1.0, base), (1.0, tiny)])
    ctx = B.Context(d=d, n=n, nu=0.05, tol=1e-10, rank_cap=64, L=3.0, precision=B.HOPF_MIXED)
    ctx.hopf_set_qr_method(qr_method)
    tx = ctx.tt_from_host(x, max_rank=max(tt.ranks(x)))
    ctx.tt_round(tx, 0.0, 10 ** 6)
    err = rel(tt.full(ctx.tt_to_host(tx)), tt.full(x))
    assert err < 1e-10
    ctx.close()


def test_mixed_step_c1_within_1e6(B):
    """C1, 20 RK4 steps in mixed precision with the oracle's ranks: relative
    L2 error to the FP64 oracle <= 1e-6 (the mixed-precision target)."""
    w, n, m0, C0, L = _c1_state()
    cores = tt.tt_svd(fullgrid.phi0_grid(m0, C0, n, L), w.tol, w.cap)
    W = model.mpo_blocks(w.d, n, L, w.nu)
    bond = model.mpo_bond_dims(w.d)
    log, oc = [], cores
    for _ in range(20):
        oc, _ = tt.rk4_step(oc, w.dt, W, bond, w.tol, w.cap, record=log)
    ctx = B.Context(d=w.d, n=n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=L, precision=B.HOPF_MIXED)
    t = ctx.tt_from_host(cores, max_rank=w.cap)
    ctx.hopf_step(t, w.dt, 20, replay=np.array(log))
    err = rel(tt.full(ctx.tt_to_host(t)), tt.full(oc))
    print(f"mixed C1 20 steps rel err {err:.2e}")
    assert err < 1e-6
