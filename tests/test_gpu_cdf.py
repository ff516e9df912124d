"""The paper's own workload on the GPU: the CDF equation (Sec. 5,
Eq. cdf-burgers, alpha = 0) and the truncated explicit Euler and midpoint
schemes (Eqs. adaptive-euler-method and adaptive-midpoint-method), through
the C ABI, against oracle.cdf and oracle.tt; then the paper's order study
(Sec. 5.1): local truncation errors against a Richardson extrapolation one
order higher, computed on the GPU."""
import numpy as np
import pytest

from oracle import cdf, fullgrid, model, tt
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2403_04946_gb300 import binding, build
    build.build()
    return binding


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def cdf_ctx(B, d, n, gamma, tol, cap, precision=0):
    ctx = B.Context(d=d, n=n, nu=gamma, tol=tol, rank_cap=cap, precision=precision)
    ctx.hopf_set_equation(B.HOPF_EQ_CDF, cdf.BOX)
    return ctx


@pytest.mark.parametrize("d,n,r", [(3, 8, 2), (4, 16, 5), (6, 32, 7)])
def test_cdf_apply_matches_oracle_core_by_core(B, d, n, r):
    gamma = 0.05
    x = synthetic.random_tt_cores(d, n, [1] + [r] * (d - 1) + [1], seed=60 + d)
    ctx = cdf_ctx(B, d, n, gamma, 1e-10, 6 * r)
    tx, ty = ctx.tt_from_host(x), ctx.tt_create(6 * r)
    ctx.hopf_apply_op(tx, ty)
    want = tt.apply_mpo(x, cdf.mpo_blocks(d, n, gamma), model.mpo_bond_dims(d))
    for g, w in zip(ctx.tt_to_host(ty), want):
        assert g.shape == w.shape and rel(g, w) < 1e-13
    ctx.close()


def test_cdf_initial_state(B):
    d, n = 5, 20
    mu = np.array([0.1, -0.2, 0.0, 0.3, 0.05])
    ctx = cdf_ctx(B, d, n, 0.05, 1e-10, 4)
    t = ctx.hopf_init_cdf(0.25, mu)
    assert ctx.tt_get_ranks(t) == [1] * (d + 1)
    want = cdf.initial_tt(d, n, mu=mu)
    idx = synthetic.random_probe_indices(d, n, 100, 7)
    assert rel(ctx.hopf_eval_points(t, idx), tt.evaluate(want, idx)) < 1e-15
    with pytest.raises(B.HopfError):
        ctx.hopf_eval_moments(t)  # moments are defined through Phi, not a CDF
    ctx.close()


def _oracle_steps(scheme, x, dt, nsteps, W, bond, tol, cap):
    step = {"euler": tt.euler_step, "midpoint": tt.midpoint_step}.get(scheme)
    log = []
    for _ in range(nsteps):
        if step is None:
            x, _ = tt.rk4_step(x, dt, W, bond, tol, cap, record=log)
        else:
            x, _ = step(x, dt, lambda y: tt.apply_mpo(y, W, bond), tol, cap, record=log)
    return x, np.array(log)


SCHEMES = pytest.mark.parametrize("scheme", ["euler", "midpoint", "rk4"])


def _code(B, scheme):
    return {"euler": B.HOPF_EULER, "midpoint": B.HOPF_MIDPOINT, "rk4": B.HOPF_RK4}[scheme]


@SCHEMES
def test_cdf_schemes_match_oracle_with_rank_replay(B, scheme):
    """d = 5, n = 24 from a shifted product of Gaussian CDFs, 4 steps,
    tol 1e-9, cap 12, the oracle's ranks replayed: <= 1e-10."""
    d, n, gamma, dt, tol, cap = 5, 24, 0.05, 0.02, 1e-9, 12
    mu = [0.2, -0.1, 0.0, 0.1, -0.2]
    x0 = cdf.initial_tt(d, n, mu=mu)
    W, bond = cdf.mpo_blocks(d, n, gamma), model.mpo_bond_dims(d)
    want, log = _oracle_steps(scheme, x0, dt, 4, W, bond, tol, cap)
    ctx = cdf_ctx(B, d, n, gamma, tol, cap)
    t = ctx.hopf_init_cdf(0.25, mu)
    out = ctx.hopf_step_scheme(t, _code(B, scheme), dt, 4, record=True, replay=log)
    assert np.array_equal(out["ranks"], log)
    got = ctx.tt_to_host(t)
    e = tt.diff_norm(got, want) / tt.norm(want)
    print(f"\nCDF {scheme}: ranks {tt.ranks(want)}, rel err {e:.2e}")
    assert e < 1e-10
    ctx.close()


@pytest.mark.parametrize("scheme", ["euler", "midpoint"])
def test_phi_schemes_match_oracle(B, scheme):
    """The same schemes on the characteristic-function PDE (C1 grid)."""
    w = synthetic.C1
    m0, C0 = model.cell_moments(w.d, w.alpha, w.beta, w.sigma, w.ell)
    L = model.default_L(C0)
    x0 = tt.tt_svd(fullgrid.phi0_grid(m0, C0, w.n, L), w.tol, w.cap)
    W, bond = model.mpo_blocks(w.d, w.n, L, w.nu), model.mpo_bond_dims(w.d)
    want, log = _oracle_steps(scheme, x0, w.dt, 10, W, bond, w.tol, w.cap)
    ctx = B.Context(d=w.d, n=w.n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=L)
    t = ctx.tt_from_host(x0, max_rank=w.cap)
    ctx.hopf_step_scheme(t, _code(B, scheme), w.dt, 10, replay=log)
    e = rel(tt.full(ctx.tt_to_host(t)), tt.full(want))
    print(f"\nPhi {scheme} 10 steps: rel err {e:.2e}")
    assert e < 1e-10
    ctx.close()


@pytest.mark.parametrize("scheme,order", [("euler", 1), ("midpoint", 2), ("rk4", 4)])
def test_richardson_order_study_on_gpu(B, scheme, order):
    """The paper's verification (Sec. 5.1, Fig. err-dim-8) for d = 8, n = 32:
    one step of dt against the order-(p+1) Richardson extrapolation
    (2^p f_{dt/2,dt/2} - f_dt) / (2^p - 1); the local error scales like
    dt^(p+1), so it falls by 2^(p+1) per halving of dt."""
    d, n, gamma, tol, cap = 8, 32, 0.05, 1e-13, 64
    mu = [0.2, -0.1, 0.0, 0.1, -0.2, 0.15, -0.05, 0.1]
    dts = (0.08, 0.04, 0.02) if scheme == "rk4" else (0.04, 0.02, 0.01)
    ctx = cdf_ctx(B, d, n, gamma, tol, cap)
    code = _code(B, scheme)
    errs = []
    for dt in dts:
        f1 = ctx.hopf_init_cdf(0.25, mu)
        ctx.hopf_step_scheme(f1, code, dt, 1)
        f2 = ctx.hopf_init_cdf(0.25, mu)
        ctx.hopf_step_scheme(f2, code, dt / 2, 2)
        dif = ctx.tt_create(2 * cap)
        ctx.tt_sum([f1, f2], [1.0, -1.0], dif)
        errs.append(2 ** order / (2 ** order - 1) * ctx.tt_norm(dif))  # ||f1 - extrapolation||
        for h in (f1, f2, dif):
            ctx.tt_free(h)
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    print(f"\n{scheme}: local errors {['%.2e' % e for e in errs]}, ratios {['%.2f' % r for r in ratios]}")
    want = 2.0 ** (order + 1)
    assert all(abs(r / want - 1) < 0.2 for r in ratios)
    ctx.close()
