"""Failure handling, memory ownership and checkpointing through the C ABI.

Every failure here is made without faulting the GPU: a NaN in the data, a
bounded wait that expires (a barrier one CTA never reaches, or a wait limit
shorter than a barrier takes), an allocator that refuses.  After each, the
same context must keep working and match the oracle.  The allocator tests
run in fresh processes: the allocator may only change while no context or
tensor exists."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import fullgrid, model, tt
import synthetic

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2403_04946_gb300 import binding, build
    build.build()
    return binding


def _c1():
    w = synthetic.C1
    m0, C0 = model.cell_moments(w.d, w.alpha, w.beta, w.sigma, w.ell)
    L = model.default_L(C0)
    return w, L, tt.tt_svd(fullgrid.phi0_grid(m0, C0, w.n, L), w.tol, w.cap)


def _round_matches_oracle(B, ctx, x, tol=1e-8, cap=100):
    want, wranks, _ = tt.round_tt(x, tol, cap)
    t = ctx.tt_from_host(x, max_rank=max(tt.ranks(x)))
    ctx.tt_round(t, tol, cap, forced_ranks=wranks)
    got = ctx.tt_to_host(t)
    ctx.tt_free(t)
    return np.linalg.norm(tt.full(got) - tt.full(want)) / np.linalg.norm(tt.full(want))


def test_nan_in_a_core_gives_enumeric_and_the_context_recovers(B):
    d, n = 4, 12
    x = synthetic.random_tt_cores(d, n, [1, 6, 20, 6, 1], seed=71)
    bad = [c.copy() for c in x]
    bad[2][3, 5, 4] = np.nan
    ctx = B.Context(d=d, n=n, nu=0.05, tol=1e-8, rank_cap=16, L=3.0)
    t = ctx.tt_from_host(bad)
    with pytest.raises(B.HopfError) as err:
        ctx.tt_round(t, 1e-8, 100)
    assert err.value.status == B.HOPF_ENUMERIC
    clean = synthetic.saturated_tt_cores(d, n, 4, seed=72)[0]
    s = ctx.tt_from_host(clean, max_rank=16)
    nan_state = [c.copy() for c in clean]
    nan_state[1][0, 3, 1] = np.nan
    tb = ctx.tt_from_host(nan_state, max_rank=16)
    with pytest.raises(B.HopfError) as err:
        ctx.hopf_step(tb, 1e-3, 1)  # the step's first rounding meets the NaN
    assert err.value.status == B.HOPF_ENUMERIC
    assert _round_matches_oracle(B, ctx, x) < 1e-12
    ctx.hopf_step(s, 1e-3, 1)
    for h in (t, s, tb):
        ctx.tt_free(h)
    ctx.close()


def test_expired_wait_gives_etimeout_and_the_context_recovers(B):
    """A barrier one CTA never reaches: the other CTA's wait runs out after
    the context's limit (0.2 s here), the call returns HOPF_ETIMEOUT, and the
    next rounding on the same context is exact again."""
    import time
    d, n = 5, 40
    x = tt.tt_sum([(1.0, synthetic.random_tt_cores(d, n, [1, 4, 4, 4, 4, 1], seed=73)),
                   (1.0, synthetic.random_tt_cores(d, n, [1, 17, 33, 33, 17, 1], seed=74, scale=1e-3))])
    ctx = B.Context(d=d, n=n, nu=0.05, tol=1e-8, rank_cap=40, L=3.0)
    ctx.hopf_set_wait_limit(0.2)
    t0 = time.perf_counter()
    st = ctx.hopf_check_watchdog()
    waited = time.perf_counter() - t0
    assert st == B.HOPF_ETIMEOUT
    assert 0.15 < waited < 3.0
    assert "expired" in ctx.lib.hopf_last_error(ctx.h).decode()
    assert _round_matches_oracle(B, ctx, x) < 1e-12
    # the default limit comes back, and the watchdog fires again after it
    ctx.hopf_set_wait_limit(0.0)
    assert _round_matches_oracle(B, ctx, x) < 1e-12
    with pytest.raises(B.HopfError):
        ctx.hopf_set_wait_limit(-1.0)
    ctx.close()


def test_checkpoint_resume_is_bitwise(B, tmp_path):
    """Step 4, save, step 3 more (A); load, step 3 (B): A == B bit for bit,
    the time stamp round-trips, and a file of another shape is refused."""
    w, L, x = _c1()
    ctx = B.Context(d=w.d, n=w.n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=L)
    t = ctx.tt_from_host(x, max_rank=w.cap)
    ctx.hopf_step(t, w.dt, 4)
    path = tmp_path / "state.hopftt"
    ctx.tt_save(t, path, time=4 * w.dt)
    ctx.hopf_step(t, w.dt, 3)
    a = ctx.tt_to_host(t)
    u, tm = ctx.tt_load(path, max_rank=w.cap)
    assert tm == 4 * w.dt
    ctx.hopf_step(u, w.dt, 3)
    b = ctx.tt_to_host(u)
    assert all(np.array_equal(p, q) for p, q in zip(a, b))
    other = B.Context(d=w.d + 1, n=w.n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=L)
    with pytest.raises(B.HopfError) as err:
        other.tt_load(path)
    assert err.value.status == B.HOPF_EINVAL
    cut = tmp_path / "cut.hopftt"
    cut.write_bytes(path.read_bytes()[:-8])
    with pytest.raises(B.HopfError):
        ctx.tt_load(cut)
    for h in (t, u):
        ctx.tt_free(h)
    other.close()
    ctx.close()


def _run(script):
    r = subprocess.run([sys.executable, "-c", textwrap.dedent(script)], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


def test_caching_allocator_backs_a_solve():
    """With PyTorch's caching allocator behind the library, a C1 step matches
    the oracle and the library's memory shows up in PyTorch's account."""
    out = _run("""
        import numpy as np, torch
        from paper_2403_04946_gb300 import binding as B
        from oracle import fullgrid, model, tt
        import synthetic
        dev = torch.cuda.current_device()
        B.hopf_set_allocator(lambda nb: torch.cuda.caching_allocator_alloc(nb, dev),
                             lambda p: torch.cuda.caching_allocator_delete(p))
        w = synthetic.C1
        m0, C0 = model.cell_moments(w.d, w.alpha, w.beta, w.sigma, w.ell)
        L = model.default_L(C0)
        x = tt.tt_svd(fullgrid.phi0_grid(m0, C0, w.n, L), w.tol, w.cap)
        base = torch.cuda.memory_allocated()
        ctx = B.Context(d=w.d, n=w.n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=L)
        t = ctx.tt_from_host(x, max_rank=w.cap)
        log = []
        want, _ = tt.rk4_step(x, w.dt, model.mpo_blocks(w.d, w.n, L, w.nu), model.mpo_bond_dims(w.d),
                              w.tol, w.cap, record=log)
        ctx.hopf_step(t, w.dt, 1, replay=np.array(log))
        held = torch.cuda.memory_allocated() - base
        got = tt.full(ctx.tt_to_host(t))
        err = np.linalg.norm(got - tt.full(want)) / np.linalg.norm(tt.full(want))
        try:
            B.hopf_set_allocator(None, None)
            changed = True
        except B.HopfError:
            changed = False  # objects alive: refused
        ctx.tt_free(t)
        ctx.close()
        B.hopf_set_allocator(None, None)
        print(err, held, changed)
    """)
    err, held, changed = out.split()
    assert float(err) < 1e-12
    assert int(held) > 0
    assert changed == "False"


def test_refusing_allocator_gives_enomem_and_the_context_recovers():
    out = _run("""
        import numpy as np, torch
        from paper_2403_04946_gb300 import binding as B
        import synthetic
        dev = torch.cuda.current_device()
        budget = {"left": 64 << 20}
        def alloc(nb):
            if nb > budget["left"]:
                return 0
            budget["left"] -= nb
            return torch.cuda.caching_allocator_alloc(nb, dev)
        B.hopf_set_allocator(alloc, lambda p: torch.cuda.caching_allocator_delete(p))
        d, n = 5, 64
        ctx = B.Context(d=d, n=n, nu=0.05, tol=1e-8, rank_cap=16, L=3.0)
        small = synthetic.random_tt_cores(d, n, [1, 4, 4, 4, 4, 1], seed=75)
        try:
            ctx.tt_create(600)          # 5 cores of 600 x 64 x 600 complex: far over the budget
            status = "ok"
        except B.HopfError as e:
            status = e.status
        t = ctx.tt_from_host(small)     # small requests still succeed
        back = ctx.tt_to_host(t)
        same = all(np.array_equal(a, b) for a, b in zip(small, back))
        ctx.tt_free(t)
        ctx.close()
        B.hopf_set_allocator(None, None)
        print(status, same)
    """)
    status, same = out.split()
    from paper_2403_04946_gb300 import binding as B
    assert int(status) == B.HOPF_ENOMEM
    assert same == "True"
