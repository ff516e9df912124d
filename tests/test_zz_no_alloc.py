"""The allocation-free point evaluation (hopf_eval_points_noalloc) against
the allocating one (hopf_eval_points), through the C ABI.

hopf_eval_points_noalloc exists for callers that cannot allocate device
memory (a monitor probing Phi between solver steps must not call cudaFree,
which waits for the whole device; a process whose memory is reserved by
another allocator may not get any).  It stages its data in fixed arrays of
the library instead.  This file is collected last on purpose, and passes
both alone in a fresh process and after the other GPU tests."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2403_04946_gb300 import binding, build
    build.build()
    return binding


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_allocating_entry_point_on_two_calls(B):
    d, n = 7, 24
    x = synthetic.random_tt_cores(d, n, [1, 5, 9, 12, 12, 9, 5, 1], seed=21)
    ctx = B.Context(d=d, n=n, nu=0.05, tol=1e-10, rank_cap=16, L=3.0)
    t = ctx.tt_from_host(x)
    # two calls in a row with different point sets: the second call must not
    # see anything left over from the first
    for npts, seed in ((1500, 1), (37, 2)):
        idx = synthetic.random_probe_indices(d, n, npts, seed)
        want = ctx.hopf_eval_points(t, idx)
        got = ctx.hopf_eval_points_noalloc(t, idx)
        assert got.shape == want.shape
        assert rel(got, want) < 1e-14
    ctx.tt_free(t)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_arrays(B):
    d, n = 4, 8
    x = synthetic.random_tt_cores(d, n, [1, 2, 2, 2, 1], seed=22)
    ctx = B.Context(d=d, n=n, nu=0.05, tol=1e-10, rank_cap=4, L=3.0)
    t = ctx.tt_from_host(x)
    too_many = synthetic.random_probe_indices(d, n, 2049, 3)
    with pytest.raises(B.HopfError) as err:
        ctx.hopf_eval_points_noalloc(t, too_many)
    assert err.value.status == B.HOPF_EINVAL
    # the context stays usable
    idx = synthetic.random_probe_indices(d, n, 10, 4)
    assert rel(ctx.hopf_eval_points_noalloc(t, idx), ctx.hopf_eval_points(t, idx)) < 1e-14
    ctx.tt_free(t)
    ctx.close()


def test_noalloc_leaves_device_memory_unchanged(B):
    """The property the entry point exists for: a burst of calls takes no
    device memory.  The first call is made before the measurement (the
    library's module, which holds the two arrays, may be loaded lazily on
    first use); after it the device's free memory must not move."""
    torch = pytest.importorskip("torch")
    d, n = 6, 16
    x = synthetic.random_tt_cores(d, n, [1, 4, 8, 8, 8, 4, 1], seed=23)
    ctx = B.Context(d=d, n=n, nu=0.05, tol=1e-10, rank_cap=8, L=3.0)
    t = ctx.tt_from_host(x)
    idx = synthetic.random_probe_indices(d, n, 2048, 5)
    first = ctx.hopf_eval_points_noalloc(t, idx)
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(25):
        got = ctx.hopf_eval_points_noalloc(t, idx)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    np.testing.assert_array_equal(got, first)
    ctx.tt_free(t)
    ctx.close()
