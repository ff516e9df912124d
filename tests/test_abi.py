"""The C-ABI library loads and exports every function include/hopf.h
declares; the binding knows each of them; a missing library fails loudly.
No compute call is made (these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hopf.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:hopf_status|void|const char\*)\s+\**\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2403_04946_gb300 import build
    return build.build()


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for call in ("hopf_init_gaussian", "hopf_apply_op", "tt_round", "hopf_step", "hopf_eval_moments"):
        assert call in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2403_04946_gb300 import binding
    assert sorted(binding.SIGNATURES) == _declared()


def test_missing_library_fails_loudly(tmp_path):
    from paper_2403_04946_gb300 import binding
    saved = binding._LIB
    binding._LIB = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            binding.load(str(tmp_path / "nope.so"))
    finally:
        binding._LIB = saved


def test_core_layout_roundtrip():
    """The binding's flattening is the paper's column-major core layout."""
    import numpy as np
    from paper_2403_04946_gb300 import binding
    import synthetic
    cores = synthetic.random_tt_cores(4, 5, [1, 2, 3, 2, 1], 0)
    ranks, flat = binding.cores_to_flat(cores)
    z = flat.view(np.complex128)
    C = cores[1]
    a, b, c = C.shape
    off = cores[0].size
    for i in range(a):
        for j in range(b):
            for k in range(c):
                assert z[off + i + a * j + a * b * k] == C[i, j, k]
    back = binding.flat_to_cores(flat, list(ranks), 5)
    for x, y in zip(cores, back):
        assert np.array_equal(x, y)


def test_argument_errors_are_status_codes_before_any_device_work(libpath):
    """Bad arguments come back as HOPF_EINVAL from the host-side checks that
    run before any CUDA call; null handles are accepted by the free calls."""
    from paper_2403_04946_gb300 import binding as B
    lib = B.load()
    out = ctypes.c_void_p(123)
    assert lib.hopf_create(None, None, ctypes.byref(out)) == B.HOPF_EINVAL
    good = dict(d=4, n=8, nu=0.05, L=1.0, tol=1e-10, rank_cap=4, precision=B.HOPF_FP64, nonlinear=1)
    for bad in (dict(d=2), dict(n=7), dict(n=2), dict(rank_cap=0), dict(tol=-1.0),
                dict(precision=5), dict(nu=-0.1)):
        p = B.HopfParams(**{**good, **bad})
        out = ctypes.c_void_p(123)
        assert lib.hopf_create(ctypes.byref(p), None, ctypes.byref(out)) == B.HOPF_EINVAL, bad
        assert out.value is None
    for call, args in (("hopf_set_L", (None, 1.0)), ("hopf_set_nu", (None, 0.1)),
                       ("hopf_set_max_ctas", (None, 4)), ("hopf_set_svd_method", (None, 0))):
        assert getattr(lib, call)(*args) == B.HOPF_EINVAL, call
    L = ctypes.c_double()
    assert lib.hopf_get_L(None, ctypes.byref(L)) == B.HOPF_EINVAL
    assert lib.hopf_step_ensemble(-1, None, None, None, 1, None) == B.HOPF_EINVAL
    assert lib.hopf_step_ensemble(1, None, None, None, 1, None) == B.HOPF_EINVAL
    h = ctypes.c_void_p(123)
    mp = B.HopfMlpParams(12, 8, 1, 3, 1, 4)
    assert lib.hopf_mlp_create(None, ctypes.byref(mp), None, ctypes.byref(h)) == B.HOPF_EINVAL
    assert lib.hopf_last_error(None) == b"null context"
    lib.hopf_destroy(None)
    lib.tt_free(None)
    lib.hopf_mlp_free(None)
