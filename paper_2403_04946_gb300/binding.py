"""Thin ctypes binding of the C ABI in include/hopf.h.

Argument marshalling only: every numerical step runs in the CUDA library
libhopf.so.  The names follow the C calls (hopf_create, hopf_init_gaussian,
hopf_apply_op, tt_round, hopf_step, hopf_eval_moments, ...).  There is no CPU
fallback: if the library is missing or cannot be loaded, ``load`` raises.

Cores cross the boundary as numpy complex128 arrays of shape (r_{k-1}, n, r_k)
in the paper's column-major layout C[i,j,k] = v[i + a j + a b k] (App. A).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhopf.so")

HOPF_OK, HOPF_EINVAL, HOPF_ENOMEM, HOPF_ECUDA, HOPF_ENUMERIC, HOPF_ETIMEOUT, HOPF_ERANKCAP = range(7)
STATUS_NAMES = ["HOPF_OK", "HOPF_EINVAL", "HOPF_ENOMEM", "HOPF_ECUDA", "HOPF_ENUMERIC",
                "HOPF_ETIMEOUT", "HOPF_ERANKCAP"]
HOPF_FP64, HOPF_MIXED = 0, 1
HOPF_SVD_AUTO, HOPF_SVD_JACOBI = 0, 1
HOPF_RK4, HOPF_EULER, HOPF_MIDPOINT = 0, 1, 2
HOPF_EQ_PHI, HOPF_EQ_CDF = 0, 1
HOPF_QR_DOUBLEFLOAT, HOPF_QR_TENSOR = 0, 1
SCHEME_ROUNDINGS = {HOPF_RK4: 8, HOPF_EULER: 2, HOPF_MIDPOINT: 3}

# Every symbol include/hopf.h declares, with (restype, argtypes).
_vp, _i, _d, _sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
_pi, _pd = C.POINTER(C.c_int), C.POINTER(C.c_double)
SIGNATURES = {
    "hopf_create": (_i, [_vp, _vp, C.POINTER(_vp)]),
    "hopf_destroy": (None, [_vp]),
    "hopf_last_error": (C.c_char_p, [_vp]),
    "hopf_set_L": (_i, [_vp, _d]),
    "hopf_get_L": (_i, [_vp, _pd]),
    "hopf_set_nu": (_i, [_vp, _d]),
    "hopf_set_svd_method": (_i, [_vp, _i]),
    "hopf_set_qr_method": (_i, [_vp, _i]),
    "hopf_set_autotune": (_i, [_vp, _i]),
    "hopf_get_autotune": (_i, [_vp, _pi, C.POINTER(C.c_float), _i, _pi]),
    "hopf_set_wait_limit": (_i, [_vp, _d]),
    "hopf_check_watchdog": (_i, [_vp]),
    "hopf_set_allocator": (_i, [_vp, _vp, _vp]),
    "tt_save": (_i, [_vp, C.c_char_p, _d]),
    "tt_load": (_i, [_vp, C.c_char_p, _i, C.POINTER(_vp), _pd]),
    "hopf_set_max_ctas": (_i, [_vp, _i]),
    "hopf_step_ensemble": (_i, [_i, _vp, _vp, _vp, _i, _vp]),
    "hopf_cell_moments": (_i, [_vp, _i, _pd, _pd, _d, _d, _pd, _pd]),
    "tt_from_host": (_i, [_vp, _pi, _pd, _i, C.POINTER(_vp)]),
    "tt_create": (_i, [_vp, _i, C.POINTER(_vp)]),
    "tt_get_ranks": (_i, [_vp, _pi]),
    "tt_size": (_i, [_vp, C.POINTER(_sz)]),
    "tt_to_host": (_i, [_vp, _pd, _sz]),
    "tt_copy": (_i, [_vp, _vp, _vp]),
    "tt_free": (None, [_vp]),
    "hopf_init_gaussian": (_i, [_vp, _pd, _pd, C.POINTER(_vp)]),
    "hopf_apply_op": (_i, [_vp, _vp, _vp]),
    "tt_round": (_i, [_vp, _vp, _d, _i, _pi, _pd]),
    "tt_sum": (_i, [_vp, _i, C.POINTER(_vp), _pd, _vp]),
    "hopf_step": (_i, [_vp, _vp, _d, _i, _pd, _pi, _pi]),
    "hopf_step_scheme": (_i, [_vp, _vp, _i, _d, _i, _pd, _pi, _pi]),
    "hopf_set_equation": (_i, [_vp, _i, _d]),
    "hopf_init_cdf": (_i, [_vp, _d, _pd, C.POINTER(_vp)]),
    "hopf_eval_moments": (_i, [_vp, _vp, _pd, _pd, _pd]),
    "hopf_eval_points": (_i, [_vp, _vp, _i, _pi, _pd]),
    "tt_norm": (_i, [_vp, _vp, _pd]),
    "tt_set_from_host": (_i, [_vp, _pi, _pd]),
    "hopf_profile_enable": (_i, [_vp, _i]),
    "hopf_profile_read": (_i, [_vp, _vp, _i]),
    "hopf_eval_points_noalloc": (_i, [_vp, _i, _pi, _pd]),
    "hopf_tc_zgemm": (_i, [_vp, _i, _i, _i, _pd, _i, _i, _pd, _i, _i, _i, _pd, _i]),
    "hopf_mlp_create": (_i, [_vp, _vp, _vp, C.POINTER(_vp)]),
    "hopf_mlp_param_count": (_i, [_vp, C.POINTER(C.c_longlong)]),
    "hopf_mlp_get_params": (_i, [_vp, _vp]),
    "hopf_mlp_set_data": (_i, [_vp, _i, _pd, _pd, _pd]),
    "hopf_mlp_train": (_i, [_vp, _i, _i, _pi, _vp, _vp]),
    "hopf_mlp_loss_grad": (_i, [_vp, _i, _pi, _vp, _vp]),
    "hopf_mlp_predict": (_i, [_vp, _i, _pd, _pd, _pd, _d, _pd, _pd, _pd]),
    "hopf_mlp_free": (None, [_vp]),
}

KERNEL_CLASSES = ["qr", "apply_q", "svd", "apply", "gemm", "sum", "small", "tc"]

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
_allocator_keepalive = []


def hopf_set_allocator(alloc=None, free=None):
    """Route the library's device allocations through alloc(bytes) -> int
    pointer (0 on failure) and free(ptr); both None restores cudaMalloc.
    Only while no context, tensor or network exists (else HopfError)."""
    lib = load()
    if alloc is None and free is None:
        st = lib.hopf_set_allocator(None, None, None)
        if st != HOPF_OK:
            raise HopfError(st, "hopf_set_allocator: objects are alive")
        _allocator_keepalive.clear()
        return
    fa = ALLOC_FN(lambda nbytes, user: alloc(nbytes) or None)
    ff = FREE_FN(lambda ptr, user: free(ptr))
    st = lib.hopf_set_allocator(C.cast(fa, C.c_void_p), C.cast(ff, C.c_void_p), None)
    if st != HOPF_OK:
        raise HopfError(st, "hopf_set_allocator: objects are alive or a function is missing")
    _allocator_keepalive[:] = [fa, ff]


class HopfProfile(C.Structure):
    _fields_ = [("ms", C.c_double * 8), ("flops", C.c_double * 8), ("bytes", C.c_double * 8),
                ("launches", C.c_longlong * 8), ("timed_launches", C.c_longlong * 8),
                ("svd_count", C.c_longlong), ("svd_sweeps", C.c_longlong)]


class HopfParams(C.Structure):
    _fields_ = [("d", C.c_int), ("n", C.c_int), ("nu", C.c_double), ("L", C.c_double),
                ("tol", C.c_double), ("rank_cap", C.c_int), ("precision", C.c_int),
                ("nonlinear", C.c_int)]


class HopfMlpParams(C.Structure):
    _fields_ = [("n_in", C.c_int), ("width", C.c_int), ("depth", C.c_int), ("n_out", C.c_int),
                ("members", C.c_int), ("max_batch", C.c_int)]


class HopfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


_LIB = None


def load(path: str = LIB_PATH):
    """Load libhopf.so (raises if it is missing: there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(_pd)


def _iptr(a):
    return a.ctypes.data_as(_pi)


def cores_to_flat(cores):
    """List of (r_{k-1}, n, r_k) complex arrays -> (ranks, interleaved doubles)."""
    ranks = [1] + [int(c.shape[2]) for c in cores]
    flat = np.concatenate([np.asarray(c, dtype=np.complex128).reshape(-1, order="F") for c in cores])
    return np.asarray(ranks, dtype=np.int32), np.ascontiguousarray(flat).view(np.float64)


def flat_to_cores(flat, ranks, n):
    z = np.ascontiguousarray(flat).view(np.complex128)
    out, off = [], 0
    for k in range(len(ranks) - 1):
        ne = ranks[k] * n * ranks[k + 1]
        out.append(np.asfortranarray(z[off:off + ne].reshape((ranks[k], n, ranks[k + 1]), order="F")))
        off += ne
    return out


@dataclass
class Context:
    """Owns one hopf_ctx; TT handles are plain ints (void*)."""

    d: int
    n: int
    nu: float
    tol: float
    rank_cap: int
    L: float = 0.0
    nonlinear: bool = True
    stream: int | None = None
    precision: int = HOPF_FP64

    def __post_init__(self):
        self.lib = load()
        p = HopfParams(self.d, self.n, self.nu, self.L, self.tol, self.rank_cap, int(self.precision),
                       1 if self.nonlinear else 0)
        h = C.c_void_p()
        st = self.lib.hopf_create(C.byref(p), C.c_void_p(self.stream) if self.stream else None, C.byref(h))
        if st != HOPF_OK:
            raise HopfError(st, "hopf_create failed")
        self.h = h

    # -- helpers --------------------------------------------------------------
    def _check(self, st, allow=(HOPF_OK,)):
        if st not in allow:
            raise HopfError(st, self.lib.hopf_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.hopf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls ----------------------------------------------------------------
    def hopf_set_L(self, L):
        self._check(self.lib.hopf_set_L(self.h, float(L)))

    def hopf_set_nu(self, nu):
        self._check(self.lib.hopf_set_nu(self.h, float(nu)))
        self.nu = float(nu)

    def hopf_set_max_ctas(self, max_ctas):
        self._check(self.lib.hopf_set_max_ctas(self.h, int(max_ctas)))

    def hopf_set_wait_limit(self, seconds):
        self._check(self.lib.hopf_set_wait_limit(self.h, float(seconds)))

    def hopf_check_watchdog(self):
        """Status of the watchdog check (HOPF_ETIMEOUT when it works)."""
        return self.lib.hopf_check_watchdog(self.h)

    def tt_save(self, t, path, time=0.0):
        self._check(self.lib.tt_save(t, str(path).encode(), float(time)))

    def tt_load(self, path, max_rank=0):
        h = C.c_void_p()
        tm = C.c_double()
        self._check(self.lib.tt_load(self.h, str(path).encode(), int(max_rank), C.byref(h), C.byref(tm)))
        return h, tm.value

    def hopf_set_qr_method(self, method):
        self._check(self.lib.hopf_set_qr_method(self.h, int(method)))

    def hopf_set_autotune(self, enable=True):
        self._check(self.lib.hopf_set_autotune(self.h, 1 if enable else 0))

    def hopf_get_autotune(self):
        """The autotuning table: one dict per tuned shape."""
        cnt = C.c_int()
        self._check(self.lib.hopf_get_autotune(self.h, None, None, 0, C.byref(cnt)))
        n = cnt.value
        shapes = (C.c_int * (4 * max(n, 1)))()
        ms = (C.c_float * (4 * max(n, 1)))()
        self._check(self.lib.hopf_get_autotune(self.h, shapes, ms, n, C.byref(cnt)))
        names = ["tensor_all", "tensor_half", "doublefloat_all", "doublefloat_half"]
        out = []
        for i in range(n):
            out.append({"m": shapes[4 * i], "p": shapes[4 * i + 1],
                        "method": "tensor" if shapes[4 * i + 2] == HOPF_QR_TENSOR else "doublefloat",
                        "ctas": shapes[4 * i + 3] or "all",
                        "ms": {names[j]: (None if ms[4 * i + j] == float("inf") else round(ms[4 * i + j], 3))
                               for j in range(4)}})
        return out

    def hopf_set_svd_method(self, method):
        self._check(self.lib.hopf_set_svd_method(self.h, int(method)))

    def hopf_get_L(self):
        v = C.c_double()
        self._check(self.lib.hopf_get_L(self.h, C.byref(v)))
        return v.value

    def hopf_cell_moments(self, alpha, beta, sigma, ell):
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        b = np.ascontiguousarray(beta, dtype=np.float64)
        m0 = np.zeros(self.d)
        C0 = np.zeros(self.d * self.d)
        self._check(self.lib.hopf_cell_moments(self.h, len(a), _dptr(a), _dptr(b), float(sigma), float(ell),
                                               _dptr(m0), _dptr(C0)))
        return m0, C0.reshape(self.d, self.d, order="F")

    def tt_from_host(self, cores, max_rank=None):
        ranks, flat = cores_to_flat(cores)
        max_rank = int(max_rank or max(ranks))
        h = C.c_void_p()
        self._check(self.lib.tt_from_host(self.h, _iptr(ranks), _dptr(flat), max_rank, C.byref(h)))
        return h

    def tt_create(self, max_rank):
        h = C.c_void_p()
        self._check(self.lib.tt_create(self.h, int(max_rank), C.byref(h)))
        return h

    def tt_get_ranks(self, t):
        r = np.zeros(self.d + 1, dtype=np.int32)
        self._check(self.lib.tt_get_ranks(t, _iptr(r)))
        return [int(x) for x in r]

    def tt_to_host(self, t):
        nd = C.c_size_t()
        self._check(self.lib.tt_size(t, C.byref(nd)))
        buf = np.zeros(nd.value, dtype=np.float64)
        self._check(self.lib.tt_to_host(t, _dptr(buf), nd.value))
        return flat_to_cores(buf, self.tt_get_ranks(t), self.n)

    def tt_copy(self, src, dst):
        self._check(self.lib.tt_copy(self.h, src, dst))

    def tt_free(self, t):
        self.lib.tt_free(t)

    def hopf_init_gaussian(self, m0, C0):
        m = np.ascontiguousarray(m0, dtype=np.float64)
        c = np.asfortranarray(C0, dtype=np.float64).reshape(-1, order="F").copy()
        h = C.c_void_p()
        self._check(self.lib.hopf_init_gaussian(self.h, _dptr(m), _dptr(c), C.byref(h)),
                    allow=(HOPF_OK, HOPF_ERANKCAP))
        return h

    def hopf_apply_op(self, t_in, t_out):
        self._check(self.lib.hopf_apply_op(self.h, t_in, t_out))

    def tt_round(self, t, tol, cap, forced_ranks=None):
        f = None if forced_ranks is None else np.ascontiguousarray(forced_ranks, dtype=np.int32)
        disc = C.c_double()
        st = self._check(self.lib.tt_round(self.h, t, float(tol), int(cap), None if f is None else _iptr(f),
                                           C.byref(disc)), allow=(HOPF_OK, HOPF_ERANKCAP))
        return disc.value, st

    def tt_sum(self, terms, coefs, out):
        arr = (C.c_void_p * len(terms))(*[t.value if isinstance(t, C.c_void_p) else t for t in terms])
        cf = np.zeros(2 * len(coefs))
        cf[0::2] = np.real(coefs)
        cf[1::2] = np.imag(coefs)
        self._check(self.lib.tt_sum(self.h, len(terms), arr, _dptr(cf), out))

    def hopf_step(self, t, dt, nsteps, record=False, replay=None):
        disc = C.c_double()
        log = np.zeros(8 * nsteps * (self.d + 1), dtype=np.int32) if record else None
        rep = None if replay is None else np.ascontiguousarray(replay, dtype=np.int32).reshape(-1)
        st = self._check(self.lib.hopf_step(self.h, t, float(dt), int(nsteps), C.byref(disc),
                                            None if log is None else _iptr(log),
                                            None if rep is None else _iptr(rep)),
                         allow=(HOPF_OK, HOPF_ERANKCAP))
        out = {"discarded": disc.value, "status": st}
        if record:
            out["ranks"] = log.reshape(8 * nsteps, self.d + 1)
        return out

    def hopf_step_scheme(self, t, scheme, dt, nsteps, record=False, replay=None):
        """nsteps of HOPF_RK4 / HOPF_EULER / HOPF_MIDPOINT (rank logs of
        SCHEME_ROUNDINGS[scheme] roundings per step)."""
        per = SCHEME_ROUNDINGS[scheme]
        disc = C.c_double()
        log = np.zeros(per * nsteps * (self.d + 1), dtype=np.int32) if record else None
        rep = None if replay is None else np.ascontiguousarray(replay, dtype=np.int32).reshape(-1)
        st = self._check(self.lib.hopf_step_scheme(self.h, t, int(scheme), float(dt), int(nsteps), C.byref(disc),
                                                   None if log is None else _iptr(log),
                                                   None if rep is None else _iptr(rep)),
                         allow=(HOPF_OK, HOPF_ERANKCAP))
        out = {"discarded": disc.value, "status": st}
        if record:
            out["ranks"] = log.reshape(per * nsteps, self.d + 1)
        return out

    def hopf_set_equation(self, equation, box):
        self._check(self.lib.hopf_set_equation(self.h, int(equation), float(box)))

    def hopf_init_cdf(self, sigma=0.25, mu=None):
        h = C.c_void_p()
        m = None if mu is None else np.ascontiguousarray(mu, dtype=np.float64)
        self._check(self.lib.hopf_init_cdf(self.h, float(sigma), None if m is None else _dptr(m), C.byref(h)))
        return h

    def hopf_eval_moments(self, t):
        mean = np.zeros(self.d)
        cov = np.zeros(self.d * self.d)
        ir = C.c_double()
        self._check(self.lib.hopf_eval_moments(self.h, t, _dptr(mean), _dptr(cov), C.byref(ir)))
        return mean, cov.reshape(self.d, self.d, order="F"), ir.value

    def hopf_eval_points(self, t, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        vals = np.zeros(2 * idx.shape[0])
        self._check(self.lib.hopf_eval_points(self.h, t, idx.shape[0], _iptr(idx), _dptr(vals)))
        return vals.view(np.complex128)

    def tt_set_from_host(self, t, cores=None, ranks=None, flat=None):
        """Overwrite t from host cores, or from (ranks, flat doubles) already
        staged (e.g. in pinned memory: flat may be a ctypes pointer)."""
        if cores is not None:
            ranks, flat = cores_to_flat(cores)
        ranks = np.ascontiguousarray(ranks, dtype=np.int32)
        ptr = flat if isinstance(flat, C.POINTER(C.c_double)) else _dptr(flat)
        self._check(self.lib.tt_set_from_host(t, _iptr(ranks), ptr))

    def tt_to_host_into(self, t, ptr, ndoubles):
        """Download into a caller buffer (ctypes double pointer)."""
        self._check(self.lib.tt_to_host(t, ptr, int(ndoubles)))

    def tt_size(self, t):
        nd = C.c_size_t()
        self._check(self.lib.tt_size(t, C.byref(nd)))
        return nd.value

    def hopf_profile_enable(self, on=True):
        self._check(self.lib.hopf_profile_enable(self.h, 1 if on else 0))

    def hopf_profile_read(self, reset=True):
        p = HopfProfile()
        self._check(self.lib.hopf_profile_read(self.h, C.byref(p), 1 if reset else 0))
        out = {name: {"ms": p.ms[i], "flops": p.flops[i], "bytes": p.bytes[i],
                      "launches": int(p.launches[i]), "timed_launches": int(p.timed_launches[i])}
               for i, name in enumerate(KERNEL_CLASSES)}
        out["svd"]["count"] = int(p.svd_count)
        out["svd"]["sweeps"] = int(p.svd_sweeps)
        return out

    def hopf_eval_points_noalloc(self, t, idx):
        """As hopf_eval_points, staged in the library's fixed device arrays
        (no device allocation; at most 2048 points per call)."""
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        vals = np.zeros(2 * idx.shape[0])
        self._check(self.lib.hopf_eval_points_noalloc(t, idx.shape[0], _iptr(idx), _dptr(vals)))
        return vals.view(np.complex128)

    def hopf_tc_zgemm(self, A, B, opA=0, opB=0, digits=5):
        """op(A) op(B) through the tensor-core digit products (op 1 = conj
        transpose); A, B complex numpy matrices."""
        A = np.asfortranarray(A, dtype=np.complex128)
        B = np.asfortranarray(B, dtype=np.complex128)
        M, K = (A.shape[1], A.shape[0]) if opA else A.shape
        K2, N = (B.shape[1], B.shape[0]) if opB else B.shape
        if K != K2:
            raise ValueError("inner dimensions differ")
        Cm = np.zeros((M, N), dtype=np.complex128, order="F")
        flat = lambda X: X.reshape(-1, order="F").view(np.float64)  # views of the F-ordered data
        self._check(self.lib.hopf_tc_zgemm(self.h, M, N, K, _dptr(flat(A)), A.shape[0], int(opA), _dptr(flat(B)),
                                           B.shape[0], int(opB), int(digits), _dptr(flat(Cm)), M))
        return Cm

    def tt_norm(self, t):
        v = C.c_double()
        self._check(self.lib.tt_norm(self.h, t, C.byref(v)))
        return v.value


def hopf_step_ensemble(members, dt, nsteps):
    """hopf_step_ensemble: advances every (Context, tt) member by nsteps RK4
    steps, all members at once (one host thread per member inside the
    library, each on its context's stream).  dt: one value or one per
    member.  Returns the per-member statuses; raises on a failure."""
    lib = load()
    k = len(members)
    ctxs = (C.c_void_p * k)(*[m[0].h.value for m in members])
    tts = (C.c_void_p * k)(*[t.value if isinstance(t, C.c_void_p) else t for _, t in members])
    dts = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (k,)))
    sts = np.zeros(k, dtype=np.int32)
    st = lib.hopf_step_ensemble(k, ctxs, tts, _dptr(dts), int(nsteps), _iptr(sts))
    if st not in (HOPF_OK, HOPF_ERANKCAP):
        bad = [i for i in range(k) if sts[i] not in (HOPF_OK, HOPF_ERANKCAP)]
        msg = members[bad[0]][0].lib.hopf_last_error(members[bad[0]][0].h).decode() if bad else ""
        raise HopfError(st, msg)
    return [int(x) for x in sts]


def _fptr(a):
    return a.ctypes.data_as(C.c_void_p)


class Mlp:
    """hopf_mlp_*: the surrogate network ensemble of the library (BF16
    weights, FP32 activations and accumulation, Adam).  Parameters cross
    the boundary as float32 arrays [members][P] in the header's packed
    layout; data and predictions as float64."""

    def __init__(self, ctx, n_in, width, depth, n_out, members, max_batch, init):
        self.ctx, self.lib = ctx, ctx.lib
        self.p = HopfMlpParams(n_in, width, depth, n_out, members, max_batch)
        self.P = self.param_count(self.lib, self.p)
        init = np.ascontiguousarray(init, dtype=np.float32).reshape(members, self.P)
        h = C.c_void_p()
        ctx._check(self.lib.hopf_mlp_create(ctx.h, C.byref(self.p), _fptr(init), C.byref(h)))
        self.h = h

    @staticmethod
    def param_count(lib, p):
        P = C.c_longlong()
        st = lib.hopf_mlp_param_count(C.byref(p), C.byref(P))
        if st != HOPF_OK:
            raise HopfError(st, "hopf_mlp_param_count: bad network shape")
        return int(P.value)

    def close(self):
        if self.h:
            self.lib.hopf_mlp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = np.zeros((self.p.members, self.P), dtype=np.float32)
        self.ctx._check(self.lib.hopf_mlp_get_params(self.h, _fptr(out)))
        return out

    def set_data(self, x, y):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        stats = np.zeros(2 * (self.p.n_in + self.p.n_out))
        self.ctx._check(self.lib.hopf_mlp_set_data(self.h, x.shape[0], _dptr(x), _dptr(y), _dptr(stats)))
        ni = self.p.n_in
        return (stats[:ni], stats[ni:2 * ni]), (stats[2 * ni:2 * ni + self.p.n_out], stats[2 * ni + self.p.n_out:])

    def train(self, idx, lr):
        """idx: int [iters][members][batch]; lr: [iters].  Returns the batch
        losses [iters][members]."""
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        iters, _, batch = idx.shape
        lr = np.ascontiguousarray(lr, dtype=np.float32)
        loss = np.zeros((iters, self.p.members), dtype=np.float32)
        self.ctx._check(self.lib.hopf_mlp_train(self.h, iters, batch, _iptr(idx), _fptr(lr), _fptr(loss)))
        return loss

    def loss_grad(self, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        loss = np.zeros(self.p.members, dtype=np.float32)
        grad = np.zeros((self.p.members, self.P), dtype=np.float32)
        self.ctx._check(self.lib.hopf_mlp_loss_grad(self.h, idx.shape[1], _iptr(idx), _fptr(loss), _fptr(grad)))
        return loss, grad

    def predict(self, x, kappa, base=None, scale=None, members=False):
        x = np.ascontiguousarray(x, dtype=np.float64)
        nq = x.shape[0]
        bs = None if base is None else np.ascontiguousarray(base, dtype=np.float64).reshape(nq, self.p.n_out)
        sc = None if scale is None else np.ascontiguousarray(scale, dtype=np.float64).reshape(nq)
        y = np.zeros((nq, self.p.n_out))
        bound = np.zeros(nq)
        ym = np.zeros((self.p.members, nq, self.p.n_out)) if members else None
        self.ctx._check(self.lib.hopf_mlp_predict(
            self.h, nq, _dptr(x), None if bs is None else _dptr(bs), None if sc is None else _dptr(sc),
            float(kappa), _dptr(y), _dptr(bound), _dptr(ym) if members else None))
        return (y, bound, ym) if members else (y, bound)
