"""ctypes binding of libmertens (include/libmertens.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers may be given as torch tensors or raw integer device
pointers; streams as torch.cuda.Stream, raw handles or None.  There is no CPU
fallback: if the library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

MERTENS_OK = 0
MERTENS_EINVAL = 1
MERTENS_ENOMEM = 2
MERTENS_ECUDA = 3
MERTENS_ETIMEOUT = 4
MERTENS_ENOTREADY = 5
MERTENS_ENOTSUP = 6
MERTENS_EOVERFLOW = 7


class mertens_u128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_uint64)]


class mertens_query_info(ctypes.Structure):
    _fields_ = [("n", mertens_u128), ("u", mertens_u128), ("X", ctypes.c_uint64),
                ("y_max", ctypes.c_uint64), ("direct_terms", ctypes.c_uint64),
                ("gathered_terms", ctypes.c_uint64)]


class mertens_run_stats(ctypes.Structure):
    _fields_ = [("total_ms", ctypes.c_double), ("sieve_ms", ctypes.c_double),
                ("scan_ms", ctypes.c_double), ("update_ms", ctypes.c_double),
                ("dense_ms", ctypes.c_double), ("gather_ms", ctypes.c_double),
                ("resolve_ms", ctypes.c_double), ("runs", ctypes.c_uint64),
                ("blocks", ctypes.c_uint64), ("y_sieved", ctypes.c_uint64),
                ("terms", ctypes.c_uint64), ("kernels", ctypes.c_uint64),
                ("dense_y", ctypes.c_uint64), ("gather_j", ctypes.c_uint64),
                ("sieve_updates", ctypes.c_double),
                ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64),
                ("gather_j_exec", ctypes.c_uint64), ("dense_odd_skip", ctypes.c_uint64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                           ctypes.c_void_p)

# Every symbol include/libmertens.h declares.
EXPORTS = [
    "mertens_strerror", "mertens_last_error", "mertens_set_allocator", "mertens_plan",
    "mertens_run", "mertens_result", "mertens_destroy", "mertens_describe",
    "mertens_plan_info", "mertens_plan_set_profiling", "mertens_run_stats_get",
    "mertens_sieve_mu", "mertens_sieve_M", "mertens_sieve_M_noalloc",
    "mertens_set_tuning", "mertens_get_tuning", "mertens_autotune",
    "mertens_server_create", "mertens_server_submit", "mertens_server_poll",
    "mertens_server_wait", "mertens_server_times", "mertens_server_stats_get",
    "mertens_server_destroy", "mertens_plan_window", "mertens_window_result",
    "mertens_table_create", "mertens_table_info", "mertens_plan_on_table", "mertens_table_destroy",
    "mertens_server_use_table", "mertens_scan_extremes", "mertens_probe_int_peaks",
    "mertens_resolve", "mertens_window_accumulate", "mertens_resolve_exchange",
    "mertens_division_constants",
]


class mertens_extremes(ctypes.Structure):
    _fields_ = [("M_last", ctypes.c_int64), ("M_max", ctypes.c_int64), ("M_min", ctypes.c_int64),
                ("y_M_max", ctypes.c_uint64), ("y_M_min", ctypes.c_uint64),
                ("R_max_M", ctypes.c_int64), ("R_min_M", ctypes.c_int64),
                ("y_R_max", ctypes.c_uint64), ("y_R_min", ctypes.c_uint64),
                ("R_max", ctypes.c_double), ("R_min", ctypes.c_double)]


class mertens_int_peaks(ctypes.Structure):
    _fields_ = [("mulhi_terms_per_s", ctypes.c_double), ("imad32_per_s", ctypes.c_double),
                ("alu_pairs_per_s", ctypes.c_double), ("sms", ctypes.c_int),
                ("fquot_terms_per_s", ctypes.c_double)]


class mertens_tuning(ctypes.Structure):
    _fields_ = [("u_factor", ctypes.c_double), ("dense_c", ctypes.c_double),
                ("gather_scale", ctypes.c_double), ("block_cap", ctypes.c_uint64)]


class mertens_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("answered", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("max_inflight", ctypes.c_uint64),
                ("max_batch_seen", ctypes.c_uint64), ("failed", ctypes.c_uint64)]

_lock = threading.Lock()
_lib = None


class MertensError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        self.code = code
        super().__init__(f"{where}: {detail} (status {code})")


def load():
    """Builds (if stale) and loads libmertens.so; raises if that fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        u64, i64, sz, c_int = ctypes.c_uint64, ctypes.c_int64, ctypes.c_size_t, ctypes.c_int
        lib.mertens_strerror.argtypes = [c_int]
        lib.mertens_strerror.restype = ctypes.c_char_p
        lib.mertens_last_error.argtypes = []
        lib.mertens_last_error.restype = ctypes.c_char_p
        lib.mertens_set_allocator.argtypes = [ALLOC_FN, FREE_FN, P]
        lib.mertens_set_allocator.restype = c_int
        lib.mertens_plan.argtypes = [ctypes.POINTER(P), ctypes.POINTER(mertens_u128), sz,
                                     mertens_u128, u64]
        lib.mertens_plan.restype = c_int
        lib.mertens_plan_window.argtypes = [ctypes.POINTER(P), ctypes.POINTER(mertens_u128), sz,
                                            mertens_u128, u64, u64, u64]
        lib.mertens_plan_window.restype = c_int
        lib.mertens_window_result.argtypes = [P, sz, P, P, sz, ctypes.POINTER(sz),
                                              ctypes.POINTER(i64)]
        lib.mertens_window_result.restype = c_int
        lib.mertens_table_create.argtypes = [ctypes.POINTER(P), u64, mertens_u128, P]
        lib.mertens_table_create.restype = c_int
        lib.mertens_table_info.argtypes = [P, ctypes.POINTER(u64), ctypes.POINTER(mertens_u128),
                                           ctypes.POINTER(sz)]
        lib.mertens_table_info.restype = c_int
        lib.mertens_plan_on_table.argtypes = [ctypes.POINTER(P), P, ctypes.POINTER(mertens_u128),
                                              sz, mertens_u128, u64]
        lib.mertens_plan_on_table.restype = c_int
        lib.mertens_server_use_table.argtypes = [P, P]
        lib.mertens_server_use_table.restype = c_int
        lib.mertens_scan_extremes.argtypes = [u64, u64, i64, ctypes.POINTER(mertens_extremes), P]
        lib.mertens_scan_extremes.restype = c_int
        lib.mertens_resolve.argtypes = [mertens_u128, u64, P, P, P]
        lib.mertens_resolve.restype = c_int
        lib.mertens_window_accumulate.argtypes = [P, sz, P, sz, P, P]
        lib.mertens_window_accumulate.restype = c_int
        lib.mertens_resolve_exchange.argtypes = [mertens_u128, u64, P, P, P]
        lib.mertens_resolve_exchange.restype = c_int
        lib.mertens_division_constants.argtypes = [u64, P, P, P, P]
        lib.mertens_division_constants.restype = c_int
        lib.mertens_probe_int_peaks.argtypes = [ctypes.POINTER(mertens_int_peaks), P]
        lib.mertens_probe_int_peaks.restype = c_int
        lib.mertens_table_destroy.argtypes = [P]
        lib.mertens_table_destroy.restype = None
        lib.mertens_run.argtypes = [P, P]
        lib.mertens_run.restype = c_int
        lib.mertens_result.argtypes = [P, sz, ctypes.POINTER(i64), P, sz,
                                       ctypes.POINTER(sz)]
        lib.mertens_result.restype = c_int
        lib.mertens_destroy.argtypes = [P]
        lib.mertens_destroy.restype = None
        lib.mertens_describe.argtypes = [mertens_u128, mertens_u128,
                                         ctypes.POINTER(mertens_query_info)]
        lib.mertens_describe.restype = c_int
        lib.mertens_plan_info.argtypes = [P, sz, ctypes.POINTER(mertens_query_info)]
        lib.mertens_plan_info.restype = c_int
        lib.mertens_plan_set_profiling.argtypes = [P, c_int]
        lib.mertens_plan_set_profiling.restype = c_int
        lib.mertens_run_stats_get.argtypes = [P, ctypes.POINTER(mertens_run_stats)]
        lib.mertens_run_stats_get.restype = c_int
        lib.mertens_sieve_mu.argtypes = [u64, u64, P, P]
        lib.mertens_sieve_mu.restype = c_int
        lib.mertens_sieve_M.argtypes = [u64, u64, i64, P, P]
        lib.mertens_sieve_M.restype = c_int
        lib.mertens_sieve_M_noalloc.argtypes = [u64, u64, i64, P, P]
        lib.mertens_sieve_M_noalloc.restype = c_int
        u32 = ctypes.c_uint32
        lib.mertens_set_tuning.argtypes = [ctypes.POINTER(mertens_tuning)]
        lib.mertens_set_tuning.restype = c_int
        lib.mertens_get_tuning.argtypes = [ctypes.POINTER(mertens_tuning)]
        lib.mertens_get_tuning.restype = c_int
        lib.mertens_autotune.argtypes = [ctypes.POINTER(mertens_u128), sz, c_int,
                                         ctypes.POINTER(mertens_tuning),
                                         ctypes.POINTER(ctypes.c_double)]
        lib.mertens_autotune.restype = c_int
        lib.mertens_server_create.argtypes = [ctypes.POINTER(P), c_int, sz, u32, u32]
        lib.mertens_server_create.restype = c_int
        lib.mertens_server_submit.argtypes = [P, mertens_u128, ctypes.POINTER(u64)]
        lib.mertens_server_submit.restype = c_int
        lib.mertens_server_poll.argtypes = [P, u64, ctypes.POINTER(i64)]
        lib.mertens_server_poll.restype = c_int
        lib.mertens_server_wait.argtypes = [P, u64, ctypes.POINTER(i64), ctypes.c_double]
        lib.mertens_server_wait.restype = c_int
        lib.mertens_server_times.argtypes = [P, u64, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        lib.mertens_server_times.restype = c_int
        lib.mertens_server_stats_get.argtypes = [P, ctypes.POINTER(mertens_server_stats)]
        lib.mertens_server_stats_get.restype = c_int
        lib.mertens_server_destroy.argtypes = [P]
        lib.mertens_server_destroy.restype = None
        _lib = lib
        return lib


def _check(rc: int, where: str):
    if rc != MERTENS_OK:
        lib = load()
        detail = lib.mertens_last_error().decode() or lib.mertens_strerror(rc).decode()
        raise MertensError(rc, where, detail)


def u128(v: int) -> mertens_u128:
    v = int(v)
    if v < 0 or v >= 1 << 128:
        raise ValueError("value out of the unsigned 128-bit range")
    return mertens_u128(v & ((1 << 64) - 1), v >> 64)


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    raise TypeError("expected a torch tensor or an integer device pointer")


def _stream(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    raise TypeError("expected a torch.cuda.Stream, a raw handle or None")


# ---- the C-ABI calls, same names ------------------------------------------

def mertens_strerror(code: int) -> str:
    return load().mertens_strerror(code).decode()


def mertens_last_error() -> str:
    return load().mertens_last_error().decode()


def mertens_plan(n, u: int = 0, block_len: int = 0) -> int:
    """Returns an opaque plan handle for the targets n (int or list of ints)."""
    lib = load()
    ns = [int(n)] if isinstance(n, (int, np.integer)) else [int(v) for v in n]
    arr = (mertens_u128 * len(ns))(*[u128(v) for v in ns])
    h = ctypes.c_void_p()
    _check(lib.mertens_plan(ctypes.byref(h), arr, len(ns), u128(u), int(block_len)),
           "mertens_plan")
    return int(h.value)


def mertens_plan_window(n, y_first: int, y_last: int, u: int = 0, block_len: int = 0) -> int:
    """A plan that runs only the sieve blocks of y in [y_first, y_last] (no
    resolve); read it with mertens_window_result."""
    lib = load()
    ns = [int(n)] if isinstance(n, (int, np.integer)) else [int(v) for v in n]
    arr = (mertens_u128 * len(ns))(*[u128(v) for v in ns])
    h = ctypes.c_void_p()
    _check(lib.mertens_plan_window(ctypes.byref(h), arr, len(ns), u128(u), int(block_len),
                                   int(y_first), int(y_last)), "mertens_plan_window")
    return int(h.value)


def mertens_window_result(plan: int, i: int = 0):
    """(S_loc, coef, mu_sum) of target i of a window plan: the window adds
    S_loc + C * coef (uint64 arrays, mod 2^64) to the entries' sums, C =
    M(y_first - 1); mu_sum = M(y_last) - M(y_first - 1)."""
    lib = load()
    X = mertens_plan_info(plan, i)["X"]
    S = np.zeros(X, dtype=np.uint64)
    c = np.zeros(X, dtype=np.uint64)
    ln = ctypes.c_size_t()
    mu = ctypes.c_int64()
    _check(lib.mertens_window_result(plan, i, S.ctypes.data, c.ctypes.data, X, ctypes.byref(ln),
                                     ctypes.byref(mu)), "mertens_window_result")
    return S, c, int(mu.value)


def mertens_table_create(y_max: int, n_max: int, stream=None) -> int:
    """Sieves M(y), y <= y_max, into a resident device table (with the
    update's target-independent parts for n <= n_max); returns its handle."""
    h = ctypes.c_void_p()
    _check(load().mertens_table_create(ctypes.byref(h), int(y_max), u128(n_max),
                                       _stream(stream)), "mertens_table_create")
    return int(h.value)


def mertens_table_info(table: int) -> dict:
    y = ctypes.c_uint64()
    nm = mertens_u128()
    b = ctypes.c_size_t()
    _check(load().mertens_table_info(table, ctypes.byref(y), ctypes.byref(nm), ctypes.byref(b)),
           "mertens_table_info")
    return dict(y_max=y.value, n_max=nm.lo | (nm.hi << 64), bytes=b.value)


def mertens_plan_on_table(table: int, n, u: int = 0, block_len: int = 0) -> int:
    """A plan whose M(y) comes from the resident table (no sieve)."""
    lib = load()
    ns = [int(n)] if isinstance(n, (int, np.integer)) else [int(v) for v in n]
    arr = (mertens_u128 * len(ns))(*[u128(v) for v in ns])
    h = ctypes.c_void_p()
    _check(lib.mertens_plan_on_table(ctypes.byref(h), table, arr, len(ns), u128(u),
                                     int(block_len)), "mertens_plan_on_table")
    return int(h.value)


def mertens_server_use_table(srv: int, table: int) -> None:
    _check(load().mertens_server_use_table(srv, table), "mertens_server_use_table")


def mertens_scan_extremes(y_first: int, y_last: int, carry: int, stream=None) -> dict:
    """Extremes of M(y) and M(y)/sqrt(y) for y in [y_first, y_last], given
    carry = M(y_first - 1)."""
    e = mertens_extremes()
    _check(load().mertens_scan_extremes(int(y_first), int(y_last), int(carry), ctypes.byref(e),
                                        _stream(stream)), "mertens_scan_extremes")
    return {name: getattr(e, name) for name, _ in mertens_extremes._fields_}


def mertens_resolve(n: int, u: int, S, stream=None) -> np.ndarray:
    """M(floor(n/x)), x = 1..X, from the entries' update sums S (uint64, X = n//u)."""
    S = np.ascontiguousarray(S, dtype=np.uint64)
    out = np.zeros(S.size, dtype=np.int64)
    if S.size != int(n) // int(u):
        raise ValueError("S must have floor(n/u) entries")
    _check(load().mertens_resolve(u128(n), int(u), S.ctypes.data, out.ctypes.data,
                                  _stream(stream)), "mertens_resolve")
    return out


def mertens_window_mu_sum(plan: int, i: int = 0) -> int:
    """The window's mu sum M(y_last) - M(y_first - 1) alone (8 bytes read)."""
    ln = ctypes.c_size_t()
    mu = ctypes.c_int64()
    _check(load().mertens_window_result(plan, i, None, None, 0, ctypes.byref(ln),
                                        ctypes.byref(mu)), "mertens_window_result")
    return int(mu.value)


def mertens_window_accumulate(plan: int, i: int, mu_before, X2_dev, stream=None) -> None:
    """Adds target i's window sums S_loc + C coef, C = sum(mu_before), into the
    exchange buffer X2_dev (device, 2 X int64 words: low and high 32-bit
    halves of each entry's sum)."""
    mus = np.ascontiguousarray([int(v) for v in mu_before], dtype=np.int64)
    _check(load().mertens_window_accumulate(plan, i, mus.ctypes.data if mus.size else None,
                                            mus.size, _ptr(X2_dev), _stream(stream)),
           "mertens_window_accumulate")


def mertens_resolve_exchange(n: int, u: int, X2_dev, M_dev, stream=None) -> None:
    """M(floor(n/x)), x = 1..X, into M_dev (device, X int64) from the
    exchange buffer X2_dev (device, 2 X int64 halves)."""
    _check(load().mertens_resolve_exchange(u128(n), int(u), _ptr(X2_dev), _ptr(M_dev),
                                           _stream(stream)), "mertens_resolve_exchange")


def mertens_division_constants(d: int) -> dict:
    """The kernels' invariant-divisor constants for divisor d (host only)."""
    m64, m32 = ctypes.c_uint64(), ctypes.c_uint32()
    l64, s32 = ctypes.c_uint32(), ctypes.c_uint32()
    _check(load().mertens_division_constants(int(d), ctypes.byref(m64), ctypes.byref(l64),
                                             ctypes.byref(m32), ctypes.byref(s32)),
           "mertens_division_constants")
    return dict(m64=m64.value, l64=l64.value, m32=m32.value, s32=s32.value)


def mertens_probe_int_peaks(stream=None) -> dict:
    """Measured integer rates of the current device (roofline denominators)."""
    r = mertens_int_peaks()
    _check(load().mertens_probe_int_peaks(ctypes.byref(r), _stream(stream)),
           "mertens_probe_int_peaks")
    return {name: getattr(r, name) for name, _ in mertens_int_peaks._fields_}


def mertens_table_destroy(table: int) -> None:
    if table:
        load().mertens_table_destroy(table)


def mertens_run(plan: int, stream=None) -> None:
    _check(load().mertens_run(plan, _stream(stream)), "mertens_run")


def mertens_result(plan: int, i: int = 0, entries: bool = False, cap: int | None = None):
    """(M(n_i), array or None): the array holds M(floor(n_i/x)) for x = 1..X_i."""
    lib = load()
    m = ctypes.c_int64()
    ln = ctypes.c_size_t()
    if entries:
        info = mertens_plan_info(plan, i)
        cnt = info["X"] if cap is None else min(cap, info["X"])
        out = np.zeros(cnt, dtype=np.int64)
        _check(lib.mertens_result(plan, i, ctypes.byref(m), out.ctypes.data, cnt,
                                  ctypes.byref(ln)), "mertens_result")
        return int(m.value), out
    _check(lib.mertens_result(plan, i, ctypes.byref(m), None, 0, ctypes.byref(ln)),
           "mertens_result")
    return int(m.value), None


def mertens_result_into(plan: int, i: int, out: np.ndarray) -> int:
    """Copies target i's array into the host buffer `out` (int64); returns M(n_i)."""
    lib = load()
    m = ctypes.c_int64()
    ln = ctypes.c_size_t()
    _check(lib.mertens_result(plan, i, ctypes.byref(m), out.ctypes.data, out.size,
                              ctypes.byref(ln)), "mertens_result")
    return int(m.value)


def mertens_destroy(plan: int) -> None:
    if plan:
        load().mertens_destroy(plan)


def _info_dict(info: mertens_query_info) -> dict:
    return dict(n=info.n.lo | (info.n.hi << 64), u=info.u.lo | (info.u.hi << 64), X=info.X,
                y_max=info.y_max, direct_terms=info.direct_terms,
                gathered_terms=info.gathered_terms)


def mertens_describe(n: int, u: int = 0) -> dict:
    info = mertens_query_info()
    _check(load().mertens_describe(u128(n), u128(u), ctypes.byref(info)), "mertens_describe")
    return _info_dict(info)


def mertens_plan_info(plan: int, i: int = 0) -> dict:
    info = mertens_query_info()
    _check(load().mertens_plan_info(plan, i, ctypes.byref(info)), "mertens_plan_info")
    return _info_dict(info)


def mertens_plan_set_profiling(plan: int, enable: bool = True) -> None:
    _check(load().mertens_plan_set_profiling(plan, 1 if enable else 0),
           "mertens_plan_set_profiling")


def mertens_run_stats_get(plan: int) -> dict:
    st = mertens_run_stats()
    _check(load().mertens_run_stats_get(plan, ctypes.byref(st)), "mertens_run_stats_get")
    return {name: getattr(st, name) for name, _ in mertens_run_stats._fields_}


def mertens_sieve_mu(y1: int, length: int, mu_dev, stream=None) -> None:
    _check(load().mertens_sieve_mu(int(y1), int(length), _ptr(mu_dev), _stream(stream)),
           "mertens_sieve_mu")


def mertens_sieve_M(y1: int, length: int, carry: int, M_dev, stream=None) -> None:
    _check(load().mertens_sieve_M(int(y1), int(length), int(carry), _ptr(M_dev),
                                  _stream(stream)), "mertens_sieve_M")


def mertens_sieve_M_noalloc(y1: int, length: int, carry: int, M_dev, stream=None) -> None:
    """mertens_sieve_M without any device allocation (fixed library scratch;
    len <= 2^21, y1 + len - 1 < 2^40; overlapping calls race)."""
    _check(load().mertens_sieve_M_noalloc(int(y1), int(length), int(carry), _ptr(M_dev),
                                          _stream(stream)), "mertens_sieve_M_noalloc")


def _tuning_dict(t: mertens_tuning) -> dict:
    return {name: getattr(t, name) for name, _ in mertens_tuning._fields_}


def mertens_get_tuning() -> dict:
    t = mertens_tuning()
    _check(load().mertens_get_tuning(ctypes.byref(t)), "mertens_get_tuning")
    return _tuning_dict(t)


def mertens_set_tuning(u_factor=None, dense_c=None, gather_scale=None, block_cap=None) -> dict:
    """Sets the given fields (others keep their value); returns the tuning."""
    cur = mertens_get_tuning()
    for k, v in (("u_factor", u_factor), ("dense_c", dense_c), ("gather_scale", gather_scale),
                 ("block_cap", block_cap)):
        if v is not None:
            cur[k] = v
    t = mertens_tuning(float(cur["u_factor"]), float(cur["dense_c"]),
                       float(cur["gather_scale"]), int(cur["block_cap"]))
    _check(load().mertens_set_tuning(ctypes.byref(t)), "mertens_set_tuning")
    return cur


def mertens_autotune(n, runs: int = 1):
    """(best tuning dict, ms per run) for the targets n, not applied."""
    ns = [int(n)] if isinstance(n, (int, np.integer)) else [int(v) for v in n]
    arr = (mertens_u128 * len(ns))(*[u128(v) for v in ns])
    best = mertens_tuning()
    ms = ctypes.c_double()
    _check(load().mertens_autotune(arr, len(ns), int(runs), ctypes.byref(best), ctypes.byref(ms)),
           "mertens_autotune")
    return _tuning_dict(best), float(ms.value)


def mertens_server_create(device: int = 0, mem_budget_bytes: int = 0, max_inflight: int = 0,
                          max_batch: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().mertens_server_create(ctypes.byref(h), int(device), int(mem_budget_bytes),
                                        int(max_inflight), int(max_batch)),
           "mertens_server_create")
    return int(h.value)


def mertens_server_submit(srv: int, n: int) -> int:
    t = ctypes.c_uint64()
    _check(load().mertens_server_submit(srv, u128(n), ctypes.byref(t)), "mertens_server_submit")
    return int(t.value)


def mertens_server_poll(srv: int, ticket: int):
    """M(n) of the ticket's query, or None while it is not answered yet."""
    m = ctypes.c_int64()
    rc = load().mertens_server_poll(srv, int(ticket), ctypes.byref(m))
    if rc == MERTENS_ENOTREADY:
        return None
    _check(rc, "mertens_server_poll")
    return int(m.value)


def mertens_server_wait(srv: int, ticket: int, timeout_s: float = -1.0) -> int:
    m = ctypes.c_int64()
    _check(load().mertens_server_wait(srv, int(ticket), ctypes.byref(m), float(timeout_s)),
           "mertens_server_wait")
    return int(m.value)


def mertens_server_times(srv: int, ticket: int):
    """(submit_ns, done_ns) on the host steady clock; done_ns = 0 if pending."""
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().mertens_server_times(srv, int(ticket), ctypes.byref(a), ctypes.byref(b)),
           "mertens_server_times")
    return int(a.value), int(b.value)


def mertens_server_stats_get(srv: int) -> dict:
    st = mertens_server_stats()
    _check(load().mertens_server_stats_get(srv, ctypes.byref(st)), "mertens_server_stats_get")
    return {name: getattr(st, name) for name, _ in mertens_server_stats._fields_}


def mertens_server_destroy(srv: int) -> None:
    if srv:
        load().mertens_server_destroy(srv)


_alloc_keepalive = []


def mertens_set_allocator(alloc=None, release=None, ctx=None) -> None:
    """Installs a device-memory hook (ctypes callbacks) or, with no argument,
    restores cudaMalloc/cudaFree."""
    lib = load()
    if alloc is None:
        _check(lib.mertens_set_allocator(ALLOC_FN(), FREE_FN(), None), "mertens_set_allocator")
        _alloc_keepalive.clear()
        return
    a, r = ALLOC_FN(alloc), FREE_FN(release)
    _alloc_keepalive[:] = [a, r]
    _check(lib.mertens_set_allocator(a, r, ctx), "mertens_set_allocator")


def use_torch_allocator() -> None:
    """Routes the library's device allocations through PyTorch's caching
    allocator on the current device."""
    import torch

    def _alloc(nbytes, stream, ctx):
        dev = torch.cuda.current_device()
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0))
        except RuntimeError:
            return 0

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    mertens_set_allocator(_alloc, _free)


# ---- convenience ----------------------------------------------------------

def mertens(n, u: int = 0, block_len: int = 0, entries: bool = False, stream=None):
    """M(n) (or M(n_i) for a list, one shared sieve pass), computed on the GPU.

    With entries=True each result is (M(n_i), array of M(floor(n_i/x)))."""
    single = isinstance(n, (int, np.integer))
    ns = [int(n)] if single else [int(v) for v in n]
    plan = mertens_plan(ns, u, block_len)
    try:
        mertens_run(plan, stream)
        out = [mertens_result(plan, i, entries) for i in range(len(ns))]
    finally:
        mertens_destroy(plan)
    res = [o if entries else o[0] for o in out]
    return res[0] if single else res
