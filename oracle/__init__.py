"""Plain CPU oracle for the Mertens function (arXiv:1108.0135).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_1108_0135_gb300``) never imports, links or calls it, and the two share
no code.

The arithmetic lives in ``mertens_oracle.c`` (plain C, single thread); this
module only compiles it with gcc and marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mertens_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_SO)) or os.path.getmtime(_SO) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i64, i32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32
            lib.oracle_mu_trial.argtypes = [u64]
            lib.oracle_mu_trial.restype = ctypes.c_int
            lib.oracle_isqrt_u128.argtypes = [u64, u64]
            lib.oracle_isqrt_u128.restype = u64
            lib.oracle_mu_window.argtypes = [u64, u64, ctypes.c_void_p]
            lib.oracle_mu_window.restype = ctypes.c_int
            lib.oracle_mertens_table.argtypes = [u64, ctypes.c_void_p]
            lib.oracle_mertens_table.restype = ctypes.c_int
            lib.oracle_mertens_array.argtypes = [u64, u64, u64, u64, ctypes.c_void_p]
            lib.oracle_mertens_array.restype = ctypes.c_int
            lib.oracle_count_terms.argtypes = [u64, u64, ctypes.POINTER(u64),
                                               ctypes.POINTER(u64)]
            lib.oracle_count_terms.restype = ctypes.c_int
            lib.oracle_window_sums.argtypes = [u64, u64, u64, u64, u64, u64, u64,
                                               ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.POINTER(i64)]
            lib.oracle_window_sums.restype = ctypes.c_int
            _lib = lib
    return _lib


def _split(n: int):
    if n < 0 or n >= 1 << 128:
        raise ValueError("n out of range")
    return n & ((1 << 64) - 1), n >> 64


def mu_trial(m: int) -> int:
    """mu(m) by trial division (Sec. 1 definition)."""
    return int(_load().oracle_mu_trial(m))


def isqrt(v: int) -> int:
    lo, hi = _split(v)
    return int(_load().oracle_isqrt_u128(lo, hi))


def mu_window(y1: int, length: int) -> np.ndarray:
    """mu(y) for y in [y1, y1+length) by the naive block sieve of Sec. 3."""
    out = np.zeros(length, dtype=np.int8)
    rc = _load().oracle_mu_window(y1, length, out.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_mu_window({y1}, {length}) failed: {rc}")
    return out


def mertens_table(L: int) -> np.ndarray:
    """M(y) for y = 0..L (int32), L < 2^31."""
    out = np.zeros(L + 1, dtype=np.int32)
    rc = _load().oracle_mertens_table(L, out.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_mertens_table({L}) failed: {rc}")
    return out


def mertens_array(n: int, X: int, L: int = 0) -> np.ndarray:
    """The array M(floor(n/x)) for x = 1..X (int64), by the Sec. 2 recursion.

    ``L`` is the plain-table limit (raised to floor(sqrt(n)) if smaller)."""
    lo, hi = _split(n)
    out = np.zeros(X, dtype=np.int64)
    rc = _load().oracle_mertens_array(lo, hi, X, L, out.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_mertens_array(n={n}, X={X}, L={L}) failed: {rc}")
    return out


def mertens(n: int, L: int = 0) -> int:
    """M(n) alone."""
    return int(mertens_array(n, 1, L)[0])


def count_terms(n: int, u: int):
    """(direct, gathered) update-term counts by enumeration (small n only)."""
    d, g = ctypes.c_uint64(), ctypes.c_uint64()
    rc = _load().oracle_count_terms(n, u, ctypes.byref(d), ctypes.byref(g))
    if rc != 0:
        raise ValueError("oracle_count_terms failed")
    return int(d.value), int(g.value)


def window_sums(n: int, u: int, y1: int, length: int, x_first: int = 1, x_last: int = 0):
    """One y-window's carry-free share of the update (Sec. 2 split form):
    (S, coef, mu_sum) for entries x_first..x_last (default: all X = n//u),
    S and coef as uint64 arrays (mod 2^64).  The window's terms of entry x
    are S[x] + M(y1-1) coef[x]; mu_sum is the window's sum of mu."""
    lo, hi = _split(n)
    if x_last == 0:
        x_last = n // u
    cnt = x_last - x_first + 1
    S = np.zeros(max(cnt, 0), dtype=np.uint64)
    coef = np.zeros(max(cnt, 0), dtype=np.uint64)
    mus = ctypes.c_int64()
    rc = _load().oracle_window_sums(lo, hi, u, y1, length, x_first, x_last, S.ctypes.data,
                                    coef.ctypes.data, ctypes.byref(mus))
    if rc != 0:
        raise ValueError(f"oracle_window_sums(n={n}, u={u}, y1={y1}, len={length}) failed: {rc}")
    return S, coef, int(mus.value)
