"""The C-ABI library without a GPU: it builds, loads, exports every symbol
include/libmertens.h declares, and its host-only planning calls agree with
the oracle's enumeration."""
import ctypes
import math
import os
import re

import pytest

import oracle
import paper_1108_0135_gb300 as pm
from tests.conftest import ROOT


def header_functions():
    text = open(os.path.join(ROOT, "include", "libmertens.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(mertens_[A-Za-z_0-9]+)\s*\(",
                           text, flags=re.M))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = pm.load()
    declared = header_functions()
    assert len(declared) >= 13
    assert set(declared) == set(pm.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_strerror_covers_codes():
    for code in range(8):
        assert pm.mertens_strerror(code) != "unknown status"
    assert pm.mertens_strerror(99) == "unknown status"


@pytest.mark.parametrize("n", [2, 3, 10, 97, 100, 399])
def test_describe_term_counts_match_enumeration(n):
    s = math.isqrt(n)
    for u in range(s + 1, n + 1):
        info = pm.mertens_describe(n, u)
        assert info["X"] == n // u
        assert (info["direct_terms"], info["gathered_terms"]) == oracle.count_terms(n, u)


def test_describe_full_size_counts():
    info = pm.mertens_describe(10**16, 4 * 10**10)
    assert info["X"] == 250_000
    total = info["direct_terms"] + info["gathered_terms"]
    assert 1.99e11 < total < 2.0e11
    info = pm.mertens_describe(10**12, 10**8)
    assert info["X"] == 10_000 and info["y_max"] == 10**12 // 10_001


@pytest.mark.parametrize("n,u,code", [
    (0, 0, pm.MERTENS_EINVAL),
    (100, 10, pm.MERTENS_EINVAL),       # u must exceed floor(sqrt(n))
    (100, 101, pm.MERTENS_EINVAL),      # u must not exceed n
    (2**127, 0, pm.MERTENS_EINVAL),     # n must be below 2^127
    (2**80, 2**41, pm.MERTENS_ENOTSUP), # 2^39 array entries
])
def test_invalid_arguments_rejected_without_gpu(n, u, code):
    with pytest.raises(pm.MertensError) as ei:
        pm.mertens_describe(n, u)
    assert ei.value.code == code
    with pytest.raises(pm.MertensError) as ei:
        pm.mertens_plan([n], u)
    assert ei.value.code == code


@pytest.mark.parametrize("n,u", [
    (2**63, 2**63 // 5),
    (2**64 + 12345, (2**64 + 12345) // 7),
    (10**20, 10**20 // 1000),
    (11609864264058592345, 11609864264058592345 // 3000),
])
def test_describe_two_word_targets(n, u):
    """Closed-form term counts for targets at and above 2^63, recomputed here
    with Python integers (k = n // x, s = isqrt(k))."""
    info = pm.mertens_describe(n, u)
    X = n // u
    assert info["n"] == n and info["X"] == X
    d = g = 0
    for x in range(1, X + 1):
        k = n // x
        s = math.isqrt(k)
        d += s
        g += max(0, k // (s + 1) - (X // x + 1) + 1)
    assert (info["direct_terms"], info["gathered_terms"]) == (d, g)
    assert info["y_max"] == max(math.isqrt(n), n // (X + 1))


def test_server_without_usable_device_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pm.MertensError) as ei:
        pm.mertens_server_create(0)
    assert ei.value.code in (pm._lib.MERTENS_ECUDA, pm.MERTENS_EINVAL)


def test_tuning_validation_and_effect_on_auto_u():
    old = pm.mertens_get_tuning()
    try:
        with pytest.raises(pm.MertensError):
            pm.mertens_set_tuning(u_factor=0.0)
        with pytest.raises(pm.MertensError):
            pm.mertens_set_tuning(block_cap=1000)
        pm.mertens_set_tuning(u_factor=0.5)
        u5 = pm.mertens_describe(10**15)["u"]
        pm.mertens_set_tuning(u_factor=1.0)
        u10 = pm.mertens_describe(10**15)["u"]
        assert abs(u10 / u5 - 2.0) < 1e-6
        assert pm.mertens_describe(10**15, 10**10)["u"] == 10**10   # explicit u wins
    finally:
        pm.mertens_set_tuning(**old)


def test_plan_rejects_empty_batch():
    lib = pm.load()
    h = ctypes.c_void_p()
    rc = lib.mertens_plan(ctypes.byref(h), None, 0, pm._lib.u128(0), 0)
    assert rc == pm.MERTENS_EINVAL and not h.value


def header_structs():
    """{typedef name: [(C type, field name), ...]} of the header's structs."""
    text = open(os.path.join(ROOT, "include", "libmertens.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*([a-z_0-9]+)\s*;", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            ctype, rest = decl.split(None, 1)
            fields += [(ctype, f.strip()) for f in rest.split(",")]
        out[name] = fields
    return out


def test_ctypes_structs_match_the_header():
    """Every struct the binding passes by pointer has the header's fields, in
    its order and with its C types (a mismatch would shift every later
    field)."""
    cmap = {"uint64_t": ctypes.c_uint64, "int64_t": ctypes.c_int64, "uint32_t": ctypes.c_uint32,
            "int32_t": ctypes.c_int32, "int": ctypes.c_int, "double": ctypes.c_double,
            "mertens_u128": pm._lib.mertens_u128}
    structs = header_structs()
    checked = 0
    for name, fields in structs.items():
        cls = getattr(pm._lib, name, None)
        if cls is None:
            continue
        got = [(f, t) for f, t in cls._fields_]
        want = [(f, cmap[t]) for t, f in fields]
        assert got == want, name
        checked += 1
    assert checked >= 6
