"""CUDA path against the CPU oracle, element by element, bit-exact.

Every call goes through the C ABI (libmertens.so via its ctypes binding).
Small cases compare whole arrays; the full-size n = 10^16 configuration is
checked against Table 1 of the paper and on sampled entries the oracle
computes one by one.
"""
import functools
import math
import os

import numpy as np
import pytest

import oracle
import paper_1108_0135_gb300 as pm
from paper_1108_0135_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILE = 32768
BYTE_TILE = 131072


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pm.load()
    yield


def gpu_array(n, u=0, block_len=0):
    plan = pm.mertens_plan([n], u, block_len)
    try:
        pm.mertens_run(plan)
        m, arr = pm.mertens_result(plan, 0, entries=True)
    finally:
        pm.mertens_destroy(plan)
    return m, arr


# ---- a1, a2: the sieve ------------------------------------------------------

@pytest.mark.parametrize("y1,length", [
    (1, 3 * TILE + 1234),
    (10**6 + 3, 2 * TILE + 17),
    (10**9 - 5, TILE + 1),
    (10**12 + 12345, 2 * TILE + 999),
    (2**40 - 1000, TILE + 31),
    (999_983 * 999_983 - 300, 700),     # a prime square inside the window
    (1, 1), (2, 5), (7, 60),            # tiny windows
    # byte sieve: tiles below and above the 2^26 switch to one threshold per
    # tile, a ragged last tile, the top of its range (y < 2^42), and past it
    (2**26 - 3 * BYTE_TILE + 5, 6 * BYTE_TILE + 3),
    (2**41 + 12345, 2 * BYTE_TILE + 7),
    (2**42 - BYTE_TILE - 77, BYTE_TILE + 70),
    (2**42 + 5, 1000),
    # weight scale 3 above 2^42
    (10**13 + 12345, 2 * BYTE_TILE + 9),
    (2**47 + 999, BYTE_TILE + 5),
])
def test_sieve_mu_matches_oracle(y1, length):
    mu = torch.empty(length + 16, dtype=torch.int8, device="cuda")
    pm.mertens_sieve_mu(y1, length, mu)
    torch.cuda.synchronize()
    got = mu[:length].cpu().numpy()
    ref = oracle.mu_window(y1, length)
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, f"first mismatch at y={y1 + bad[0]}: {got[bad[0]]} vs {ref[bad[0]]}"


def test_sieve_M_from_one_matches_table():
    length = 5 * 10**6 + 7
    M = torch.empty(length, dtype=torch.int32, device="cuda")
    pm.mertens_sieve_M(1, length, 0, M)
    ref = oracle.mertens_table(length)[1:]
    assert np.array_equal(M.cpu().numpy(), ref)


def test_sieve_M_with_carry_far_from_one():
    y1, length = 10**9 + 7, 3 * TILE + 5
    carry = oracle.mertens(y1 - 1, L=10**6)
    M = torch.empty(length, dtype=torch.int32, device="cuda")
    pm.mertens_sieve_M(y1, length, carry, M)
    ref = carry + np.cumsum(oracle.mu_window(y1, length).astype(np.int64))
    assert np.array_equal(M.cpu().numpy().astype(np.int64), ref)


@pytest.mark.parametrize("y1,length", [
    (1, 3 * 10**6 + 11),
    (2**26 - 5 * 65536 + 77, 11 * 65536 + 3),    # per-y thresholds, then per tile
    (7 * 10**9 + 1, 4 * BYTE_TILE + 999),
    (4 * 10**10 - (1 << 24), 1 << 24),           # the top of the n = 10^16 sieve range
    (3 * 10**11 + 17, 300 * BYTE_TILE + 5),      # primes above 2^17: bucketed
    (2**45 + 3, 70 * BYTE_TILE + 1),             # weight scale 3, 5.9e6 sieving primes
])
def test_sieve_kernels_agree(y1, length, monkeypatch):
    """The default kernel (scale-2 bytes with 96 Ki-y tiles where it is exact),
    its 64 Ki-y variant, the persistent bucketed byte kernel, the per-tile
    scale-4/3 byte kernel and the 16-bit kernel (each forced by its switch)
    give the same M(y), and match the oracle's mu."""
    # the carry only shifts every M(y); far out it is left at 0
    carry = 0 if y1 == 1 or y1 > 10**12 else oracle.mertens(y1 - 1, L=10**7)
    out = []
    for env, val in ((None, None), ("MERTENS_T2_TILE", "64"), ("MERTENS_SIEVE_BUCKETS", "1"),
                     ("MERTENS_SIEVE_TILES", "1"), ("MERTENS_SIEVE16", "1")):
        if env:
            monkeypatch.setenv(env, val)
        M = torch.empty(length, dtype=torch.int32, device="cuda")
        pm.mertens_sieve_M(y1, length, carry, M)
        out.append(M.cpu().numpy())
        if env:
            monkeypatch.delenv(env)
    for i in range(1, len(out)):
        assert np.array_equal(out[0], out[i]), i
    ref = carry + np.cumsum(oracle.mu_window(y1, length).astype(np.int64))
    assert np.array_equal(out[0].astype(np.int64), ref)


def test_bounded_copy_wait_reports_timeout_and_device_stays_usable(monkeypatch):
    """The sieve's bulk-copy wait is bounded: with MERTENS_TEST_STALL_COPY the
    barrier is told to expect 16 bytes that never arrive, the wait gives up
    (about a second), the call reports MERTENS_ETIMEOUT, and the next call on
    the same device is correct."""
    y1, length = 2**30 + 1, BYTE_TILE + 100
    M = torch.empty(length, dtype=torch.int32, device="cuda")
    # the per-tile scale-4 byte kernel (forced) and the default scale-2 kernel
    # both load their tile's pattern by a bulk copy; the scale-4 one is tested
    monkeypatch.setenv("MERTENS_SIEVE_TILES", "1")
    monkeypatch.setenv("MERTENS_TEST_STALL_COPY", "1")
    with pytest.raises(pm.MertensError) as ei:
        pm.mertens_sieve_M(y1, length, 0, M)
    assert ei.value.code == pm._lib.MERTENS_ETIMEOUT
    monkeypatch.delenv("MERTENS_TEST_STALL_COPY")
    pm.mertens_sieve_M(y1, length, 0, M)
    ref = np.cumsum(oracle.mu_window(y1, length).astype(np.int64))
    assert np.array_equal(M.cpu().numpy().astype(np.int64), ref)


def test_sieve_rejects_bad_arguments():
    mu = torch.empty(64, dtype=torch.int8, device="cuda")
    with pytest.raises(pm.MertensError):
        pm.mertens_sieve_mu(0, 10, mu)
    with pytest.raises(pm.MertensError):
        pm.mertens_sieve_mu(1, 10, mu.data_ptr() + 1)   # not 16-byte aligned


# ---- a1..a4: whole arrays ---------------------------------------------------

def test_every_small_n_every_u():
    M = oracle.mertens_table(2000)
    for n in range(1, 121):
        us = [1] if n == 1 else range(math.isqrt(n) + 1, n + 1)
        for u in us:
            m, arr = gpu_array(n, u)
            X = n // u
            x = np.arange(1, X + 1)
            assert m == M[n]
            assert np.array_equal(arr, M[n // x].astype(np.int64)), (n, u)


def test_small_n_auto_parameters_and_tiny_blocks():
    M = oracle.mertens_table(20000)
    for n in list(range(1, 400, 7)) + [4096, 4097, 8191, 12288, 19999]:
        m, arr = gpu_array(n)
        assert m == M[n], n
        for bl in (1, 3, 64):
            if n <= 2000:
                m2, arr2 = gpu_array(n, 0, bl)
                assert m2 == M[n] and np.array_equal(arr, arr2), (n, bl)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_cases_against_recursion(seed):
    for n, u, bl in workloads.random_small_cases(seed, 25, 10**10):
        m, arr = gpu_array(n, u, bl)
        X = n // u
        ref = oracle.mertens_array(n, X, L=min(max(math.isqrt(n), 10**6), 10**7))
        assert np.array_equal(arr, ref), (n, u, bl)


def test_config_1e12_full_array():
    cfg = workloads.SINGLE_1E12
    n, u, L = cfg["n"][0], cfg["u"], cfg["block_len"]
    m, arr = gpu_array(n, u, L)
    ref = oracle.mertens_array(n, n // u, L=10**8)
    assert np.array_equal(arr, ref)


def test_1e9_same_code_path_vs_brute_force_table():
    n = 10**9
    m, arr = gpu_array(n, 4 * 10**6, 1 << 20)
    M = oracle.mertens_table(40_000_000)
    # entries x >= 25 have k <= 4e7: compare them with the plain table
    x = np.arange(25, len(arr) + 1)
    assert np.array_equal(arr[24:], M[n // x].astype(np.int64))
    assert m == oracle.mertens(n, L=10**7)


def test_sec1_extreme_ratio_value():
    n = 7766842813
    m, _ = gpu_array(n)
    assert abs(m) == 50286 and m == oracle.mertens(n, L=10**7)


def test_dense_cutoff_does_not_change_results():
    n, u = 10**11 + 7, 3 * 10**7
    ref = oracle.mertens_array(n, n // u, L=10**7)
    old = os.environ.get("MERTENS_DENSE_C")
    try:
        for c in ("1.0", "1.6", "3.0", "7.5"):
            os.environ["MERTENS_DENSE_C"] = c
            _, arr = gpu_array(n, u, 1 << 22)
            assert np.array_equal(arr, ref), c
    finally:
        if old is None:
            os.environ.pop("MERTENS_DENSE_C", None)
        else:
            os.environ["MERTENS_DENSE_C"] = old


@functools.lru_cache(maxsize=None)
def _oracle_array(n, X):
    return oracle.mertens_array(n, X, L=10**7)


@pytest.mark.parametrize("mode", ["0", "2", None])
@pytest.mark.parametrize("n,u,bl", [(10**11 + 7, 3 * 10**7, 1 << 22),
                                    (10**12 + 39, 10**8, 1 << 24)])
def test_gather_quotient_paths(n, u, bl, mode, monkeypatch):
    """The shared-memory gather takes a term's quotient floor(k/j) by the
    multiply-high magics (0), by a float estimate with a 64-bit remainder (2)
    or, by default here, with a 32-bit one: all give the oracle's array."""
    if mode is None:
        monkeypatch.delenv("MERTENS_GATHER_QUOT", raising=False)
    else:
        monkeypatch.setenv("MERTENS_GATHER_QUOT", mode)
    ref = _oracle_array(n, n // u)
    _, arr = gpu_array(n, u, bl)
    assert np.array_equal(arr, ref)


def _run_arrays(ns, u, bl):
    plan = pm.mertens_plan(ns, u, bl)
    try:
        pm.mertens_run(plan)
        out = [pm.mertens_result(plan, i, entries=True)[1] for i in range(len(ns))]
        st = pm.mertens_run_stats_get(plan)
    finally:
        pm.mertens_destroy(plan)
    return out, st


@pytest.mark.parametrize("ns,u,bl", [([10**12 + 39], 10**8, 1 << 24),
                                     ([10**13 + 1], 0, 0),
                                     ([10**12, 10**12 + 5 * 10**8 + 3, 7 * 10**11 + 1], 0, 1 << 24)])
def test_shared_even_terms_same_arrays(ns, u, bl, monkeypatch):
    """Entry 2x takes part of its gathered terms from entry x's even j
    (floor(floor(n/x)/2j) = floor(floor(n/2x)/j)); the arrays are the same
    with the sharing switched off (MERTENS_SHARE=0), and fewer terms are
    evaluated with it."""
    monkeypatch.setenv("MERTENS_SHARE", "0")
    off, st_off = _run_arrays(ns, u, bl)
    monkeypatch.delenv("MERTENS_SHARE")
    on, st_on = _run_arrays(ns, u, bl)
    for a, b in zip(off, on):
        assert np.array_equal(a, b)
    assert st_off["gather_j_exec"] == st_off["gather_j"] == st_on["gather_j"]
    assert st_on["gather_j_exec"] < 0.8 * st_on["gather_j"]
    if ns[0] == 10**12 + 39:
        assert np.array_equal(on[0], _oracle_array(ns[0], ns[0] // u))


def test_batch_same_alone_and_in_mix():
    ns = [10**12 + i * 10**6 + (i * 7919) % 1000 for i in range(8)] + [10**9 + 1, 12345]
    plan = pm.mertens_plan(ns)
    try:
        pm.mertens_run(plan)
        mixed = [pm.mertens_result(plan, i, entries=True) for i in range(len(ns))]
        infos = [pm.mertens_plan_info(plan, i) for i in range(len(ns))]
    finally:
        pm.mertens_destroy(plan)
    for n, (m, arr), info in zip(ns, mixed, infos):
        m1, arr1 = gpu_array(n, info["u"])
        assert m == m1 and np.array_equal(arr, arr1), n
    for i in (0, 7, 8, 9):
        n = ns[i]
        ref = oracle.mertens_array(n, infos[i]["X"], L=10**8 if n > 10**10 else 0)
        assert np.array_equal(mixed[i][1], ref), n


def test_run_twice_same_plan():
    plan = pm.mertens_plan([10**11])
    try:
        pm.mertens_run(plan)
        a = pm.mertens_result(plan, 0, entries=True)
        pm.mertens_run(plan)
        b = pm.mertens_result(plan, 0, entries=True)
    finally:
        pm.mertens_destroy(plan)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_result_before_run_is_not_ready():
    plan = pm.mertens_plan([1000])
    try:
        with pytest.raises(pm.MertensError) as ei:
            pm.mertens_result(plan, 0)
        assert ei.value.code == pm.MERTENS_ENOTREADY
        with pytest.raises(pm.MertensError):
            pm.mertens_result(plan, 1)
    finally:
        pm.mertens_destroy(plan)


def test_autotune_picks_parameters_that_keep_results():
    n = 10**12 + 3
    best, ms = pm.mertens_autotune([n], runs=1)
    assert ms > 0 and best["u_factor"] > 0 and best["dense_c"] > 0
    old = pm.mertens_get_tuning()
    try:
        ref = gpu_array(n)
        pm.mertens_set_tuning(**best)
        got = gpu_array(n)
        X = len(got[1])
        assert got[0] == ref[0] == oracle.mertens(n, L=10**8)
        assert np.array_equal(got[1], oracle.mertens_array(n, X, L=10**8))
    finally:
        pm.mertens_set_tuning(**old)


# ---- Table 1 values beyond 10^16 ----------------------------------------------

def test_table1_1e18_auto_parameters(table1):
    m, arr = gpu_array(10**18)
    assert m == table1[10**18] == -46758740
    # the array's last entry, k = floor(n/X) ~ 1.1e12, by the oracle recursion
    k = 10**18 // len(arr)
    assert arr[-1] == oracle.mertens(k, L=2 * 10**7)


def test_batch_of_close_targets_1e17(table1):
    # Sec. 2: close values share one sieve pass; n_0 = 10^17 is in Table 1
    ns = [10**17 + i * 10**9 for i in range(8)]
    plan = pm.mertens_plan(ns)
    try:
        pm.mertens_run(plan)
        res = [pm.mertens_result(plan, i, entries=True) for i in range(len(ns))]
        infos = [pm.mertens_plan_info(plan, i) for i in range(len(ns))]
    finally:
        pm.mertens_destroy(plan)
    assert res[0][0] == table1[10**17] == -21830254
    # the same target alone, with the batch's u, gives the same array
    for i in (0, 5):
        m1, arr1 = gpu_array(ns[i], infos[i]["u"])
        assert res[i][0] == m1 and np.array_equal(res[i][1], arr1)
    # the last entry (smallest k ~ 8e11) of two more targets by the oracle
    for i in (3, 7):
        X = len(res[i][1])
        assert res[i][1][X - 1] == oracle.mertens(ns[i] // X, L=10**8), i


@pytest.fixture(scope="module")
def batch_1e17():
    """The 64-target batch n_i = 10^17 + i 10^9 in one plan (one sieve pass),
    with the automatic batch u: every target's whole array and plan info."""
    cfg = workloads.BATCH_1E17
    ns = cfg["n"]
    plan = pm.mertens_plan(ns, cfg["u"], 0)
    try:
        pm.mertens_run(plan)
        res = [pm.mertens_result(plan, i, entries=True) for i in range(len(ns))]
        infos = [pm.mertens_plan_info(plan, i) for i in range(len(ns))]
    finally:
        pm.mertens_destroy(plan)
    return ns, res, infos


def test_batch_1e17_full_size_table1(batch_1e17, table1):
    ns, res, infos = batch_1e17
    assert len(ns) == 64 and ns[0] == 10**17
    assert res[0][0] == table1[10**17] == -21830254
    # one u for the whole batch (Sec. 2: close targets share the sieve)
    assert len({i["u"] for i in infos}) == 1


@pytest.mark.parametrize("part", range(4))
def test_batch_1e17_full_size_alone_equals_batched(batch_1e17, part):
    """Each of the 64 targets alone, with the batch's u, gives the same whole
    array as in the batch (16 targets per part)."""
    ns, res, infos = batch_1e17
    for i in range(16 * part, 16 * part + 16):
        m1, arr1 = gpu_array(ns[i], infos[i]["u"])
        assert res[i][0] == m1, i
        assert np.array_equal(res[i][1], arr1), i


@pytest.mark.parametrize("i", [1, 63])
def test_batch_1e17_full_size_entries_against_oracle(batch_1e17, i):
    """Targets 1 and 63: M(n_i) by Table 1's neighbour is not printed, so the
    entries with the smallest k (k = floor(n/x) near the batch's u, a few
    10^12: the oracle's Sec. 2 recursion at about a second each) are compared
    one by one: the last two and six seeded ones from the last quarter."""
    ns, res, _ = batch_1e17
    n, arr = ns[i], res[i][1]
    X = len(arr)
    rng = np.random.default_rng(1000 + i)
    xs = [X, X - 1] + [int(v) for v in rng.integers(X - X // 4, X, size=6)]
    for x in xs:
        assert arr[x - 1] == oracle.mertens(n // x, L=10**8), (i, x)


# ---- two-word entries (k >= 2^63) ----------------------------------------------
# MERTENS_WIDE_FROM moves the bound above which an entry takes the two-word
# kernel, so that kernel can be compared with the oracle where the oracle is
# cheap: first on every entry (k >= 2) of small targets, then on the first
# entries of n ~ 10^12.

def test_two_word_kernel_on_every_entry_small_n(monkeypatch):
    monkeypatch.setenv("MERTENS_WIDE_FROM", "2")
    M = oracle.mertens_table(2000)
    for n in range(1, 121, 2):
        us = [1] if n == 1 else range(math.isqrt(n) + 1, n + 1)
        for u in us:
            m, arr = gpu_array(n, u)
            x = np.arange(1, n // u + 1)
            assert m == M[n]
            assert np.array_equal(arr, M[n // x].astype(np.int64)), (n, u)
        m, arr = gpu_array(n, 0, 3)   # blocks of 3 y
        assert m == M[n], n


@pytest.mark.parametrize("n,u,bl,wide_from", [
    (10**12 + 12345, 10**8, 2**24, 10**11),      # x <= 10 two-word
    (10**12 - 1, 3 * 10**7, 2**20, 2 * 10**9),   # x <= 499, short blocks
    (999_999_999_989, 0, 0, 10**6),              # every entry but the last ones
])
def test_two_word_kernel_matches_oracle(n, u, bl, wide_from, monkeypatch):
    ref_m, ref_arr = gpu_array(n, u, bl)
    monkeypatch.setenv("MERTENS_WIDE_FROM", str(wide_from))
    m, arr = gpu_array(n, u, bl)
    assert m == ref_m and np.array_equal(arr, ref_arr)
    assert np.array_equal(arr, oracle.mertens_array(n, len(arr), L=10**8))


def test_two_word_target_1e20(table1):
    """Sec. 5 Table 1: M(10^20); entries x <= 10 take the two-word kernel and
    the sieve runs to ~10^13 (byte sieve at weight scale 3)."""
    n = 10**20
    m, arr = gpu_array(n)
    assert m == table1[n] == 461113106
    X = len(arr)
    assert arr[X - 1] == oracle.mertens(n // X, L=2 * 10**7)
    # Sec. 5: one large run also yields the smaller Table 1 values as array
    # entries, M(floor(n/x)): x = 10 (a two-word entry), 100, 1000, 10^4
    for x in (10, 100, 1000, 10**4):
        assert arr[x - 1] == table1[n // x], x


@pytest.mark.parametrize("n", [11609864264058592345, 10**19])
def test_two_word_targets_paper_values(n, table1):
    """Sec. 5 Table 1 and Sec. 6: M(10^19) and the new extreme value, both
    above 2^63 (entry x = 1 takes the two-word kernel)."""
    m, arr = gpu_array(n)
    assert m == table1[n]
    # Sec. 5's self-consistency: entries x = 10, 100, 1000 of the 10^19 run
    # are M(10^18), M(10^17), M(10^16) of Table 1
    if n == 10**19:
        for x in (10, 100, 1000):
            assert arr[x - 1] == table1[n // x], x
    # the entries with the smallest k, by the oracle recursion
    X = len(arr)
    for x in (X, X - 1, X - 1000):
        assert arr[x - 1] == oracle.mertens(n // x, L=2 * 10**7), x
    # entry x = 2 (k = floor(n/2) < 2^63) equals a separate one-word run
    m2, _ = gpu_array(n // 2)
    assert arr[1] == m2


# ---- windows: contributions affine in the window's carry ------------------------

def _resolve_host(n, S):
    """M[x] = 1 - S[x] - sum_{j>=2} M[xj] (mod 2^64), x = X..1, read as int64."""
    X = len(S)
    R = [0] * (X + 1)
    for x in range(X, 0, -1):
        if n // x == 1:
            R[x] = 1
            continue
        acc = sum(R[x * j] for j in range(2, X // x + 1))
        R[x] = (1 - int(S[x - 1]) - acc) % 2**64
    return np.array(R[1:], dtype=np.uint64).view(np.int64)


def _windows_sum(n, u, cuts, block_lens):
    """S of a whole run assembled from windows [cuts[i], cuts[i+1]-1], each
    S_loc + C coef with C = M(window start - 1) chained from the mu sums."""
    total = None
    carry = 0
    for (a, b), bl in zip(zip(cuts[:-1], cuts[1:]), block_lens):
        plan = pm.mertens_plan_window([n], a, b - 1, u, bl)
        try:
            pm.mertens_run(plan)
            S, coef, mu = pm.mertens_window_result(plan, 0)
        finally:
            pm.mertens_destroy(plan)
        part = S + np.uint64(carry % 2**64) * coef   # wraps mod 2^64
        total = part if total is None else total + part
        carry += mu
    return total


@pytest.mark.parametrize("wide_from", [None, 10**11])
def test_windows_partition_equals_whole_run(wide_from, monkeypatch):
    if wide_from:
        monkeypatch.setenv("MERTENS_WIDE_FROM", str(wide_from))
    n, u = 10**12 + 12345, 10**8
    m, arr = gpu_array(n, u, 2**22)
    ymax = pm.mertens_describe(n, u)["y_max"]
    # the first cut splits the dense part (y_c ~ 1.6 sqrt(k) <= 1.6e6)
    cuts = [1, 700_001, 5_000_001, ymax + 1]
    S = _windows_sum(n, u, cuts, [2**18, 2**20 + 3, 0])
    got = _resolve_host(n, S)
    assert np.array_equal(got, arr)
    assert np.array_equal(got, oracle.mertens_array(n, n // u, L=10**8))


@pytest.mark.parametrize("wide_from", [None, 10**11])
def test_window_accumulate_and_resolve_on_device(wide_from, monkeypatch):
    """The device exchange: windows of a partition, each added into one
    exchange buffer by mertens_window_accumulate with the mu sums of the
    windows below it (the carry), resolve from the buffer on the device --
    the same array as a whole run and as the oracle."""
    if wide_from:
        monkeypatch.setenv("MERTENS_WIDE_FROM", str(wide_from))
    n, u = 10**12 + 12345, 10**8
    m, arr = gpu_array(n, u, 2**22)
    ymax = pm.mertens_describe(n, u)["y_max"]
    cuts = [1, 700_001, 5_000_001, ymax + 1]
    X = n // u
    buf = torch.zeros(2 * X, dtype=torch.int64, device="cuda")
    mus = []
    # windows added in reverse order: the sum does not depend on it
    plans = []
    try:
        for (a, b), bl in zip(zip(cuts[:-1], cuts[1:]), [2**18, 2**20 + 3, 0]):
            plans.append(pm.mertens_plan_window([n], a, b - 1, u, bl))
            pm.mertens_run(plans[-1])
            mus.append(pm.mertens_window_mu_sum(plans[-1], 0))
        for g in reversed(range(len(plans))):
            pm.mertens_window_accumulate(plans[g], 0, mus[:g], buf)
    finally:
        for p in plans:
            pm.mertens_destroy(p)
    M = torch.empty(X, dtype=torch.int64, device="cuda")
    pm.mertens_resolve_exchange(n, u, buf, M)
    got = M.cpu().numpy()
    assert np.array_equal(got, arr)
    assert np.array_equal(got, oracle.mertens_array(n, X, L=10**8))


def test_sharded_target_one_rank_equals_whole_run():
    """shard.ShardedTarget with one rank: the window [1, y_max] through a
    window plan, then mertens_resolve on its sums, equals a whole run."""
    from paper_1108_0135_gb300 import shard
    n, u = 10**12 + 12345, 10**8
    m, arr = gpu_array(n, u, 2**22)
    t = shard.ShardedTarget(n, u, 2**22)
    try:
        got = t.step()
        got2 = t.step()
    finally:
        t.close()
    assert np.array_equal(got, arr) and np.array_equal(got2, arr)


def test_window_two_word_target_at_1e13():
    """n = 10^20 with u ~ n^(2/3): four 2^22-y blocks from y = 10^13, against
    carry-free sums from the oracle's mu window (entries x <= 10 are two-word)."""
    n, u = 10**20, 21544346900318
    y1, L = 10**13, 4 * 2**22
    y2 = y1 + L - 1
    plan = pm.mertens_plan_window([n], y1, y2, u, 2**22)
    try:
        pm.mertens_run(plan)
        S, coef, mu = pm.mertens_window_result(plan, 0)
    finally:
        pm.mertens_destroy(plan)
    Mloc = np.cumsum(oracle.mu_window(y1, L).astype(np.int64))
    assert mu == int(Mloc[-1])
    X = n // u
    assert len(S) == X
    want_S, want_c = {}, {}
    for x in range(1, X + 1):
        k = n // x
        ja = max(X // x + 1, k // (y2 + 1) + 1)
        jb = k // y1                          # below the dense cut-off and sqrt(k)
        if jb < ja:
            continue
        want_c[x] = jb - ja + 1
        want_S[x] = sum(int(Mloc[k // j - y1]) for j in range(ja, jb + 1)) % 2**64
    got_c = {int(i) + 1: int(v) for i, v in enumerate(coef) if v}
    got_S = {int(i) + 1: int(v) for i, v in enumerate(S) if v}
    assert got_c == want_c
    assert got_S == {x: v for x, v in want_S.items() if v}


def _window_plan_sums(n, u, y1, length, block_len):
    plan = pm.mertens_plan_window([n], y1, y1 + length - 1, u, block_len)
    try:
        pm.mertens_run(plan)
        return pm.mertens_window_result(plan, 0)
    finally:
        pm.mertens_destroy(plan)


def test_window_two_word_full_block_at_1e13_against_oracle():
    """One whole 2^28-y block of the n = 10^20 window (u = 2.15e13, from
    y = 10^13): every entry's carry-free sum and coefficient equal the
    oracle's 128-bit window sums (entries x <= 10 are two-word)."""
    cfg = workloads.WINDOW_1E20
    n, u, y1, L = cfg["n"][0], cfg["u"], cfg["y_first"], cfg["block_len"]
    S, coef, mu = _window_plan_sums(n, u, y1, L, L)
    oS, oc, omu = oracle.window_sums(n, u, y1, L)
    assert mu == omu
    assert len(S) == len(oS) == n // u
    assert np.array_equal(coef, oc)
    assert np.array_equal(S, oS)
    assert int(np.count_nonzero(oc[:10])) > 0      # two-word entries have terms here


def test_window_two_word_direct_terms_against_oracle():
    """A 2^20-y window at y = 3e9 of n = 10^20: entries x <= 11 have
    s = floor(sqrt(k)) above it, so it holds only their direct terms
    M(y)(floor(k/y) - floor(k/(y+1))) -- with 128-bit quotients for x <= 10 --
    and gathered terms of the entries x >= 129.  Compared with the oracle's
    window sums.  Entries 11..128 are left out: their dense cut-off
    (about 1.4 sqrt(k), shared by groups of 32 entries) lies at or above the
    window, where the update takes the mu-form of the same terms, whose
    carry-free part differs by a boundary term."""
    n, u = 10**20, workloads.WINDOW_1E20["u"]
    y1, L = 3 * 10**9, 2**20
    S, coef, mu = _window_plan_sums(n, u, y1, L, L)
    oS, oc, omu = oracle.window_sums(n, u, y1, L)
    assert mu == omu
    x = np.arange(1, n // u + 1)
    keep = (x <= 10) | (x >= 129)
    assert np.array_equal(coef[keep], oc[keep])
    assert np.array_equal(S[keep], oS[keep])
    assert all(int(oc[i]) > L for i in range(10))   # direct coefficients of the two-word entries


# ---- interval scan: extremes of M(y) and M(y)/sqrt(y) ---------------------------

def _extremes_host(y1, M):
    """Exact extremes of M(y) and M(y)/sqrt(y), y = y1 + i (ties: smallest y)."""
    ys = np.arange(y1, y1 + len(M), dtype=np.int64)
    out = {"M_max": int(M.max()), "y_M_max": int(ys[np.argmax(M)]),
           "M_min": int(M.min()), "y_M_min": int(ys[np.argmin(M)])}
    R = M / np.sqrt(ys.astype(np.float64))
    for key, best in (("max", np.max(R)), ("min", np.min(R))):
        cand = np.nonzero(np.abs(R - best) <= 1e-9 * max(1.0, abs(best)))[0]
        pick = None
        for i in cand:
            m, y = int(M[i]), int(ys[i])
            if pick is None:
                pick = (m, y)
                continue
            pm_, py = pick
            # exact: m/sqrt(y) vs pm_/sqrt(py), by signs and squares
            a = (m > 0) - (m < 0)
            b = (pm_ > 0) - (pm_ < 0)
            if a != b:
                better = a > b if key == "max" else a < b
            else:
                l, r = m * m * py, pm_ * pm_ * y
                gt = l > r if a >= 0 else l < r       # m/sqrt(y) > pm_/sqrt(py)
                lt = l < r if a >= 0 else l > r
                better = gt if key == "max" else lt
                if l == r:
                    better = y < py
            if better:
                pick = (m, y)
        out["R_%s_M" % key], out["y_R_%s" % key] = pick
    return out


@pytest.mark.parametrize("y1,length", [(1, 2_000_000), (10**9 + 7, 3 * 10**6 + 11)])
def test_scan_extremes_against_oracle(y1, length):
    carry = 0 if y1 == 1 else oracle.mertens(y1 - 1, L=10**6)
    M = carry + np.cumsum(oracle.mu_window(y1, length).astype(np.int64))
    got = pm.mertens_scan_extremes(y1, y1 + length - 1, carry)
    want = _extremes_host(y1, M)
    assert got["M_last"] == int(M[-1])
    for k, v in want.items():
        assert got[k] == v, k


def test_scan_finds_the_sec1_extreme():
    """Sec. 1: |M(n)|/sqrt(n) = 0.570591 at n = 7766842813 (the largest
    value known before the paper): the scan of 10^6 y either side finds it."""
    n = 7766842813
    a, b = n - 10**6, n + 10**6
    got = pm.mertens_scan_extremes(a, b, oracle.mertens(a - 1, L=10**6))
    ratio, y = max((abs(got["R_max"]), got["y_R_max"]), (abs(got["R_min"]), got["y_R_min"]))
    assert y == n and round(ratio, 6) == 0.570591


def test_scan_over_blocks_is_consistent():
    """Ten sieve blocks of 2^30 y from y = 1: M_last is M(10^10) (oracle), and
    two halves, the second from the first one's M_last, give the same
    extremes as the whole."""
    y2 = 10**10
    whole = pm.mertens_scan_extremes(1, y2, 0)
    assert whole["M_last"] == oracle.mertens(y2, L=10**7)
    cut = 3 * 2**30 + 12345
    h1 = pm.mertens_scan_extremes(1, cut, 0)
    h2 = pm.mertens_scan_extremes(cut + 1, y2, h1["M_last"])
    assert h2["M_last"] == whole["M_last"]
    assert whole["M_max"] == max(h1["M_max"], h2["M_max"])
    assert whole["M_min"] == min(h1["M_min"], h2["M_min"])
    best = max((h1["R_max"], h1["y_R_max"]), (h2["R_max"], h2["y_R_max"]))
    assert whole["y_R_max"] == best[1]
    worst = min((h1["R_min"], h1["y_R_min"]), (h2["R_min"], h2["y_R_min"]))
    assert whole["y_R_min"] == worst[1]


# ---- resident M(y) table -------------------------------------------------------

@pytest.fixture(scope="module")
def table_2e26():
    t = pm.mertens_table_create(2**26 + 12345, 10**13)
    yield t
    pm.mertens_table_destroy(t)


def _run_on_table(table, ns, u=0, block_len=0):
    plan = pm.mertens_plan_on_table(table, ns, u, block_len)
    try:
        pm.mertens_run(plan)
        res = [pm.mertens_result(plan, i, entries=True) for i in range(len(ns))]
    finally:
        pm.mertens_destroy(plan)
    return res


def test_table_lookups_are_the_sieve(table_2e26):
    """Targets n <= y_max are read from the table: M(n) by the plain table."""
    info = pm.mertens_table_info(table_2e26)
    assert info["y_max"] == 2**26 + 12345 and info["n_max"] == 10**13
    ns = [1, 2, 1000, 10**6 + 3, 2**26, 2**26 + 12345]
    M = oracle.mertens_table(2**26 + 12345)
    for n, (m, arr) in zip(ns, _run_on_table(table_2e26, ns)):
        assert m == M[n] and len(arr) == 1, n


@pytest.mark.parametrize("n,block_len", [
    (10**12, 0), (10**12 + 12345, 2**22), (7 * 10**12 + 1, 2**20 + 2048), (2**26 + 12346, 0),
    (10**13, 0), (10**13 - 77, 2**22),
])
def test_plans_on_table_match_oracle(table_2e26, n, block_len):
    """u is at least what the table reaches (min(n, y_max + 1)); where the
    automatic u is larger (10^13: about 2.1e8 against 2^26 + 12346) the blocks
    above the table are sieved and the carry into the first of them is the
    table's M(y)."""
    plan = pm.mertens_plan_on_table(table_2e26, [n], 0, block_len)
    try:
        u = pm.mertens_plan_info(plan, 0)["u"]
        pm.mertens_run(plan)
        m, arr = pm.mertens_result(plan, 0, entries=True)
    finally:
        pm.mertens_destroy(plan)
    assert u >= min(n, 2**26 + 12346)
    assert len(arr) == n // u
    assert np.array_equal(arr, oracle.mertens_array(n, n // u, L=10**8))
    # and a sieving plan with the same u agrees
    m2, arr2 = gpu_array(n, u)
    assert m == m2 and np.array_equal(arr, arr2)


def test_two_word_entries_on_table(table_2e26, monkeypatch):
    """Entries forced through the two-word kernel read M(y) from the table."""
    n = 10**12 + 12345
    (m, arr), = _run_on_table(table_2e26, [n])
    monkeypatch.setenv("MERTENS_WIDE_FROM", str(10**9))
    (m2, arr2), = _run_on_table(table_2e26, [n])
    assert m2 == m and np.array_equal(arr2, arr)
    assert m == oracle.mertens(n, L=10**8)


def test_batch_on_table_same_as_alone(table_2e26):
    """Each target of a batch on the table, alone on the table with the
    batch's u for it, gives the same whole array."""
    ns = [10**12 + 7, 3 * 10**11, 5 * 10**7, 10**13, 123_456_789_012]
    plan = pm.mertens_plan_on_table(table_2e26, ns)
    try:
        us = [pm.mertens_plan_info(plan, i)["u"] for i in range(len(ns))]
        pm.mertens_run(plan)
        batch = [pm.mertens_result(plan, i, entries=True) for i in range(len(ns))]
    finally:
        pm.mertens_destroy(plan)
    for n, u, (m, arr) in zip(ns, us, batch):
        (m1, arr1), = _run_on_table(table_2e26, [n], u)
        assert m == m1 and np.array_equal(arr, arr1), n


def test_table_refuses_what_it_cannot_serve(table_2e26):
    with pytest.raises(pm.MertensError) as ei:
        pm.mertens_plan_on_table(table_2e26, [10**13 + 1])      # above n_max
    assert ei.value.code == pm.MERTENS_ENOTSUP
    small = pm.mertens_table_create(10**5, 10**12)
    try:
        with pytest.raises(pm.MertensError):
            pm.mertens_plan_on_table(small, [10**9], 0, 1000)   # block not a multiple of 2048
        (m, _), = _run_on_table(small, [10**9])
        assert m == oracle.mertens(10**9, L=10**6)
        # the dense cut-offs of 10^12 (about 1.4e6) lie beyond the table's
        # squarefree list (y <= 10^5)
        with pytest.raises(pm.MertensError) as ei:
            pm.mertens_plan_on_table(small, [10**12])
        assert ei.value.code == pm.MERTENS_ENOTSUP
    finally:
        pm.mertens_table_destroy(small)


# ---- full size: n = 10^16, u = 4e10, block 2^28 ------------------------------

def test_table1_1e16_full_configuration(table1):
    cfg = workloads.SINGLE_1E16
    n, u, L = cfg["n"][0], cfg["u"], cfg["block_len"]
    m, arr = gpu_array(n, u, L)
    assert m == table1[10**16] == -3195437
    # sampled entries: k = floor(n/x) <= 1e11, each by the oracle recursion
    rng = np.random.default_rng(16)
    for x in sorted(rng.integers(100_000, len(arr) + 1, size=6)) + [len(arr)]:
        k = n // int(x)
        assert arr[int(x) - 1] == oracle.mertens(k, L=10**7), x
