"""Pins for the CPU oracle (no GPU).

The oracle is the yardstick for the CUDA path, so it is checked here against
facts that do not come from its own code: a library Moebius function, closed
forms, the identity that the paper's recursion starts from (Sec. 2), brute
force on small inputs and the value implied by the ratio quoted in Sec. 1.
"""
import math

import numpy as np
import pytest

import oracle
from tests.conftest import read_golden

sympy = pytest.importorskip("sympy")


def test_mu_trial_matches_library_mobius():
    # sympy's mobius factors independently of the oracle's trial division.
    for m in range(1, 3001):
        assert oracle.mu_trial(m) == int(sympy.mobius(m)), m


def test_mu_window_matches_trial_division_from_one():
    mu = oracle.mu_window(1, 100_000)
    ref = np.array([oracle.mu_trial(m) for m in range(1, 100_001)], dtype=np.int8)
    assert np.array_equal(mu, ref)


@pytest.mark.parametrize("y1,length", [(10**9 - 17, 400), (10**12 + 12345, 150),
                                       (2**40 - 75, 150), (999_983 * 999_983 - 60, 121)])
def test_mu_window_far_from_one_matches_library(y1, length):
    mu = oracle.mu_window(y1, length)
    ref = np.array([int(sympy.mobius(y)) for y in range(y1, y1 + length)], dtype=np.int8)
    assert np.array_equal(mu, ref)


def test_mu_closed_forms():
    primes = list(sympy.primerange(2, 20_000))
    mu = oracle.mu_window(1, 20_000**2 // 100)
    lim = len(mu)
    for p in primes:
        assert mu[p - 1] == -1, p                      # mu(p) = -1
        if p * p <= lim:
            assert mu[p * p - 1] == 0, p               # mu(p^2) = 0
    for p, q in [(2, 3), (3, 5), (101, 103), (1999, 1997)]:
        assert mu[p * q - 1] == 1                      # two distinct primes
    for p, q, r in [(2, 3, 5), (7, 11, 13), (97, 89, 83)]:
        assert mu[p * q * r - 1] == -1                 # three distinct primes


def test_identity_sum_of_M_floor_is_one():
    # Sec. 2: sum_{x=1}^{n} M(floor(n/x)) = 1, for every n up to 10^4.
    M = oracle.mertens_table(10_000)
    for n in range(1, 10_001):
        x = np.arange(1, n + 1)
        assert int(M[n // x].astype(np.int64).sum()) == 1, n


def test_table_prefix_of_mu():
    M = oracle.mertens_table(50_000)
    mu = oracle.mu_window(1, 50_000)
    assert M[0] == 0
    assert np.array_equal(np.diff(M.astype(np.int64)), mu.astype(np.int64))


def test_recursion_matches_table_every_small_n():
    # The recursion at the smallest table size L = floor(sqrt(n)) recurses
    # through every distinct quotient above sqrt(n).
    M = oracle.mertens_table(20_000)
    for n in range(1, 20_001):
        assert oracle.mertens(n, L=math.isqrt(n)) == M[n], n


def test_recursion_full_array_matches_table():
    M = oracle.mertens_table(3000)
    for n in range(1, 3001, 7):
        arr = oracle.mertens_array(n, n, L=math.isqrt(n))
        x = np.arange(1, n + 1)
        assert np.array_equal(arr, M[n // x].astype(np.int64)), n


def test_recursion_sampled_n_up_to_2e7():
    M = oracle.mertens_table(20_000_000)
    rng = np.random.default_rng(7)
    for n in rng.integers(20_000, 20_000_000, size=40):
        n = int(n)
        X = max(1, n // (math.isqrt(n) * 3))
        arr = oracle.mertens_array(n, X, L=math.isqrt(n) + int(rng.integers(0, 500)))
        x = np.arange(1, X + 1)
        assert np.array_equal(arr, M[n // x].astype(np.int64)), n


def test_sec1_ratio_value():
    # Sec. 1 quotes |M(n)/sqrt(n)| = 0.570591 at n = 7766842813.
    (n, ratio), = read_golden("sec1_ratio.txt")
    m = oracle.mertens(n, L=10**8)
    assert round(abs(m) / math.sqrt(n), 6) == ratio
    assert abs(m) == 50286


def test_independent_of_table_size():
    n = 10**11 + 3
    ref = oracle.mertens_array(n, 50, L=math.isqrt(n))
    for L in (math.isqrt(n) + 1, 10**6, 3 * 10**6):
        assert np.array_equal(oracle.mertens_array(n, 50, L=L), ref)


def test_count_terms_by_brute_enumeration():
    # direct terms: y = 1..s; gathered terms: j >= 2 with floor(k/j) > s whose
    # product x*j leaves the array (x*j > X).  Enumerated over every j.
    for n in range(2, 400):
        s_n = math.isqrt(n)
        for u in range(s_n + 1, n + 1, 3):
            X = n // u
            d = g = 0
            for x in range(1, X + 1):
                k = n // x
                s = math.isqrt(k)
                d += s
                g += sum(1 for j in range(2, k + 1) if k // j > s and x * j > X)
            assert oracle.count_terms(n, u) == (d, g), (n, u)


def test_isqrt_u128_matches_library():
    # math.isqrt is Python's own integer square root, independent of the
    # oracle's bisection; values across the whole 128-bit range and at the
    # squares' edges
    rng = np.random.default_rng(128)
    vals = [0, 1, 2, 3, 4, 2**64 - 1, 2**64, 2**126, 2**128 - 1,
            (2**64 - 1) ** 2, (2**64 - 1) ** 2 - 1, 10**38, 11609864264058592345]
    for bits in range(1, 129, 3):
        for _ in range(20):
            v = int(rng.integers(0, 2**62)) * 2**66 + int(rng.integers(0, 2**62)) * 4 + 3
            vals.append(v % (1 << bits))
    for r in (3037000499, 4294967295, 10**10, 10**19 + 7):
        vals += [r * r - 1, r * r, r * r + 1]
    for v in vals:
        assert oracle.isqrt(v) == math.isqrt(v), v


def _resolve_host(n, S):
    """M[x] = 1 - S[x] - sum_{j=2}^{X/x} M[xj] (mod 2^64), x = X..1 (Sec. 2),
    read as int64; the entry with k = 1 is M(1) = 1."""
    X = len(S)
    R = [0] * (X + 1)
    for x in range(X, 0, -1):
        if n // x == 1:
            R[x] = 1
            continue
        acc = sum(R[x * j] for j in range(2, X // x + 1))
        R[x] = (1 - int(S[x - 1]) - acc) % 2**64
    return np.array(R[1:], dtype=np.uint64).view(np.int64)


@pytest.mark.parametrize("n,u,cuts", [
    (10**6, 2000, [1, 2, 500, 1001, 1999]),
    (999_983, 1500, [1, 700, 701, 1499]),
    (12_345_678, 40_000, [1, 3513, 3514, 9000, 20_001]),
    (2**36 + 15, 2 * 10**7, [1, 200_001, 262_144, 262_145, 3 * 10**6]),
])
def test_window_sums_partition_resolves_to_array(n, u, cuts):
    """Windows that cover [1, u) with chained carries C = M(window start - 1)
    sum to the entries' whole update sums; resolving those (Sec. 2) gives the
    recursion's array and the plain table.  A wrong coefficient, a dropped
    term or an off-by-one window edge changes some entry."""
    X = n // u
    total = np.zeros(X, dtype=np.uint64)
    carry = 0
    bounds = cuts + [u]
    for a, b in zip(bounds[:-1], bounds[1:]):
        S, coef, mus = oracle.window_sums(n, u, a, b - a)
        total += S + np.uint64(carry % 2**64) * coef     # wraps mod 2^64
        carry += mus
    got = _resolve_host(n, total)
    assert np.array_equal(got, oracle.mertens_array(n, X, L=min(10**7, max(math.isqrt(n), 10**6))))
    if n <= 2 * 10**7:
        M = oracle.mertens_table(n)
        x = np.arange(1, X + 1)
        assert np.array_equal(got, M[n // x].astype(np.int64))


def test_window_sums_two_word_direct_by_summation_by_parts():
    """n = 10^20 + 12345: entries x <= 10 have k >= 2^63 and s > 3 10^9, so a
    window at 3 10^9 holds only direct terms.  Their coefficients telescope to
    floor(k/y1) - floor(k/(y2+1)), and summation by parts gives
    S = sum mu(y) floor(k/y) - Mw(y2) floor(k/(y2+1)); both in Python integers."""
    n = 10**20 + 12345
    u = round(n ** (2 / 3))
    y1, L = 3 * 10**9, 4000
    y2 = y1 + L - 1
    S, coef, mus = oracle.window_sums(n, u, y1, L, 1, 10)
    mu = [int(v) for v in oracle.mu_window(y1, L)]
    assert mus == sum(mu)
    for x in range(1, 11):
        k = n // x
        assert k >= 2**63 and math.isqrt(k) > y2
        assert int(coef[x - 1]) == (k // y1 - k // (y2 + 1)) % 2**64
        want = sum(m * (k // (y1 + i)) for i, m in enumerate(mu)) - mus * (k // (y2 + 1))
        assert int(S[x - 1]) == want % 2**64, x


def test_window_sums_two_word_gathered_by_y():
    """The same target at y = 10^13 (all terms gathered): counted per y rather
    than per j -- the j with floor(k/j) = y number
    min(floor(k/y), jhi) - max(floor(k/(y+1)), jlo - 1) -- in Python integers,
    for two-word and one-word entries."""
    n = 10**20 + 12345
    u = round(n ** (2 / 3))
    X = n // u
    y1, L = 10**13, 100_000
    xs = list(range(1, 13)) + [1000, X // 2, X]
    Mw = np.cumsum(oracle.mu_window(y1, L).astype(np.int64))
    for x in xs:
        S, coef, _ = oracle.window_sums(n, u, y1, L, x, x)
        k = n // x
        s = math.isqrt(k)
        jlo, jhi = k // u + 1, k // (s + 1)
        want_S = want_c = 0
        for i in range(L):
            y = y1 + i
            c = min(k // y, jhi) - max(k // (y + 1), jlo - 1)
            if c > 0:
                want_S += int(Mw[i]) * c
                want_c += c
        assert int(coef[0]) == want_c and int(S[0]) == want_S % 2**64, x
