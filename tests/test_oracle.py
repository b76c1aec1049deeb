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
