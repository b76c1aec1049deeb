"""The seeded input generators (CPU): every draw is a valid input of the
method, the draws repeat for a seed, and the serving stream has the stated
shape (n log-uniform over the range, Poisson arrivals at the stated rate)."""
import math

import numpy as np

from paper_1108_0135_gb300 import workloads


def test_random_small_cases_are_valid_and_seeded():
    cases = workloads.random_small_cases(7, 400, 10**10)
    assert cases == workloads.random_small_cases(7, 400, 10**10)
    assert cases != workloads.random_small_cases(8, 400, 10**10)
    for n, u, bl in cases:
        assert 1 <= n <= 10**10
        r = math.isqrt(n)
        assert (r < u <= n) or (n == 1 and u == 1)
        assert bl >= 1
        assert 1 <= -(-u // bl) <= 41          # one to about forty sieve blocks
    # the draws spread over the orders of magnitude
    assert len({len(str(n)) for n, _, _ in cases}) >= 8


def test_serving_stream_shape():
    t, n = workloads.serving_stream(seed=11, count=4000, lo_exp=10.0, hi_exp=16.0,
                                    rate_per_s=500.0)
    t2, n2 = workloads.serving_stream(seed=11, count=4000, lo_exp=10.0, hi_exp=16.0,
                                      rate_per_s=500.0)
    assert np.array_equal(t, t2) and list(n) == list(n2)
    assert len(t) == len(n) == 4000
    assert np.all(np.diff(t) > 0) and t[0] > 0
    n = np.asarray([int(v) for v in n], dtype=np.float64)
    assert n.min() >= 1e10 and n.max() <= 1e16
    # log-uniform: each decade holds about a sixth of the queries
    counts = np.histogram(np.log10(n), bins=6, range=(10.0, 16.0))[0]
    assert np.all(np.abs(counts - 4000 / 6) < 5 * math.sqrt(4000 / 6))
    # Poisson arrivals: exponential gaps with mean 1/rate (coefficient of variation ~1)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * 500.0 - 1.0) < 0.1
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1


def test_fixed_configurations():
    assert workloads.SINGLE_1E16["n"] == [10**16] and workloads.SINGLE_1E16["u"] == 4 * 10**10
    assert workloads.SINGLE_1E12["n"] == [10**12] and workloads.SINGLE_1E12["u"] == 10**8
    b = workloads.BATCH_1E17["n"]
    assert len(b) == 64 and b[0] == 10**17 and b[63] == 10**17 + 63 * 10**9
    w = workloads.WINDOW_1E20
    assert w["y_last"] - w["y_first"] + 1 == 64 * w["block_len"] and w["y_first"] == 10**13
