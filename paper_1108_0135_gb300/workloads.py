"""Seeded synthetic inputs for the isolated-value Mertens computation.

The method's only inputs are integers: targets n, a sieve limit u and a sieve
block length.  This module produces them (fixed configurations and seeded
random draws) and nothing else: it holds none of the method's arithmetic, so
both the CUDA path and the CPU oracle can take their inputs from it.
"""
from __future__ import annotations

import numpy as np

# Single query n = 10^12, u = 10^8, block 2^24 (array of 10^4 entries).
SINGLE_1E12 = dict(name="single n=1e12 u=1e8 L=2^24", n=[10**12], u=10**8, block_len=1 << 24)
# Single query n = 10^16, u = 4e10, block 2^28 (array of 2.5e5 entries).
SINGLE_1E16 = dict(name="single n=1e16 u=4e10 L=2^28", n=[10**16], u=4 * 10**10, block_len=1 << 28)
# 64 close targets n_i = 10^17 + i*10^9 sharing one sieve pass.
BATCH_1E17 = dict(name="batch 64 x (1e17 + i*1e9)", n=[10**17 + i * 10**9 for i in range(64)],
                  u=0, block_len=1 << 28)
# Single query n = 10^18 on the 64-bit path.
SINGLE_1E18 = dict(name="single n=1e18", n=[10**18], u=0, block_len=1 << 28)
# Two-word target n = 10^20 (u ~ n^(2/3)): a fixed window of 64 sieve blocks
# of 2^28 y starting at y = 10^13.
WINDOW_1E20 = dict(name="n=1e20 window of 64 x 2^28 y from y=1e13", n=[10**20],
                   u=21544346900318, block_len=1 << 28, y_first=10**13,
                   y_last=10**13 + 64 * (1 << 28) - 1)


def random_small_cases(seed: int, count: int, n_max: int):
    """Seeded (n, u, block_len) triples with n <= n_max, every u valid
    (floor(sqrt(n)) < u <= n) and block lengths chosen so that the sieve runs
    in 1 to about 40 blocks whose ends fall at ragged places."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        e = rng.uniform(0.0, np.log10(n_max))
        n = int(max(1, min(n_max, int(10 ** e))))
        r = int(np.floor(np.sqrt(n)))
        while r * r > n:
            r -= 1
        while (r + 1) * (r + 1) <= n:
            r += 1
        lo = max(r + 1, 2) if n > 1 else 1
        hi = n
        if lo > hi:
            u = n
        else:
            # log-uniform between just above sqrt(n) and n
            f = rng.uniform(0.0, 1.0)
            u = int(round(lo * (hi / lo) ** f))
            u = min(max(u, lo), hi)
        blocks = int(rng.integers(1, 41))
        block_len = max(1, -(-u // blocks) + int(rng.integers(0, 97)))
        out.append((n, u, block_len))
    return out


def serving_stream(seed: int = 20261203, count: int = 10_000, lo_exp: float = 10.0,
                   hi_exp: float = 16.0, rate_per_s: float = 1000.0):
    """Poisson arrivals of queries with n log-uniform in [10^lo_exp, 10^hi_exp].

    Returns (arrival_times_s, n_values) as numpy arrays."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps)
    e = rng.uniform(lo_exp, hi_exp, size=count)
    n = np.floor(10.0 ** e).astype(np.int64)
    return t, n
