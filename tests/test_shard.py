"""Sharding one target over ranks by y-windows (CPU, gloo, world size 2).

Each rank computes its window's carry-free pieces with a plain reference of
the Sec. 2 split form (direct terms M(y)(floor(k/y) - floor(k/(y+1))) for
y <= s, gathered terms M(floor(k/j)) for floor(X/x) < j <= floor(k/(s+1))),
on M(y) from the oracle's table; the exchange step
(paper_1108_0135_gb300.shard.exchange: all-gather of the mu sums, the
addition of S_loc + C coef into a buffer of 32-bit halves, all-reduce) and a
host resolve must give the oracle's array.  On a GPU the addition is the
library's mertens_window_accumulate; here, without one, a plain stand-in with
the same contract fills the buffer.  The window cuts come from
shard.window_bounds.
"""
import math
import os
import socket

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")


def _window_pieces(n, u, a, b, M):
    """(S_loc, coef, mu_sum) of window [a, b] for every entry x = 1..X."""
    X = n // u
    S = np.zeros(X, dtype=np.uint64)
    c = np.zeros(X, dtype=np.uint64)
    base = int(M[a - 1]) if a >= 1 else 0
    for x in range(1, X + 1):
        k = n // x
        s = math.isqrt(k)
        sl = cf = 0
        for y in range(max(a, 1), min(b, s) + 1):
            dq = k // y - k // (y + 1)
            sl += (int(M[y]) - base) * dq
            cf += dq
        for j in range(X // x + 1, k // (s + 1) + 1):
            y = k // j
            if a <= y <= b:
                sl += int(M[y]) - base
                cf += 1
        S[x - 1] = sl % 2**64
        c[x - 1] = cf % 2**64
    mu = int(M[b]) - base if b >= a else 0
    return S, c, mu


def _resolve(n, S):
    X = len(S)
    R = [0] * (X + 1)
    for x in range(X, 0, -1):
        if n // x == 1:
            R[x] = 1
            continue
        acc = sum(R[x * j] for j in range(2, X // x + 1))
        R[x] = (1 - int(S[x - 1]) - acc) % 2**64
    return np.array(R[1:], dtype=np.uint64).view(np.int64)


def _worker(rank, world, port, n, u, out_path):
    import torch.distributed as dist

    from paper_1108_0135_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        M = oracle.mertens_table(n + 1)
        a, b = shard.window_bounds(n, u, world)[rank]
        S_loc, coef, mu = _window_pieces(n, u, a, b, M)

        def accumulate(before, buf):
            # the contract of mertens_window_accumulate, in Python integers
            C = sum(before)
            for i in range(len(S_loc)):
                v = (int(S_loc[i]) + C * int(coef[i])) % 2**64
                buf[2 * i] += v & 0xFFFFFFFF
                buf[2 * i + 1] += v >> 32

        buf = shard.exchange(accumulate, mu, n // u, rank, world, torch.device("cpu"))
        if rank == 0:
            h = buf.numpy()
            S = [(int(h[2 * i]) + (int(h[2 * i + 1]) << 32)) % 2**64 for i in range(n // u)]
            np.save(out_path, _resolve(n, np.array(S, dtype=np.uint64)))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n,u", [(20_000, 400), (99_991, 2_000)])
def test_two_ranks_exchange_and_resolve(n, u, tmp_path):
    import torch.multiprocessing as mp

    out = str(tmp_path / "M.npy")
    mp.start_processes(_worker, args=(2, _free_port(), n, u, out), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(out)
    assert np.array_equal(got, oracle.mertens_array(n, n // u, L=10**5))


def test_work_model_matches_measured_step():
    """The work density integrates to about the measured n = 10^16 step (0.19 s
    on one GB300), so sieve and update work are weighed in the same unit."""
    from paper_1108_0135_gb300 import _lib as L
    from paper_1108_0135_gb300 import shard

    n, u = 10**16, 4 * 10**10
    info = L.mertens_describe(n, u)
    ys = np.unique(np.concatenate([np.geomspace(1.0, float(info["y_max"]), 8192),
                                   np.linspace(1.0, float(info["y_max"]), 8192)]))
    w = shard.work_density(ys, n, info["X"])
    total = float(np.sum(0.5 * (w[1:] + w[:-1]) * np.diff(ys)))
    assert 0.12 < total < 0.3
    sieve = shard.SIEVE_S_PER_Y * info["y_max"]
    assert 0.2 < sieve / total < 0.5          # the sieve is about a third of the step


def test_window_bounds_partition():
    from paper_1108_0135_gb300 import _lib as L
    from paper_1108_0135_gb300 import shard

    for n, u, world in [(10**16, 4 * 10**10, 2), (10**16, 4 * 10**10, 8), (10**12, 10**8, 3),
                        (5000, 100, 4)]:
        ymax = L.mertens_describe(n, u)["y_max"]
        w = shard.window_bounds(n, u, world)
        assert len(w) == world and w[0][0] == 1
        ends = [b for _, b in w if b >= _]
        assert max(ends) == ymax
        for (a0, b0), (a1, b1) in zip(w, w[1:]):
            if b1 >= a1:
                assert a1 == b0 + 1          # contiguous, disjoint, ascending
        if ymax >= 2048 * world:
            assert all(b >= a for a, b in w)
