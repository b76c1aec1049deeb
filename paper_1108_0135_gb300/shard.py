"""One target sharded over ranks (one process per GPU) by y-windows.

Every window's contribution to an entry's update sum is affine in the
window's carry M(y_first - 1) (Sec. 2-3: direct and gathered terms are sums
of M(y) = M_loc(y) + carry), so the ranks run disjoint windows of
[1, y_max] independently through window plans, which keep S_loc and the
coefficient of the carry on the device.  The exchange is an all-gather of
the windows' mu sums (a rank's carry is the sum of those before it), the
library's addition of S_loc + C coef (mod 2^64) into a device buffer, and one
all-reduce of those buffers; rank 0 then resolves from its device buffer.
Nothing of the method's arithmetic runs here.  Windows are cut at equal estimated work
(the sieve is uniform in y, the update terms crowd at small y).
"""
from __future__ import annotations

import math

import numpy as np

from . import _lib as L

# Measured per-unit costs on GB300 (n = 10^16 workload: 68 ms of sieve for
# 4e10 y, 58 ms for 1.0e11 dense terms, 65 ms for 6.2e10 gathered terms), in
# seconds: sieve per y, dense (squarefree) term, gathered term.  Integrated
# over [1, y_max] they give 0.19 s, the measured step.
SIEVE_S_PER_Y = 1.7e-12
DENSE_S_PER_TERM = 0.58e-12
GATHER_S_PER_TERM = 1.05e-12


def work_density(y: np.ndarray, n: int, X: int, c: float = 1.4) -> np.ndarray:
    """Estimated seconds per unit y at y: the sieve, the dense terms of the
    entries whose cut-off c sqrt(k) is above y (a fraction 6/pi^2 of y are
    squarefree), and the gathered terms k/y^2 of the entries whose cut-off is
    below y (k = n/x summed over those x: n ln(X / x_c))."""
    y = np.asarray(y, dtype=np.float64)
    xc = np.minimum(float(X), c * c * float(n) / (y * y))    # entries with cut-off >= y
    dense = 6.0 / math.pi ** 2 * xc
    gathered = float(n) / (y * y) * np.log(np.maximum(float(X) / np.maximum(xc, 1.0), 1.0))
    return SIEVE_S_PER_Y + DENSE_S_PER_TERM * dense + GATHER_S_PER_TERM * gathered


def window_bounds(n: int, u: int, world: int):
    """[(y_first, y_last)] for `world` ranks covering [1, y_max], cut at equal
    estimated work; cuts fall on multiples of 2048."""
    info = L.mertens_describe(n, u)
    X, ymax = info["X"], info["y_max"]
    if world <= 1 or ymax < 2048 * world:
        return [(1, ymax)] + [(ymax + 1, ymax)] * (world - 1)
    ys = np.unique(np.concatenate([np.geomspace(1.0, float(ymax), 8192),
                                   np.linspace(1.0, float(ymax), 8192)]))
    w = work_density(ys, n, X)
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (w[1:] + w[:-1]) * np.diff(ys))])
    cuts = [1]
    for g in range(1, world):
        y = float(np.interp(cum[-1] * g / world, cum, ys))
        c = max(cuts[-1] + 2048, (int(y) // 2048) * 2048 + 1)
        cuts.append(min(c, ymax + 1))
    cuts.append(ymax + 1)
    return [(cuts[g], cuts[g + 1] - 1) for g in range(world)]


def exchange(accumulate, mu_sum: int, X: int, rank: int, world: int, device=None):
    """The exchange step; this function only moves bytes.  The windows' mu
    sums (8 bytes per rank) are all-gathered; `accumulate(mu_before, buf)`
    -- the library's mertens_window_accumulate, which forms the carry
    C = sum(mu_before) and adds S_loc + C coef (mod 2^64) on the device --
    fills a zeroed exchange buffer of 2 X int64 words (the low and high 32-bit
    halves of every entry's sum); one all-reduce (SUM) of those buffers gives
    every rank the whole update sums, with no signed overflow in any backend.
    Returns the buffer (on `device`)."""
    import torch

    buf = torch.zeros(2 * X, dtype=torch.int64, device=device)
    if world > 1:
        import torch.distributed as dist

        mus = [torch.zeros(1, dtype=torch.int64, device=device) for _ in range(world)]
        dist.all_gather(mus, torch.tensor([int(mu_sum)], dtype=torch.int64, device=device))
        before = [int(m.item()) for m in mus[:rank]]
    else:
        before = []
    accumulate(before, buf)
    if world > 1:
        dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    return buf


class ShardedTarget:
    """A target prepared for repeated sharded runs: this rank's window plan
    is made once; step() runs it, exchanges on the device, and resolves on
    rank 0 from the device buffer."""

    def __init__(self, n: int, u: int, block_len: int = 0, rank: int = 0, world: int = 1,
                 device=None):
        import torch

        self.n, self.u, self.rank, self.world = int(n), int(u), rank, world
        self.device = device if device is not None else torch.device("cuda")
        self.X = self.n // self.u
        self.window = window_bounds(self.n, self.u, world)[rank]
        y1, y2 = self.window
        self.plan = L.mertens_plan_window([self.n], y1, y2, self.u, block_len) if y2 >= y1 else 0

    def step(self, stream=None):
        """One sharded run; rank 0 returns M(floor(n/x)), x = 1..X (int64
        numpy array), the other ranks None."""
        import torch

        mu = 0
        if self.plan:
            L.mertens_run(self.plan, stream)
            mu = L.mertens_window_mu_sum(self.plan, 0)

        def accumulate(before, buf):
            if self.plan:
                L.mertens_window_accumulate(self.plan, 0, before, buf, stream)

        buf = exchange(accumulate, mu, self.X, self.rank, self.world, self.device)
        if self.rank != 0:
            return None
        M = torch.empty(self.X, dtype=torch.int64, device=self.device)
        L.mertens_resolve_exchange(self.n, self.u, buf, M, stream)
        return M.cpu().numpy()

    def close(self):
        if self.plan:
            L.mertens_destroy(self.plan)
            self.plan = 0


def run(n: int, u: int, block_len: int = 0, rank: int = 0, world: int = 1, device=None,
        stream=None):
    """M(floor(n/x)), x = 1..floor(n/u), on rank 0 (None elsewhere): this
    rank's window through a window plan, the exchange, then resolve."""
    t = ShardedTarget(n, u, block_len, rank, world, device)
    try:
        return t.step(stream)
    finally:
        t.close()
