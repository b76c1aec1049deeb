"""One target sharded over ranks (one process per GPU) by y-windows.

Every window's contribution to an entry's update sum is affine in the
window's carry M(y_first - 1) (Sec. 2-3: direct and gathered terms are sums
of M(y) = M_loc(y) + carry), so the ranks run disjoint windows of
[1, y_max] independently through window plans, which return S_loc, the
coefficient of the carry and the window's mu sum.  The exchange is an
all-gather of the mu sums (a rank's carry is the sum of those before it) and
one all-reduce of the entries' sums S = sum over ranks of S_loc + C coef
(mod 2^64); rank 0 then resolves.  Windows are cut at equal estimated work
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


def combine(S_loc: np.ndarray, coef: np.ndarray, mu_sum: int, rank: int, world: int,
            device=None) -> np.ndarray:
    """The exchange step.  Every rank passes its window's S_loc, coef and mu
    sum; every rank gets S = sum_g (S_loc,g + C_g coef_g) mod 2^64 with
    C_g = sum_{h<g} mu_h.  The all-reduce carries the 32-bit halves of the
    64-bit sums, so no backend sees a signed overflow."""
    import torch
    import torch.distributed as dist

    mus = [torch.zeros(1, dtype=torch.int64, device=device) for _ in range(world)]
    dist.all_gather(mus, torch.tensor([int(mu_sum)], dtype=torch.int64, device=device))
    carry = sum(int(m.item()) for m in mus[:rank])
    part = S_loc.astype(np.uint64) + np.uint64(carry % 2**64) * coef.astype(np.uint64)
    halves = np.stack([part & np.uint64(0xFFFFFFFF), part >> np.uint64(32)]).astype(np.int64)
    t = torch.from_numpy(halves).to(device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    h = t.cpu().numpy().astype(np.uint64)
    return (h[1] << np.uint64(32)) + h[0]


class ShardedTarget:
    """A target prepared for repeated sharded runs: this rank's window plan
    is made once; step() runs it, exchanges, and resolves on rank 0."""

    def __init__(self, n: int, u: int, block_len: int = 0, rank: int = 0, world: int = 1,
                 device=None):
        self.n, self.u, self.rank, self.world, self.device = int(n), int(u), rank, world, device
        self.X = self.n // self.u
        self.window = window_bounds(self.n, self.u, world)[rank]
        y1, y2 = self.window
        self.plan = L.mertens_plan_window([self.n], y1, y2, self.u, block_len) if y2 >= y1 else 0

    def step(self, stream=None):
        if self.plan:
            L.mertens_run(self.plan, stream)
            S_loc, coef, mu = L.mertens_window_result(self.plan, 0)
        else:
            S_loc = np.zeros(self.X, dtype=np.uint64)
            coef = np.zeros(self.X, dtype=np.uint64)
            mu = 0
        S = combine(S_loc, coef, mu, self.rank, self.world, self.device) if self.world > 1 \
            else S_loc
        if self.rank != 0:
            return None
        return L.mertens_resolve(self.n, self.u, S, stream)

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
