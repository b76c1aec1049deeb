"""The shared-memory gather's float-estimate quotient, modelled on the CPU.

A gathered term inside a tile [t1, t1 + 2^15) has y - t1 = floor(R / j) with
R = k - t1 j.  The kernel estimates it in single precision -- R and j built
from exact 16/23-bit pieces, stepped by fused multiply-adds from the start of
a lane's run, 1/j from rcp.approx (at most one ulp off), the product less
17/32 rounded to an integer through the 1.5 * 2^23 bias -- and corrects it
with the exact remainder.  This test replays those float32 operations exactly
(every fused multiply-add rounded once, from exact rationals) with the
reciprocal pushed one ulp either way, and checks every quotient against
integer division: runs ascending in j (the lane loop, R falling by t1) and
descending by 32 (the warp loop, R rising by 32 t1), random tiles and the
edges (R a multiple of j, one below, j around 2^24, 2^29 and 2^31).
"""
import math
from fractions import Fraction

import numpy as np

TILE = 32768
f32 = np.float32


def _rn32(q: Fraction) -> np.float32:
    """The float32 nearest to the rational q (ties to even): one rounding."""
    if q == 0:
        return f32(0.0)
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    scale = Fraction(2) ** (e - 23)
    m = a / scale
    r = math.floor(m)
    frac = m - r
    if frac > Fraction(1, 2) or (frac == Fraction(1, 2) and r % 2 == 1):
        r += 1
    return f32(sign * float(r * scale))


def fma(a, b, c):
    return _rn32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def fadd(a, b):
    return _rn32(Fraction(float(a)) + Fraction(float(b)))


def float_of(v: int) -> np.float32:
    lo, hi = v & 0xFFFFFFFF, v >> 32
    assert hi < 2**23
    fh, fa, fb = f32(hi), f32(lo >> 16), f32(lo & 0xFFFF)   # exact pieces
    return fma(fh, f32(4294967296.0), fma(fa, f32(65536.0), fb))


def rcp(jf: np.float32, ulps: int) -> np.float32:
    r = _rn32(1 / Fraction(float(jf)))
    return f32(float(r) + ulps * float(np.spacing(r)))


def quotient(Rf, jf, R, j, lim, ulps, wide):
    t = fadd(fma(Rf, rcp(jf, ulps), f32(-0.53125)), f32(12582912.0))
    assert 2**23 <= float(t) < 2**24                  # the bias keeps integer spacing
    qs = int(t) - 12582912
    if wide:
        rem = R - qs * j
    else:
        rem = ((R & 0xFFFFFFFF) - ((qs & 0xFFFFFFFF) * j)) & 0xFFFFFFFF
    q = (qs + (1 if rem >= j else 0)) & 0xFFFFFFFF
    return min(q, lim)


def _check_lane_run(k, t1, jb, cnt):
    R0 = k - t1 * jb
    Rf0, jf0, t1f = float_of(R0), float_of(jb), float_of(t1)
    wide = k // t1 >= 2**31
    for i in range(cnt):
        j = jb + i
        R = k - t1 * j
        Rf, jf = fma(f32(i), -t1f, Rf0), fadd(jf0, f32(i))
        for ulps in (-1, 1):
            assert quotient(Rf, jf, R, j, TILE - 1, ulps, wide) == R // j, (k, t1, j, ulps)


def _check_warp_run(k, t1, j0, jb):
    R0, dR = k - t1 * j0, 32 * t1
    Rf0, jf0, dRf = float_of(R0), float_of(j0), float_of(dR)
    wide = k // t1 >= 2**31
    j, i = j0, 0
    while j >= jb:
        R = k - t1 * j
        Rf, jf = fma(f32(i), dRf, Rf0), fma(f32(i), f32(-32.0), jf0)
        for ulps in (-1, 1):
            assert quotient(Rf, jf, R, j, TILE - 1, ulps, wide) == R // j, (k, t1, j, ulps)
        j -= 32
        i += 1


def _tile_case(rng, jmid):
    """A tile t1 > j (gathered terms have y > sqrt(k) > j) with terms for j near jmid."""
    t1 = int(max(jmid + 1, 2048) * rng.uniform(1.0, 3.0))
    k = jmid * (t1 + int(rng.integers(0, TILE)))
    jt = min(k // t1, math.isqrt(k))
    jb = k // (t1 + TILE) + 1
    return k, t1, jb, jt


def test_random_tiles_both_loop_forms():
    rng = np.random.default_rng(20260)
    done = 0
    while done < 120:
        jmid = max(2, int(2 ** rng.uniform(1, 31.4)))
        k, t1, jb, jt = _tile_case(rng, jmid)
        if jt < jb:
            continue
        _check_lane_run(k, t1, jb, min(12, jt - jb + 1))
        lane = int(rng.integers(0, 32))
        if jt - lane >= jb:
            _check_warp_run(k, t1, jt - lane, max(jb, jt - lane - 32 * 8))
        done += 1


def test_exact_multiples_and_powers_of_two():
    # R = N j (the estimate sits just under an integer) and R = N j - 1
    for j in (3, 2**24 - 1, 2**24 + 1, 2**29 - 3, 2**29 + 5, 2**31 - 1, 2**31 + 7, 3 * 10**9):
        t1 = j + 12345
        for N in (0, 1, 2, 255, TILE - 2, TILE - 1):
            for off in (0, 1, j - 1):
                R = N * j + off
                if R >= TILE * j:
                    continue
                k = R + t1 * j
                _check_lane_run(k, t1, j, 1)
                _check_warp_run(k, t1, j, j)
