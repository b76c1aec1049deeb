"""The byte sieve's decision rule and its word-parallel decode, modelled on the CPU.

The byte kernels keep, per y, A = the sum of odd weights w(p) (the odd integer
nearest S log2 p) over the sieving primes p <= P dividing y, and a square
flag.  All weights are odd, so A's parity is the prime count's parity; the
unsieved cofactor of y is 1 or one prime above P, and a tile threshold thr
(even, at most two units under T = S log2 y - (S/2) log2 P) separates the two
cases wherever the host admits the kernel ((S/2) log2 P >= omega + 2.5,
thr < 126, biased bytes below 2^8).  The device adds 127 - thr to every byte
and reads mu = -1 from bit 0 xor bit 7.  Then four y per 32-bit word are
turned into prefix sums by one multiply and packed to int16 with byte
permutes.  These tests replay both steps in Python on windows where the
kernel runs and compare with sympy's Moebius function and plain prefix sums.
"""
import math

import numpy as np
import pytest

sympy = pytest.importorskip("sympy")

TILE = 131072


def weight(p: int, S: int) -> int:
    """The odd integer nearest S log2 p."""
    return 2 * math.floor((S * math.log2(p) - 1.0) / 2.0 + 0.5) + 1


def omega_max(y: int) -> int:
    w, prod = 0, 1
    for p in sympy.primerange(2, 100):
        prod *= p
        if prod > y:
            break
        w += 1
    return w


def gate(y2: int, P: int, S: int) -> bool:
    half = 0.5 * S * math.log2(P)
    E = omega_max(y2)
    thr = S * math.log2(y2) - half
    return P >= 1024 and half >= E + 2.5 and thr < 126.0 and 127.0 + half + E + 3.0 < 255.0


def tile_threshold(t1: int, P: int, S: int) -> int:
    return math.floor(S * math.log2(t1) - 0.5 * S * math.log2(P)) & ~1


def window_bytes(y0: int, n: int, P: int, S: int):
    """A (weight sums) and square flags for y0 .. y0+n-1, by a plain sieve."""
    A = np.zeros(n, dtype=np.int64)
    sq = np.zeros(n, dtype=bool)
    for p in sympy.primerange(2, P + 1):
        p = int(p)
        A[(-y0) % p::p] += weight(p, S)
        pp = p * p
        if pp < y0 + n:
            sq[(-y0) % pp::pp] = True
    return A, sq


def bytes_of(y: int, P: int, S: int):
    """A and the square flag of one y from its factorisation."""
    f = sympy.factorint(y)
    return (sum(weight(p, S) for p in f if p <= P),
            any(e >= 2 for p, e in f.items() if p <= P))


def decode_byte(A: int, sqf: bool, thr: int) -> int:
    """The device rule: byte W = A + 127 - thr; mu = -1 iff bit 0 xor bit 7."""
    if sqf:
        return 0
    W = A + 127 - thr
    assert 0 <= W < 256
    neg = (W ^ (W >> 7)) & 1
    return -1 if neg else 1


@pytest.mark.parametrize("y0,S", [
    (2**26 + 12345, 4),            # first tile-threshold tiles
    (10**9 + 7, 4),
    (10**12 - 5000, 4),
    (2**41 + 99, 4),               # near the top of S = 4
    (10**13 + 12345, 3),           # S = 3 above 2^42
    (2**46 - 3000, 3),
])
def test_decision_rule_on_windows(y0, S):
    n = 1500
    y2 = y0 + (1 << 28)            # the end of a 2^28-y block holding the window
    P = math.isqrt(y2)
    assert gate(y2, P, S)
    A, sq = window_bytes(y0, n, P, S)
    for i in range(n):
        y = y0 + i
        thr = tile_threshold(max(y - y % TILE, 2**26), P, S)   # from the tile's start
        want = int(sympy.mobius(y))
        # the tile threshold or one even step lower: both must decide alike
        for th in (thr, thr - 2):
            assert decode_byte(int(A[i]), bool(sq[i]), th) == want, (y, th)


def test_decision_rule_hard_cases():
    """Many small primes (largest omega) and a prime just above P."""
    S = 4
    y2 = 10**12 + (1 << 28)
    P = math.isqrt(y2)
    assert gate(y2, P, S)
    thr = tile_threshold(10**12, P, S)
    p19 = 2 * 3 * 5 * 7 * 11 * 13 * 17 * 19          # 8 or more distinct primes
    cases = [p19 * m for m in range(-(-10**12 // p19), y2 // p19 + 1)]
    p31 = p19 * 23 * 29 * 31                          # 11, the most below 10^12 + 2^28
    cases += [p31 * m for m in range(-(-10**12 // p31), y2 // p31 + 1)]
    q = int(sympy.nextprime(P))
    cases += [p * q for p in (2, 3, 5, 7, 11, 101, 1009) if 10**12 <= p * q < y2]
    q2 = int(sympy.nextprime(10**12 // 7919))
    cases += [7919 * q2, 7919 * int(sympy.nextprime(q2))]
    cases = [y for y in cases if 10**12 <= y < y2]
    assert len(cases) > 20
    for y in cases:
        A, sqf = bytes_of(y, P, S)
        want = int(sympy.mobius(y))
        for th in (thr, thr - 2):
            assert decode_byte(A, sqf, th) == want, y


def _byte_perm(x: int, y: int, s: int) -> int:
    b = [(x >> (8 * i)) & 255 for i in range(4)] + [(y >> (8 * i)) & 255 for i in range(4)]
    return sum(b[(s >> (4 * i)) & 7] << (8 * i) for i in range(4))


def test_word_decode_and_int16_packing():
    """pb/mb indicator words -> prefix sums by one multiply -> int16 pairs."""
    rng = np.random.default_rng(4242)
    for trial in range(300):
        mu = rng.choice([-1, 0, 1], size=16, p=[0.3, 0.4, 0.3])
        valid = 16 if trial % 3 else int(rng.integers(0, 17))   # ragged tail
        rb = int(rng.integers(-1536, 1537))                      # M before these 16 y
        got, tot = [], 0
        for k in range(4):
            pb = mb = 0
            for j in range(4):
                i = 4 * k + j
                if i >= valid:
                    continue
                if mu[i] == 1:
                    pb |= 1 << (8 * j)
                elif mu[i] == -1:
                    mb |= 1 << (8 * j)
            D = (((pb - mb + 0x01010101) & 0xFFFFFFFF) * 0x01010101 + 0x00010203) & 0xFFFFFFFF
            # the 32-bit (rb - 4) times 0x00010001: for negative values the high
            # half comes out one less, which the low half's carry gives back
            bx = (((rb + tot - 4) & 0xFFFFFFFF) * 0x00010001) & 0xFFFFFFFF
            for sel in (0x4140, 0x4342):
                w = ((bx + _byte_perm(D, 0x80, sel)) & 0xFFFFFFFF) ^ 0x80008000
                for h in (w & 0xFFFF, w >> 16):
                    got.append(h - 0x10000 if h >= 0x8000 else h)
            tot += (D >> 24) - 4
        masked = [int(m) if i < valid else 0 for i, m in enumerate(mu)]
        want = list(rb + np.cumsum(masked))
        assert got == want
        assert tot == sum(masked)


# ---- weight scale 2, square flag in bit 7 -------------------------------------
# The scale-2 kernel keeps byte = 1 + A (A the sum of w2(p), the odd integer
# nearest 2 log2 p) plus 128 when a sieving prime's square divides y.  The
# host admits it where log2 P >= E + 2.5, thr < 124, 1 + A stays below 127 and
# the biased bytes below 2^8; the device reads W = (byte & 127) + 126 - thr and
# mu = -1 iff bit 0 xor bit 7 of W, mu = 0 on bit 7 of the byte.

def gate2(y2: int, P: int) -> bool:
    half = math.log2(P)
    E = omega_max(y2)
    thr = 2 * math.log2(y2) - half
    amax = 2 * math.log2(y2) + E
    return (P >= 1024 and half >= E + 2.5 and thr < 124.0 and 1.0 + amax < 127.0
            and amax - (thr - 2.0) + 127.0 < 255.0)


def tile_threshold2(t1: int, P: int) -> int:
    return math.floor(2 * math.log2(t1) - math.log2(P)) & ~1


def decode_byte2(b: int, thr: int) -> int:
    assert 0 <= b < 256
    if b & 128:
        return 0
    W = (b & 127) + 126 - thr
    assert 0 <= W < 256
    return -1 if ((W ^ (W >> 7)) & 1) else 1


def byte2_of(y: int, P: int) -> int:
    f = sympy.factorint(y)
    A = sum(weight(p, 2) for p in f if p <= P)
    sq = any(e >= 2 for p, e in f.items() if p <= P)
    assert 1 + A < 128
    return 1 + A + (128 if sq else 0)


@pytest.mark.parametrize("y0", [
    2**26 + 12345,             # first tile-threshold tiles
    10**9 + 7,
    4 * 10**10 - 3000,         # the top of the n = 10^16 workload's sieve range
    10**12 - 5000,
    10**13 + 12345,
    2**46 - 3000,
    2**53 - 2000,              # near the top of the kernel's range
])
def test_scale2_decision_rule_on_windows(y0):
    n = 1200
    y2 = y0 + (1 << 28)
    P = math.isqrt(y2)
    assert gate2(y2, P)
    A, sq = window_bytes(y0, n, P, 2)
    for i in range(n):
        y = y0 + i
        b = 1 + int(A[i]) + (128 if sq[i] else 0)
        assert b == byte2_of(y, P)
        thr = tile_threshold2(max(y - y % 65536, 2**26), P)
        want = int(sympy.mobius(y))
        for th in (thr, thr - 2):
            assert decode_byte2(b, th) == want, (y, th)


def test_scale2_gate_and_hard_cases():
    """The gate admits the n = 10^16 workload's every block (y from 1 to 4e10
    in 2^28-y blocks: P from 2^14 up) and refuses blocks whose P is too small
    for the margin; many small primes and a prime just above P decode right."""
    for b in range(0, 150):
        y2 = (b + 1) << 28
        assert gate2(y2, math.isqrt(y2)), b
    assert not gate2(10**6, 1000)                 # P below 2^10
    y2 = 4 * 10**10
    P = math.isqrt(y2)
    lo = y2 - (1 << 26)
    p19 = 2 * 3 * 5 * 7 * 11 * 13 * 17 * 19
    cases = [p19 * m for m in range(lo // p19, y2 // p19 + 1)]
    q = int(sympy.nextprime(P))
    cases += [p * q for p in range(lo // q, y2 // q + 1) if sympy.isprime(p)]
    cases = [y for y in cases if lo <= y <= y2]
    assert len(cases) > 20
    for y in cases:
        want = int(sympy.mobius(y))
        thr = tile_threshold2(y - y % 65536, P)
        for th in (thr, thr - 2):
            assert decode_byte2(byte2_of(y, P), th) == want, y


def test_scale2_word_decode_and_packed_scan():
    """The scale-2 word step: nsq = 1 where bit 7 is clear, m = nsq and
    (bit 0 xor bit 7 of W), D = (nsq - 2m) 0x01010101 + 0x04040404 holds
    4 + the prefix sums of mu; and two halves' lane sums packed as
    low + 65536 high scan together and unpack exactly."""
    rng = np.random.default_rng(2022)
    thr = 74
    bias4 = (126 - thr) * 0x01010101
    for trial in range(2000):
        bytes_ = [int(v) for v in rng.integers(1, 100, size=4)]
        sq = [bool(v) for v in rng.integers(0, 3, size=4) == 0]
        ws = sum(((b | (128 if q else 0)) << (8 * j)) for j, (b, q) in enumerate(zip(bytes_, sq)))
        nsq = ~(ws >> 7) & 0x01010101
        W = ((ws & 0x7F7F7F7F) + bias4) & 0xFFFFFFFF
        m = (W ^ (W >> 7)) & nsq
        D = (((nsq - 2 * m) & 0xFFFFFFFF) * 0x01010101 + 0x04040404) & 0xFFFFFFFF
        mus = [decode_byte2(b | (128 if q else 0), thr) for b, q in zip(bytes_, sq)]
        for j in range(4):
            assert (D >> (8 * j)) & 255 == 4 + sum(mus[:j + 1]), (trial, j)
    for trial in range(500):
        a = [int(v) for v in rng.integers(-16, 17, size=32)]
        b = [int(v) for v in rng.integers(-16, 17, size=32)]
        inc = np.cumsum([x + 65536 * y for x, y in zip(a, b)])
        for lane in range(32):
            v = int(inc[lane])
            lo = ((v & 0xFFFF) ^ 0x8000) - 0x8000
            assert lo == sum(a[:lane + 1]) and (v - lo) >> 16 == sum(b[:lane + 1])
