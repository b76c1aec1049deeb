"""Division by invariant divisors as the update kernels take it, modelled on the CPU.

The dense update and the global gather path take floor(k/d) for k < 2^63 as
mulhi64(m, 2k) >> l with l = ceil(log2 d) = bitlength(d - 1) and
m = floor(2^(63+l) / d) + 1 (Granlund and Montgomery, PLDI 1994, Sec. 4); the
sieve's first multiples take floor(v/d) for v < 2^31 as mulhi32(m, v) >> (l-1)
with m = floor(2^(31+l) / d) + 1.  These tests recompute both forms with Python
integers and hold them to integer division on the divisors and numerators
where such constants break first: powers of two and their neighbours, the
largest numerators, multiples of d and one below.
"""
import numpy as np

M64 = (1 << 64) - 1


def magic64(d: int):
    l = (d - 1).bit_length()
    return ((1 << (63 + l)) // d) + 1, l


def div64(k: int, m: int, l: int) -> int:
    assert 0 <= k < 1 << 63 and m <= M64
    return ((m * (2 * k)) >> 64) >> l


def magic32(d: int):
    l = (d - 1).bit_length()
    return ((1 << (31 + l)) // d) + 1, l - 1


def div32(v: int, m: int, s: int) -> int:
    assert 0 <= v < 1 << 31 and m < 1 << 32
    return ((m * v) >> 32) >> s


def _divisors(rng, top_bits):
    ds = {1, 2, 3, 5, 7, 641, 65537, 2**31 - 1}
    for b in range(1, top_bits):
        ds.update({2**b - 1, 2**b, 2**b + 1})
    ds.update(int(x) for x in rng.integers(2, 2**top_bits, size=300))
    return sorted(d for d in ds if 1 <= d < 2**top_bits)


def test_64_bit_magics():
    rng = np.random.default_rng(1108)
    for d in _divisors(rng, 40):
        m, l = magic64(d)
        assert m <= M64
        top = (1 << 63) - 1
        ks = {0, 1, d - 1, d, d + 1, top, top - 1, top - (top % d), top - (top % d) - 1}
        ks.update(int(x) for x in rng.integers(0, 2**63, size=40))
        q = top // d
        ks.update({q * d, q * d - 1, (q // 2) * d - 1})
        for k in ks:
            if 0 <= k < 1 << 63:
                assert div64(k, m, l) == k // d, (k, d)


def test_32_bit_magics():
    rng = np.random.default_rng(2011)
    for d in _divisors(rng, 31):
        if d < 2:
            continue
        m, s = magic32(d)
        assert m < 1 << 32
        top = (1 << 31) - 1
        vs = {0, 1, d - 1, d, top, top - (top % d), top - (top % d) - 1}
        vs.update(int(x) for x in rng.integers(0, 2**31, size=40))
        for v in vs:
            if 0 <= v < 1 << 31:
                assert div32(v, m, s) == v // d, (v, d)


def test_a_smaller_shift_breaks():
    """The shift must be ceil(log2 d): one less gives wrong quotients somewhere,
    so the test above would notice a slip in the constant's construction."""
    bad = 0
    for d in range(2**20 + 1, 2**20 + 2001):
        l = (d - 1).bit_length() - 1
        m = ((1 << (63 + l)) // d) + 1
        k = ((2**63 - 1) // d) * d - 1          # the largest k one below a multiple
        bad += div64(k, m, l) != k // d
    assert bad > 0


def test_library_constants_are_these():
    """The built library's own constants (mertens_division_constants: the
    restoring long division on the host side of the kernels' set-up) equal
    the ones modelled above, on the same divisors; no GPU is needed."""
    import paper_1108_0135_gb300 as pm

    rng = np.random.default_rng(1108)
    ds = _divisors(rng, 40) + [2**62 + 1, 2**63 - 1, 3 * 2**60 + 7]
    for d in ds:
        c = pm.mertens_division_constants(d)
        assert (c["m64"], c["l64"]) == magic64(d), d
        if 2 <= d < 2**31:
            assert (c["m32"], c["s32"]) == magic32(d), d
        else:
            assert c["m32"] == 0 and c["s32"] == 0, d
