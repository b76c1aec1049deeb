"""The rule by which the plan shares gathered terms between entries x and 2x,
modelled on the host and checked by brute force.

Entry x's gathered terms are M(floor(k_x/j)) for j in [JLO_x, JC0_x], with
k_x = floor(n/x), JLO_x = floor(X/x) + 1 and JC0_x = floor(k_x/(yc_x + 1))
for the entry's dense cut-off yc_x (Sec. 2's split form with the dense
part below yc).  Since floor(floor(n/x)/(2j')) = floor(floor(n/2x)/j'), entry
x's term at j = 2j' is entry 2x's term at j'.  The plan lets an entry with an
even number of factors 2 add its even-j terms to entry 2x, which then
evaluates only j' > floor(JC0_x/2) itself, when that half lies in
[JLO_2x, JC0_2x].  These tests check, with arbitrary values in place of M
and arbitrary valid cut-offs, that every entry still receives each of its
terms exactly once.
"""
import math
import random

import pytest


def _entries(n, u, rng):
    X = n // u
    ent = []
    for x in range(1, X + 1):
        k = n // x
        s = math.isqrt(k)
        jlo = X // x + 1
        jhi = k // (s + 1)
        top = k // jlo - 1 if jlo <= jhi else s
        yc = rng.randint(s, max(s, top))  # any valid cut-off
        ent.append((k, jlo, k // (yc + 1)))
    return X, ent


def _share(X, ent):
    """The plan's rule: (own first j per entry, receiver index or None)."""
    own = [jlo for _, jlo, _ in ent]
    emit = [None] * X
    for x in range(1, X // 2 + 1):
        if ((x & -x).bit_length() - 1) & 1:
            continue  # x itself receives from x/2: not a source
        k1, jlo1, jc1 = ent[x - 1]
        k2, jlo2, jc2 = ent[2 * x - 1]
        if jc1 < jlo1:
            continue
        half = jc1 // 2
        if half < jlo2 or half > jc2:
            continue
        emit[x - 1] = 2 * x - 1
        own[2 * x - 1] = half + 1
    return own, emit


@pytest.mark.parametrize("n,u", [(10**6, 2000), (10**6 + 7, 1001), (3 * 10**5 + 1, 700),
                                 (2**20, 1025), (999_983, 4000)])
def test_every_term_once(n, u):
    rng = random.Random(n ^ u)
    X, ent = _entries(n, u, rng)
    own, emit = _share(X, ent)
    G = {}

    def term(k, j):
        y = k // j
        if y not in G:
            G[y] = rng.getrandbits(40)
        return G[y]

    got = [0] * X
    for e, (k, jlo, jc) in enumerate(ent):
        for j in range(own[e], jc + 1):
            got[e] += term(k, j)
        if emit[e] is not None:
            got[emit[e]] += sum(term(k, j) for j in range(jlo, jc + 1) if j % 2 == 0)
    for e, (k, jlo, jc) in enumerate(ent):
        want = sum(term(k, j) for j in range(jlo, jc + 1))
        assert got[e] == want, (n, u, e + 1)
    shared = sum(max(0, jc - own[e] + 1) for e, (_, _, jc) in enumerate(ent))
    full = sum(max(0, jc - jlo + 1) for _, jlo, jc in ent)
    assert shared < full


def test_floor_identity_behind_the_rule():
    rng = random.Random(5)
    for _ in range(2000):
        n = rng.randrange(1, 10**30)
        x = rng.randrange(1, 10**6)
        j = rng.randrange(1, 10**6)
        assert (n // (2 * x)) // j == (n // x) // (2 * j) == n // (2 * x * j)
