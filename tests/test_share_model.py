"""The rule by which the plan shares gathered terms along chains x, 2x, 4x,
8x, 16x of one target, modelled on the host and checked by brute force.

Entry x's gathered terms are M(floor(k_x/j)) for j in [JLO_x, JC0_x], with
k_x = floor(n/x), JLO_x = floor(X/x) + 1 and JC0_x = floor(k_x/(yc_x + 1))
for the entry's dense cut-off yc_x (Sec. 2's split form with the dense
part below yc).  Since floor(floor(n/x)/(2j')) = floor(floor(n/2x)/j'), entry
x's term at j = 2j' is entry 2x's term at j'.  A link x -> 2x is valid when
h = floor(JC0_x/2) lies in [JLO_2x, JC0_2x]; entry 2x then evaluates only
j' > h itself, and every entry adds the sum of its own terms at j = 0 mod 2^s
to entry 2^s x along valid links (chains restart where the power of two in
x is 0 mod 5: at most four links).  These tests check, with arbitrary values
in place of M and arbitrary valid cut-offs, that every entry still receives
each of its terms exactly once.
"""
import math
import random

import pytest


def _entries(n, u, rng, cut="random"):
    X = n // u
    ent = []
    for x in range(1, X + 1):
        k = n // x
        s = math.isqrt(k)
        jlo = X // x + 1
        jhi = k // (s + 1)
        top = k // jlo - 1 if jlo <= jhi else s
        if cut == "random":
            yc = rng.randint(s, max(s, top))  # any valid cut-off
        else:  # about 1.4 sqrt(k), as the plan takes it (long valid chains)
            yc = min(max(int(1.4 * math.sqrt(k)), s), max(s, top))
        ent.append((k, jlo, k // (yc + 1)))
    return X, ent


def _share(X, ent):
    """The plan's rule: own first j per entry, and (x, L) of what it feeds."""
    own = [jlo for _, jlo, _ in ent]
    link = [False] * (X // 2 + 1)
    for x in range(1, X // 2 + 1):
        if ((2 * x) & -(2 * x)).bit_length() % 5 == 1:
            continue  # 2x starts a chain (its power of two is 0 mod 5)
        _, _, jc1 = ent[x - 1]
        _, jlo2, jc2 = ent[2 * x - 1]
        h = jc1 // 2
        if h < jlo2 or h > jc2:
            continue
        link[x] = True
        own[2 * x - 1] = h + 1
    levels = [0] * X
    for x in range(1, X // 2 + 1):
        L, y = 0, x
        while L < 4 and 2 * y <= X and link[y]:
            L, y = L + 1, 2 * y
        levels[x - 1] = L
    return own, levels


@pytest.mark.parametrize("n,u", [(10**6, 2000), (10**6 + 7, 1001), (3 * 10**5 + 1, 700),
                                 (2**20, 1025), (999_983, 4000)])
@pytest.mark.parametrize("cut", ["random", "plan"])
def test_every_term_once(n, u, cut):
    rng = random.Random(n ^ u)
    X, ent = _entries(n, u, rng, cut)
    own, levels = _share(X, ent)
    G = {}

    def term(k, j):
        y = k // j
        if y not in G:
            G[y] = rng.getrandbits(40)
        return G[y]

    got = [0] * X
    for e, (k, jlo, jc) in enumerate(ent):
        x = e + 1
        for j in range(own[e], jc + 1):
            got[e] += term(k, j)
            for s in range(1, levels[e] + 1):
                if j % (1 << s) == 0:
                    got[(x << s) - 1] += term(k, j)
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


def _mobius_upto(N):
    mu = [1] * (N + 1)
    mu[0] = 0
    is_comp = [False] * (N + 1)
    for p in range(2, N + 1):
        if not is_comp[p]:
            for m in range(p, N + 1, p):
                is_comp[m] = is_comp[m] or m != p
                mu[m] = -mu[m]
            for m in range(p * p, N + 1, p * p):
                mu[m] = 0
    return mu


def test_dense_form_odd_terms_of_2x_are_even_terms_of_x():
    """The dense form's sharing: for k' = floor(k/2), the odd squarefree
    y <= b give sum mu(y) floor(k'/y) = -sum over the even squarefree
    y' <= 2b of mu(y') floor(k/y') (y' = 2y; mu(2y) = -mu(y) for odd y)."""
    N = 5000
    mu = _mobius_upto(N)
    rng = random.Random(11)
    for _ in range(200):
        k = rng.randrange(2, 10**15)
        b = rng.randrange(1, N // 2)
        lhs = sum(mu[y] * ((k // 2) // y) for y in range(1, b + 1, 2))
        rhs = -sum(mu[y] * (k // y) for y in range(2, 2 * b + 1, 2))
        assert lhs == rhs, (k, b)
    # the table itself against its definition on a few values
    assert [mu[i] for i in (1, 2, 3, 4, 6, 30, 12, 105)] == [1, -1, -1, 0, 1, -1, 0, -1]
