/*
 * mertens_oracle.c -- plain, slow, obviously correct CPU definition of the
 * Mertens function, written from the paper "Computing the Mertens function
 * on a GPU" (arXiv:1108.0135).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or call this file.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * constant with the CUDA library.
 *
 * Every function is single threaded and uses only plain loops, 64-bit
 * integers and gcc's unsigned __int128 (the paper, Sec. 5, relies on the same
 * 128-bit type above 2^64).  No blocking, no fusion, no reordering beyond the
 * definitions it follows.
 *
 * What each part follows:
 *   oracle_mu_trial      mu(m) straight from its definition (Sec. 1).
 *   oracle_mu_window     the naive block sieve of Sec. 3 (multiply by -p,
 *                        zero on p^2, compare |A| with y).
 *   oracle_mertens_table M(y) = sum of mu up to y (Sec. 1), y <= L.
 *   oracle_mertens_array the recursion of Sec. 2, M(v) = 1 - sum_{x>=2}
 *                        M(floor(v/x)), with the sum split at t = s+1,
 *                        s = floor(sqrt(v)), evaluated bottom-up over the
 *                        distinct quotients floor(n/d).  It returns the
 *                        paper's array M(floor(n/x)), x = 1..X (Sec. 2).
 *   oracle_isqrt         floor(sqrt(v)) by bisection.
 *   oracle_window_sums   one y-window's share of the split-form sums of
 *                        every array entry, with M(y) taken relative to
 *                        the window start (Sec. 2 split form, Sec. 3's
 *                        block-by-block y axis); 128-bit k, so it reaches
 *                        targets above 2^64.
 *
 * Reading of the garbled split formula (Sec. 2): for any integer t in [1, v],
 *   M(v) = 1 - sum_{x=2}^{floor(v/t)} M(floor(v/x))
 *            - sum_{y=1}^{t-1} (floor(v/y) - floor(v/(y+1))) * M(y),   v >= 2,
 * because x <= floor(v/t) exactly when floor(v/x) >= t, and the x with
 * floor(v/x) = y < t number floor(v/y) - floor(v/(y+1)).  We take t = s+1.
 *
 * Pinned by (tests/test_oracle.py): trial division against the window sieve,
 * the identity sum_{x=1}^n M(floor(n/x)) = 1 (Sec. 2) for every n up to 10^4,
 * the recursion against the plain table for every n up to 10^5 and sampled
 * n up to 10^9, the ratio 0.570591 at n = 7766842813 quoted in Sec. 1, and
 * closed forms (mu of primes, prime squares, products of two primes).  The
 * bisection square root against Python's integer square root over the whole
 * 128-bit range.  The window sums: windows covering [1, u) with chained
 * carries resolve to the recursion's array; above 2^64, the direct
 * coefficients telescope to floor(k/y1) - floor(k/(y2+1)), S by summation by
 * parts, and gathered terms counted per y instead of per j, in Python
 * integers.
 *
 * Reach: oracle_mertens_array needs the plain table up to floor(sqrt(n)) with
 * L < 2^31, so it refuses n >= 2^62; oracle_window_sums has no such limit on
 * n (only on the window: y2 < 2^62, len < 2^31) and is what reaches targets
 * whose k needs two words.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

/* mu(m) from its definition (Sec. 1): 0 if a prime square divides m,
 * otherwise (-1)^(number of distinct prime factors).  m >= 1. */
int oracle_mu_trial(uint64_t m)
{
    if (m == 0)
        return 0;
    int sign = 1;
    for (uint64_t p = 2; p <= m / p; p++) {
        if (m % p == 0) {
            m /= p;
            if (m % p == 0)
                return 0;
            sign = -sign;
        }
    }
    if (m > 1)
        sign = -sign;
    return sign;
}

/* floor(sqrt(v)) for v < 2^128, by bisection on r*r <= v. */
uint64_t oracle_isqrt_u128(uint64_t v_lo, uint64_t v_hi)
{
    u128 v = ((u128)v_hi << 64) | v_lo;
    u128 lo = 0, hi = UINT64_MAX; /* invariant: lo*lo <= v < (hi+1)^2 */
    while (lo < hi) {
        u128 mid = lo + (hi - lo + 1) / 2;
        if (mid * mid <= v)
            lo = mid;
        else
            hi = mid - 1;
    }
    return (uint64_t)lo;
}

/* Primes p <= B by the sieve of Eratosthenes.  Returns the count; the caller
 * frees *out. */
static size_t primes_upto(uint64_t B, uint64_t **out)
{
    if (B < 2) {
        *out = NULL;
        return 0;
    }
    uint8_t *composite = calloc(B + 1, 1);
    size_t count = 0;
    for (uint64_t i = 2; i <= B; i++) {
        if (composite[i])
            continue;
        count++;
        for (uint64_t j = i * i; j <= B; j += i)
            composite[j] = 1;
    }
    uint64_t *p = malloc(sizeof(uint64_t) * (count ? count : 1));
    size_t c = 0;
    for (uint64_t i = 2; i <= B; i++)
        if (!composite[i])
            p[c++] = i;
    free(composite);
    *out = p;
    return count;
}

/* The naive block sieve of Sec. 3 over y in [y1, y1+len-1], y1 >= 1:
 *   1. A[y] = 1 for every y of the block;
 *   2. for every prime p up to ceil(sqrt(y2)) multiply A at the multiples
 *      of p by -p;
 *   3. set A to 0 at the multiples of p^2;
 *   4. mu(y) = 0 if A = 0; sign(A) if |A| = y; otherwise -sign(A).
 * The product of distinct primes dividing y never exceeds y, so int64 holds
 * A for y2 < 2^63.  Returns 0 on success, -1 on bad arguments or memory. */
int oracle_mu_window(uint64_t y1, uint64_t len, int8_t *mu)
{
    if (y1 == 0 || len == 0)
        return len == 0 ? 0 : -1;
    uint64_t y2 = y1 + len - 1;
    if (y2 < y1 || y2 >= ((uint64_t)1 << 63))
        return -1;
    int64_t *A = malloc(sizeof(int64_t) * len);
    if (!A)
        return -1;
    for (uint64_t i = 0; i < len; i++)
        A[i] = 1;
    uint64_t r = oracle_isqrt_u128(y2, 0);
    uint64_t bound = (r * r == y2) ? r : r + 1; /* ceil(sqrt(y2)) */
    uint64_t *pr;
    size_t np = primes_upto(bound, &pr);
    for (size_t t = 0; t < np; t++) {
        uint64_t p = pr[t];
        uint64_t first = ((y1 + p - 1) / p) * p;
        for (uint64_t y = first; y <= y2 && y >= first; y += p)
            A[y - y1] *= -(int64_t)p;
        if (p <= y2 / p) {
            uint64_t pp = p * p;
            uint64_t f2 = ((y1 + pp - 1) / pp) * pp;
            for (uint64_t y = f2; y <= y2 && y >= f2; y += pp)
                A[y - y1] = 0;
        }
    }
    for (uint64_t i = 0; i < len; i++) {
        uint64_t y = y1 + i;
        int64_t a = A[i];
        if (a == 0)
            mu[i] = 0;
        else {
            int sgn = a > 0 ? 1 : -1;
            uint64_t mag = (uint64_t)(a > 0 ? a : -a);
            mu[i] = (int8_t)(mag == y ? sgn : -sgn);
        }
    }
    free(pr);
    free(A);
    return 0;
}

/* M(y) for y = 0..L (Sec. 1): M[0] = 0, M[y] = M[y-1] + mu(y).  L < 2^31,
 * so |M(y)| <= y fits int32.  Returns 0 on success. */
int oracle_mertens_table(uint64_t L, int32_t *M)
{
    if (L >= ((uint64_t)1 << 31))
        return -1;
    M[0] = 0;
    if (L == 0)
        return 0;
    int8_t *mu = malloc(L);
    if (!mu)
        return -1;
    if (oracle_mu_window(1, L, mu) != 0) {
        free(mu);
        return -1;
    }
    int64_t run = 0;
    for (uint64_t y = 1; y <= L; y++) {
        run += mu[y - 1];
        M[y] = (int32_t)run;
    }
    free(mu);
    return 0;
}

/* The paper's array (Sec. 2): out[x-1] = M(floor(n/x)) for x = 1..X, for a
 * target n = n_hi*2^64 + n_lo >= 1.
 *
 * Values v <= L come from the plain table; values v > L are the distinct
 * quotients v = floor(n/d), d = 1..D with D = floor(n/(L+1)), and are built
 * for d = D down to 1 from
 *   M(v) = 1 - sum_{x=2}^{floor(v/(s+1))} M(floor(v/x))
 *            - sum_{y=1}^{s} (floor(v/y) - floor(v/(y+1))) * M(y),
 * s = floor(sqrt(v)).  floor(v/x) = floor(n/(dx)), which is either <= L or a
 * memo entry with index dx <= D.  The table must reach floor(sqrt(n)), so the
 * caller's L is raised to that if smaller.  Sums run in signed 128-bit.
 * Returns 0 on success, -1 on bad arguments, -2 on memory, -3 if a value does
 * not fit int64. */
int oracle_mertens_array(uint64_t n_lo, uint64_t n_hi, uint64_t X, uint64_t L,
                         int64_t *out)
{
    u128 n = ((u128)n_hi << 64) | n_lo;
    if (n == 0 || X == 0 || (u128)X > n)
        return -1;
    uint64_t root = oracle_isqrt_u128(n_lo, n_hi);
    if (L < root)
        L = root;
    if (L < 1)
        L = 1;
    if ((u128)L > n)
        L = (uint64_t)n;
    if (L >= ((uint64_t)1 << 31))
        return -1;
    int32_t *M = malloc(sizeof(int32_t) * (L + 1));
    if (!M)
        return -2;
    if (oracle_mertens_table(L, M) != 0) {
        free(M);
        return -2;
    }
    u128 Dw = n / ((u128)L + 1);
    uint64_t D = (uint64_t)Dw; /* D <= n/L^(1) <= sqrt(n) < 2^64 */
    i128 *memo = malloc(sizeof(i128) * (D + 1));
    if (!memo) {
        free(M);
        return -2;
    }
    for (uint64_t d = D; d >= 1; d--) {
        u128 v = n / d;
        uint64_t s = oracle_isqrt_u128((uint64_t)v, (uint64_t)(v >> 64));
        i128 acc = 1;
        u128 xmax = v / ((u128)s + 1);
        for (u128 x = 2; x <= xmax; x++) {
            u128 w = v / x;
            if (w <= L)
                acc -= M[(uint64_t)w];
            else
                acc -= memo[(uint64_t)(d * x)];
        }
        for (uint64_t y = 1; y <= s; y++) {
            u128 c = v / y - v / ((u128)y + 1);
            acc -= (i128)c * M[y];
        }
        memo[d] = acc;
    }
    int rc = 0;
    for (uint64_t x = 1; x <= X; x++) {
        u128 v = n / x;
        i128 val = (v <= L) ? (i128)M[(uint64_t)v] : memo[x];
        if (val > (i128)INT64_MAX || val < (i128)INT64_MIN) {
            rc = -3;
            val = 0;
        }
        out[x - 1] = (int64_t)val;
    }
    free(memo);
    free(M);
    return rc;
}

/* Number of update terms of the array algorithm for target n and sieve limit
 * u (Sec. 2), counted by enumeration: for every entry x <= X = floor(n/u)
 * with k = floor(n/x) and s = floor(sqrt(k)), the direct terms are y = 1..s
 * and the gathered terms are j = floor(k/u)+1 .. floor(k/(s+1)).  Plain
 * loops; meant for small n.  Returns 0 on success. */
int oracle_count_terms(uint64_t n, uint64_t u, uint64_t *direct,
                       uint64_t *gathered)
{
    if (n == 0 || u == 0 || u > n)
        return -1;
    uint64_t X = n / u, dsum = 0, gsum = 0;
    for (uint64_t x = 1; x <= X; x++) {
        uint64_t k = n / x;
        uint64_t s = oracle_isqrt_u128(k, 0);
        for (uint64_t y = 1; y <= s; y++)
            dsum++;
        for (uint64_t j = k / u + 1; j <= k / (s + 1); j++)
            gsum++;
    }
    *direct = dsum;
    *gathered = gsum;
    return 0;
}

/* One y-window's share of the update of the array algorithm (Sec. 2 split
 * form at t = s+1; Sec. 3 walks the y axis block by block), for the entries
 * x = x_first..x_last of target n = n_hi*2^64 + n_lo with sieve limit u.
 *
 * Entry x has k = floor(n/x), s = floor(sqrt(k)), and its update terms are
 *   direct:   M(y) * (floor(k/y) - floor(k/(y+1)))  for y = 1..s,
 *   gathered: M(floor(k/j))  for j = floor(k/u)+1 .. floor(k/(s+1)).
 * The window is y in [y1, y2], y2 = y1+len-1.  Its M(y) is known only up to
 * the carry C = M(y1-1), so with Mw(y) = sum_{t=y1}^{y} mu(t) (mu from the
 * naive block sieve above) the window's terms are affine in C:
 *   sum (Mw(y) + C) * c_y = S + C * coef.
 * This returns, for every entry, S = the sum of Mw over its direct terms with
 * y in the window (times their coefficients) plus its gathered terms with
 * floor(k/j) in the window, and coef = the sum of those direct coefficients
 * plus the number of those gathered terms, both mod 2^64; and *mu_sum =
 * Mw(y2), the window's carry-out.  The gathered j with floor(k/j) in
 * [y1, y2] are exactly floor(k/(y2+1)) < j <= floor(k/y1).  Every quotient
 * is taken in 128 bits.  Returns 0 on success, -1 on bad arguments, -2 on
 * memory. */
int oracle_window_sums(uint64_t n_lo, uint64_t n_hi, uint64_t u, uint64_t y1,
                       uint64_t len, uint64_t x_first, uint64_t x_last,
                       uint64_t *S_out, uint64_t *coef_out, int64_t *mu_sum)
{
    u128 n = ((u128)n_hi << 64) | n_lo;
    if (n == 0 || u == 0 || (u128)u > n || y1 == 0 || len == 0 ||
        len >= ((uint64_t)1 << 31) || x_first == 0 || x_last < x_first ||
        (u128)x_last > n / u)
        return -1;
    uint64_t y2 = y1 + len - 1;
    if (y2 < y1 || y2 >= ((uint64_t)1 << 62))
        return -1;
    int8_t *mu = malloc(len);
    int32_t *Mw = malloc(sizeof(int32_t) * len);
    if (!mu || !Mw) {
        free(mu);
        free(Mw);
        return -2;
    }
    if (oracle_mu_window(y1, len, mu) != 0) {
        free(mu);
        free(Mw);
        return -2;
    }
    int64_t run = 0;
    for (uint64_t i = 0; i < len; i++) {
        run += mu[i];
        Mw[i] = (int32_t)run;
    }
    *mu_sum = run;
    free(mu);
    for (uint64_t x = x_first; x <= x_last; x++) {
        u128 k = n / x;
        uint64_t s = oracle_isqrt_u128((uint64_t)k, (uint64_t)(k >> 64));
        uint64_t S = 0, coef = 0;
        /* direct terms, y in [y1, min(y2, s)] */
        uint64_t ylast = y2 < s ? y2 : s;
        for (uint64_t y = y1; y <= ylast; y++) {
            u128 c = k / y - k / ((u128)y + 1);
            S += (uint64_t)c * (uint64_t)(int64_t)Mw[y - y1];
            coef += (uint64_t)c;
        }
        /* gathered terms, j in [floor(k/u)+1, floor(k/(s+1))] with
         * floor(k/j) in [y1, y2] */
        u128 jlo = k / u + 1, jhi = k / ((u128)s + 1);
        u128 ja = k / ((u128)y2 + 1) + 1, jb = k / y1;
        if (ja < jlo)
            ja = jlo;
        if (jb > jhi)
            jb = jhi;
        for (u128 j = ja; j <= jb; j++) {
            u128 w = k / j;
            S += (uint64_t)(int64_t)Mw[(uint64_t)(w - y1)];
            coef += 1;
        }
        S_out[x - x_first] = S;
        coef_out[x - x_first] = coef;
    }
    free(Mw);
    return 0;
}
