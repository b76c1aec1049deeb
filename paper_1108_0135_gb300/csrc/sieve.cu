// Steps a1 (mu_sieve) and a2 (m_scan) of the isolated-value Mertens method,
// fused into one kernel per sieve block: mu(y) by a segmented log sieve, then
// M(y) by prefix sum (arXiv:1108.0135, Sec. 3, steps 0-5 of the log sieve),
// stored as int16 relative to M at the start of each kSegY-segment; a second
// small kernel turns the segment sums into int64 segment offsets carrying
// M(y1 - 1) from the previous block.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace mert {

// ---------------------------------------------------------------------------
// a1: per-block remainders of the sieving primes.
// ---------------------------------------------------------------------------
__global__ void sieve_block_prep_kernel(uint64_t y1, uint32_t np, const uint32_t *__restrict__ p,
                                        uint32_t *__restrict__ r, uint32_t *__restrict__ qm,
                                        uint64_t *__restrict__ r2)
{
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np)
        return;
    uint64_t pp = p[t];
    r[t] = (uint32_t)(y1 % pp);
    qm[t] = (uint32_t)((y1 / pp) % pp);
    if (r2)
        r2[t] = y1 % (pp * pp);
}

struct SieveArgs {
    uint64_t y1, len;
    uint32_t np, np_small;  // primes used; [4, np_small) sieved warp-cooperatively
    uint32_t np_quarter;    // [4, np_quarter) sieved in quarter-tile pieces
    float thr_bias;         // (kLogScale/2) * log2(P), all primes <= P sieved
    const uint32_t *p, *lg, *r, *qm, *pat_even, *pat_odd;
    const uint64_t *m;
    const uint8_t *l;
    int16_t *Mloc;
    int32_t *segsum;
    int8_t *mu_out;
    uint64_t mu_base, mu_end;
};

// First multiple of p at or after t1 = y1 + a0, as an offset `off` into the
// tile, and c = (that multiple / p) mod p, which is 0 exactly when p^2 divides
// the multiple.  Uses y1 mod p and floor(y1/p) mod p of the block.
__device__ __forceinline__ void first_multiple(const SieveArgs &a, uint32_t t, uint64_t a0,
                                               uint32_t &p, uint32_t &off, uint32_t &c,
                                               uint64_t &m, unsigned &l)
{
    p = a.p[t];
    m = a.m[t];
    l = a.l[t];
    const uint64_t v = (uint64_t)a.r[t] + a0;       // t1 - floor(y1/p)*p
    const uint64_t qv = div_magic(v << 1, m, l);     // floor(v / p)
    const uint32_t off0 = (uint32_t)(v - qv * p);    // t1 mod p
    off = off0 ? p - off0 : 0u;
    const uint64_t c0 = (uint64_t)a.qm[t] + qv + (off0 ? 1u : 0u);
    c = (uint32_t)(c0 - div_magic(c0 << 1, m, l) * p);
}

// mu of one sieve half-word h given the integer threshold ithr (see below).
__device__ __forceinline__ int decode_mu(uint32_t h, int ithr)
{
    const int A = (int)(h & 1023u);
    const int cnt = (int)((h >> 10) & 15u);
    const int extra = A > ithr ? 0 : 1;  // 1: one prime factor above P remains
    const int mu = ((cnt + extra) & 1) ? -1 : 1;
    return (h & kSquareBit) ? 0 : mu;
}

// floor(8 log2 y - 4 log2 P): A exceeds it exactly when the sieved primes
// account for all of y.
__device__ __forceinline__ int thr_of(uint64_t y, float bias)
{
    return (int)floorf((float)kLogScale * __log2f(__ull2float_rn(y)) - bias);
}

// Multiples of prime t in the tile offsets [lo, hi), lanes over them.
__device__ __forceinline__ void sieve_prime_warp(const SieveArgs &a, uint32_t *w, uint32_t t,
                                                 uint64_t a0, uint32_t lo, uint32_t hi, int lane)
{
    uint32_t p, off, c;
    uint64_t m;
    unsigned l;
    first_multiple(a, t, a0, p, off, c, m, l);
    if (off < lo) {
        // steps = ceil((lo - off) / p); c = (c + steps) mod p, by the magic of p
        const uint64_t steps = div_magic((uint64_t)(lo - off + p - 1) << 1, m, l);
        off += (uint32_t)steps * p;
        const uint64_t cs = (uint64_t)c + steps;
        c = (uint32_t)(cs - div_magic(cs << 1, m, l) * p);
    }
    const uint32_t add = a.lg[t] | kCountOne;
    for (uint32_t yo = off + (uint32_t)lane * p; yo < hi; yo += 32u * p)
        atomicAdd(&w[yo >> 1], add << ((yo & 1u) << 4));
    // multiples of p^2: the first is (c ? p - c : 0) multiples of p after off
    // (p < 2048, so p^2 and these offsets fit 32 bits)
    const uint32_t p2 = p * p;
    for (uint32_t yo = off + (c ? p - c : 0u) * p + (uint32_t)lane * p2; yo < hi; yo += 32u * p2)
        atomicOr(&w[yo >> 1], kSquareBit << ((yo & 1u) << 4));
}

// One tile of kSieveTile y.  Shared half-word per y: every sieving prime p
// adds round(8 log2 p) plus one to the prime count at its multiples and sets
// the square bit at multiples of p^2; primes 2, 3, 5, 7 and their squares come
// from a periodic pattern.  Decoding is exact: with all primes <= P sieved and
// (P+1)^2 > y, the unsieved cofactor c of y is 1 or a prime > P.  The log sum
// A is within 7.5 units of 8 log2 y when c = 1 (at most 15 distinct primes,
// each rounded by <= 1/2) and at least 8 log2(P+1) - 7 units below it
// otherwise, so "A > 8 log2 y - 4 log2 P" decides c = 1 for every P >= 7
// (margins >= 3.7 units).  mu = 0 if the square bit is set, else
// (-1)^(count + [c > 1]).  Each warp then turns its 2048 y (one segment)
// into M relative to the segment start with a warp scan.
//
// Sieving work is handed out to warps through a shared counter, largest jobs
// first: primes below 128 in quarter-tile pieces, the other primes below 2048
// one per warp (lanes over multiples), then the larger primes 32 at a time
// (a lane per prime).
__global__ void __launch_bounds__(kSieveThreads, 1) mu_sieve_kernel(SieveArgs a)
{
    extern __shared__ uint32_t w[];  // kSieveWords words, two y each
    __shared__ uint32_t s_job;
    const uint64_t a0 = (uint64_t)blockIdx.x * kSieveTile;
    const uint64_t t1 = a.y1 + a0;
    const uint32_t tl = (uint32_t)((a.len - a0) < (uint64_t)kSieveTile ? (a.len - a0) : kSieveTile);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // pattern of primes 2, 3, 5, 7 and their squares
    {
        const uint32_t ph = (uint32_t)(t1 % kPatternPeriod);
        const uint32_t *pat = (ph & 1u) ? a.pat_odd : a.pat_even;
        const uint32_t j0 = ph >> 1;
        for (uint32_t i = threadIdx.x; i < (uint32_t)kSieveWords; i += kSieveThreads) {
            uint32_t idx = j0 + i;
            if (idx >= kPatternWords)
                idx -= kPatternWords;
            if (idx >= kPatternWords)
                idx -= kPatternWords;
            w[i] = pat[idx];
        }
        if (threadIdx.x == 0)
            s_job = 0;
    }
    __syncthreads();

    const uint32_t nquart = a.np_quarter > 4 ? a.np_quarter - 4 : 0;  // primes 11..127
    const uint32_t jq = 4 * nquart;
    const uint32_t js = jq + (a.np_small > a.np_quarter ? a.np_small - a.np_quarter : 0);
    const uint32_t nlarge = a.np > a.np_small ? a.np - a.np_small : 0;
    const uint32_t jobs = js + (nlarge + 31) / 32;
    for (;;) {
        uint32_t job = 0;
        if (lane == 0)
            job = atomicAdd(&s_job, 1u);
        job = __shfl_sync(0xffffffffu, job, 0);
        if (job >= jobs)
            break;
        if (job < jq) {
            const uint32_t q = job & 3u;
            const uint32_t lo = q * (kSieveTile / 4), hi = min(tl, (q + 1) * (kSieveTile / 4));
            if (lo < hi)
                sieve_prime_warp(a, w, 4 + (job >> 2), a0, lo, hi, lane);
        } else if (job < js) {
            sieve_prime_warp(a, w, a.np_quarter + (job - jq), a0, 0, tl, lane);
        } else {
            const uint32_t t = a.np_small + (job - js) * 32u + (uint32_t)lane;
            if (t < a.np) {
                uint32_t p, off, c;
                uint64_t m;
                unsigned l;
                first_multiple(a, t, a0, p, off, c, m, l);
                const uint32_t add = a.lg[t] | kCountOne;
                for (uint32_t yo = off; yo < tl; yo += p)
                    atomicAdd(&w[yo >> 1], add << ((yo & 1u) << 4));
                // p^2 > 2^22 > tile: at most one multiple of p^2, (c ? p - c : 0)
                // multiples of p after off
                const uint64_t sq = (uint64_t)off + (uint64_t)(c ? p - c : 0u) * p;
                if (sq < tl)
                    atomicOr(&w[sq >> 1], kSquareBit << (((uint32_t)sq & 1u) << 4));
            }
        }
    }
    __syncthreads();

    // decode + scan: warp owns words [wb, wb+1024) = y offsets [2wb, 2wb+2048)
    const uint32_t wb = (uint32_t)warp * 1024u;
    const uint32_t so = 2u * wb;  // segment start within the tile
    if (so >= tl)
        return;
    const uint64_t ys = t1 + so;
    const bool big = ys >= (1ull << 20);
    const int thw = big ? thr_of(ys, a.thr_bias) : 0;  // y varies by < 2^-9 in the segment
    const bool want_mu = a.mu_out && ys <= a.mu_end && ys + 2047 >= a.mu_base;
    int run = 0;
#pragma unroll 1
    for (int r = 0; r < 8; ++r) {
        const uint32_t wi = wb + (uint32_t)r * 128u + 4u * (uint32_t)lane;  // 4 words = 8 y
        const uint4 q4 = *reinterpret_cast<const uint4 *>(w + wi);
        const uint32_t ws[4] = {q4.x, q4.y, q4.z, q4.w};
        const uint32_t o0 = 2u * wi;  // tile offset of the first of the 8 y
        const uint64_t y0 = t1 + o0;
        int th[8];
        if (big) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                th[k] = thw;
        } else if (y0 >= 16384) {
            const int t0 = thr_of(y0, a.thr_bias);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                th[k] = t0;
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                th[k] = thr_of(y0 + k, a.thr_bias);
        }
        int mu[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            mu[2 * k] = decode_mu(ws[k] & 0xffffu, th[2 * k]);
            mu[2 * k + 1] = decode_mu(ws[k] >> 16, th[2 * k + 1]);
        }
        if (o0 + 8u > tl) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (o0 + k >= tl)
                    mu[k] = 0;
        }
        int loc[8], sum = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            sum += mu[k];
            loc[k] = sum;
        }
        int inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int nb = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o)
                inc += nb;
        }
        const int base = run + inc - sum;
        run += __shfl_sync(0xffffffffu, inc, 31);
        if (o0 + 8u <= tl) {
            uint4 out;
            out.x = (uint32_t)(uint16_t)(int16_t)(base + loc[0]) |
                    ((uint32_t)(uint16_t)(int16_t)(base + loc[1]) << 16);
            out.y = (uint32_t)(uint16_t)(int16_t)(base + loc[2]) |
                    ((uint32_t)(uint16_t)(int16_t)(base + loc[3]) << 16);
            out.z = (uint32_t)(uint16_t)(int16_t)(base + loc[4]) |
                    ((uint32_t)(uint16_t)(int16_t)(base + loc[5]) << 16);
            out.w = (uint32_t)(uint16_t)(int16_t)(base + loc[6]) |
                    ((uint32_t)(uint16_t)(int16_t)(base + loc[7]) << 16);
            *reinterpret_cast<uint4 *>(a.Mloc + a0 + o0) = out;
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (o0 + k < tl)
                    a.Mloc[a0 + o0 + k] = (int16_t)(base + loc[k]);
        }
        if (want_mu) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint64_t y = y0 + k;
                if (o0 + k < tl && y >= a.mu_base && y <= a.mu_end)
                    a.mu_out[y - a.mu_base] = (int8_t)mu[k];
            }
        }
    }
    if (lane == 0)
        a.segsum[(a0 + so) >> kSegShift] = run;
}

// ---------------------------------------------------------------------------
// a1 + a2, byte variant.  Same method (Sec. 3 log sieve, then the prefix sum),
// laid out for issue throughput: one byte per y and one square bit per y, so a
// tile holds 131072 y; every division of the per-tile set-up is a 32-bit
// invariant-divisor multiply; and the decode works on four y per 32-bit word.
//
// Byte of y: B0 + sum over the distinct sieving primes p | y of w(p), where
// w(p) is the odd integer nearest S log2 p (|w(p) - S log2 p| <= 1; S = 4
// below 2^42, 3 above) and B0 a bias fixed per tile.  Because every weight is
// odd, the parity of the sum is the parity of the prime count.  For
// squarefree y with unsieved cofactor c (1 or a prime > P, as in the 16-bit
// kernel) the weight sum A satisfies
//     c = 1:  A >= S log2 y - E,     c > 1:  A <= S log2 y - S log2 P + E,
// E the summed rounding error, at most the number of distinct prime factors
// (11 below 2^42, 13 below 2^54).  The threshold T = S log2 y - (S/2) log2 P
// separates the two with (S/2) log2 P - E units either side; the host takes
// this kernel only where that exceeds 2.5 (P >= 2^10), so an integer
// threshold anywhere in [T - 2, T] is exact.  Tiles at y >= 2^26 use one even
// threshold thr per tile and B0 = 127 - thr (odd), which puts the decision
// into bit 7 of the byte and the count parity (xor 1) into bit 0:  mu = -1
// exactly when bit 0 and bit 7 of the biased byte differ.  The host also
// keeps thr < 127 and the biased bytes below 2^8.
// ---------------------------------------------------------------------------
struct ByteArgs {
    uint64_t y1;
    uint32_t len;         // <= 2^30
    uint32_t np;          // primes used (all p <= P)
    uint32_t np_piece;    // [4, np_piece): p < 128, sieved in eighth-tile pieces
    uint32_t np_small;    // [np_piece, np_small): p < 2048, a warp per prime
    uint32_t np_mid;      // persistent kernel: [np_small, np_mid) p < 2^17, [np_mid, np) above
    uint32_t cap;         // persistent kernel: bucket entries per tile
    float scale;          // S: w(p) = odd integer nearest S log2 p
    float thr_half;       // (S/2) log2 P
    const uint4 *pq;
    const uint32_t *r;    // y1 mod p
    const uint64_t *r2;   // y1 mod p^2
    const uint4 *pat8;
    const uint32_t *patsq;
    int16_t *Mloc;
    int32_t *segsum;
    int8_t *mu_out;
    uint64_t mu_base, mu_end;
    uint32_t extra_tx;    // bytes announced beyond the copy (0; tests of the bounded wait)
    // persistent kernel only
    const uint32_t *pw;   // p | w(p) << 24 for p < 2^17
    const uint32_t *gsq;  // square flags of primes >= 2048 over the block (one bit per y)
    uint64_t *bucket;     // per tile of the block: cap entries (p << 24 | w << 17 | offset)
    uint32_t *err;        // kErrBucket when a bucket overflows
};

// Small-prime job (p < 2048): the multiples of p in the tile offsets [lo, hi),
// lanes over them.  Its descriptor, made in the kernel's prologue, is
// {first multiple >= lo, hi, p | w(p) << 16, first multiple of p^2 >= lo or
// kNone when p^2 > tile (that single square is marked in the prologue)}.
// The step 32p is a multiple of 4, so each lane stays on one byte of its words
// and its shifted weight is loop-invariant.
constexpr uint32_t kNone = 0xffffffffu;
constexpr uint32_t kByteJobsMax = 512;  // 8 * 27 pieces (p < 128) + 278 primes below 2048

__device__ __forceinline__ void byte_small_job(uint4 d, uint32_t *w, uint32_t *sq, uint32_t lane)
{
    const uint32_t p = d.z & 0xffffu;
    const uint32_t yo = d.x + lane * p;
    const uint32_t wsh = (d.z >> 16) << ((yo & 3u) << 3);
    const uint32_t step = 8u * p;  // words per 32 multiples
    const uint32_t end = (d.y + 3u - (yo & 3u)) >> 2;  // yo' < hi  <=>  yo' >> 2 < end
#pragma unroll 4
    for (uint32_t wi = yo >> 2; wi < end; wi += step)
        atomicAdd(&w[wi], wsh);
    if (d.w != kNone) {
        const uint32_t p2 = p * p;  // <= tile
        for (uint32_t y2o = d.w + lane * p2; y2o < d.y; y2o += 32u * p2)
            atomicOr(&sq[y2o >> 5], 1u << (y2o & 31u));
    }
}

// Descriptor of small-prime job i (see above); *single is the one multiple of
// p^2 in the range when p^2 > tile, else kNone.
__device__ __forceinline__ uint4 byte_small_desc(const ByteArgs &a, uint32_t i, uint32_t jp,
                                                 uint32_t a0, uint32_t tl, uint32_t *single)
{
    uint32_t t, lo, hi;
    if (i < jp) {
        t = 4 + (i >> 3);
        lo = (i & 7u) * (kByteTile / 8);
        hi = min(tl, lo + kByteTile / 8);
    } else {
        t = a.np_piece + (i - jp);
        lo = 0;
        hi = tl;
    }
    *single = kNone;
    if (lo >= hi)
        return make_uint4(hi, hi, 11u, kNone);
    const uint4 q = a.pq[t];
    const uint32_t p = q.x;
    const uint32_t v = a.r[t] + a0 + lo;  // < 2^31
    const uint32_t rem = v - div_magic32(v, q.y, q.w & 255u) * p;
    const uint32_t p2 = p * p;
    const uint32_t v2 = (uint32_t)a.r2[t] + a0 + lo;  // < 2^31
    const uint32_t rem2 = v2 - div_magic32(v2, q.z, (q.w >> 8) & 255u) * p2;
    uint32_t s2 = lo + (rem2 ? p2 - rem2 : 0u);
    if (p2 > (uint32_t)kByteTile) {
        *single = s2 < hi ? s2 : kNone;
        s2 = kNone;
    }
    return make_uint4(lo + (rem ? p - rem : 0u), hi, p | ((q.w >> 16) << 16), s2);
}

// Hits of one prime p >= 2048 (one lane) over the whole tile; p^2 > tile, so
// at most one multiple of p^2.
__device__ __forceinline__ void byte_large_prime(uint4 q, uint32_t r, uint64_t r2, uint32_t *w,
                                                 uint32_t *sq, uint32_t a0, uint32_t tl)
{
    const uint32_t p = q.x;
    const uint32_t wt = q.w >> 16;
    const uint32_t v = r + a0;  // < 2^31
    const uint32_t rem = v - div_magic32(v, q.y, q.w & 255u) * p;
    for (uint32_t yo = rem ? p - rem : 0u; yo < tl; yo += p)
        atomicAdd(&w[yo >> 2], __funnelshift_l(0u, wt, yo << 3));
    uint64_t o2;
    if (q.z) {  // p^2 < 2^30: 32-bit division
        const uint32_t p2 = p * p;
        const uint32_t v2 = (uint32_t)r2 + a0;  // < 2^31
        const uint32_t rem2 = v2 - div_magic32(v2, q.z, (q.w >> 8) & 255u) * p2;
        o2 = rem2 ? p2 - rem2 : 0u;
    } else {  // p^2 >= 2^30 > a0: y1 mod p^2 + a0 < 2 p^2
        const uint64_t p2 = (uint64_t)p * p;
        uint64_t v2 = r2 + a0;
        if (v2 >= p2)
            v2 -= p2;
        o2 = v2 ? p2 - v2 : 0u;
    }
    if (o2 < tl)
        atomicOr(&sq[(uint32_t)o2 >> 5], 1u << ((uint32_t)o2 & 31u));
}

// floor(S log2 y - (S/2) log2 P) for one y (tiles below 2^26).
__device__ __forceinline__ int byte_thr(uint64_t y, float scale, float thr_half)
{
    return (int)floorf(scale * __log2f(__ull2float_rn(y)) - thr_half);
}

// Decode + scan of one byte-sieve tile (shared by the byte kernels): each warp
// owns two 2048-y segments, 16 y per lane per round (see the comment above
// ByteArgs for the decision rule).
__device__ __forceinline__ void byte_tile_decode(const ByteArgs &a, const uint4 *sb,
                                                 const uint32_t *sq, uint32_t a0, uint64_t t1,
                                                 uint32_t tl, uint32_t lane, uint32_t warp)
{
    const bool tile_thr = t1 >= kByteTileThrMin;
    uint32_t bias4 = 0;
    if (tile_thr) {
        int thr = (int)floorf(a.scale * log2f(__ull2float_rn(t1)) - a.thr_half);
        thr &= ~1;
        bias4 = (uint32_t)(127 - thr) * 0x01010101u;
    }
    for (uint32_t sgi = 0; sgi < 2; ++sgi) {
        const uint32_t so = warp * (2u * kSegY) + sgi * kSegY;  // segment start in the tile
        if (so >= tl)
            break;
        const uint64_t ys = t1 + so;
        const bool want_mu = a.mu_out && ys <= a.mu_end && ys + (kSegY - 1) >= a.mu_base;
        int run = 0;
#pragma unroll 1
        for (uint32_t r = 0; r < (uint32_t)kSegY / 512u; ++r) {
            const uint32_t o0 = so + r * 512u + lane * 16u;  // first of the lane's 16 y
            const uint4 q4 = sb[o0 >> 4];
            const uint32_t sqw = sq[o0 >> 5] >> (o0 & 16u);
            const uint32_t ws[4] = {q4.x, q4.y, q4.z, q4.w};
            uint32_t D[4], pbs[4], mbs[4];
            int tot = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                // square flag of byte j at bit 8j
                const uint32_t sqb = ((sqw >> (4 * k)) & 15u) * 0x00204081u;
                uint32_t neg;
                if (tile_thr) {
                    const uint32_t W = ws[k] + bias4;
                    neg = (W ^ (W >> 7)) & 0x01010101u;
                } else {
                    neg = 0;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint32_t A = (ws[k] >> (8 * j)) & 255u;
                        const int th = byte_thr(t1 + o0 + 4 * k + j, a.scale, a.thr_half);
                        // count parity xor [c > 1]
                        const uint32_t bit = (A & 1u) ^ ((int)A > th ? 0u : 1u);
                        neg |= bit << (8 * j);
                    }
                }
                uint32_t pb = ~sqb & ~neg & 0x01010101u;  // mu = +1
                uint32_t mb = ~sqb & neg;                 // mu = -1
                if (o0 + 4u * k + 4u > tl) {
                    const uint32_t keep = o0 + 4u * k >= tl ? 0u
                                          : 0xffffffffu >> (8u * (o0 + 4u * k + 4u - tl));
                    pb &= keep;
                    mb &= keep;
                }
                pbs[k] = pb;
                mbs[k] = mb;
                // byte j: 4 + sum of mu over bytes 0..j, in [0, 8]
                D[k] = (pb - mb + 0x01010101u) * 0x01010101u + 0x00010203u;
                tot += (int)(D[k] >> 24) - 4;
            }
            int inc = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int nb = __shfl_up_sync(0xffffffffu, inc, o);
                if ((int)lane >= o)
                    inc += nb;
            }
            int rb = run + inc - tot;  // M relative to the segment, before the lane's 16 y
            run += __shfl_sync(0xffffffffu, inc, 31);
            uint32_t out[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                // halfword = 0x8000 + value, so no borrow crosses halves; the
                // xor turns 0x8000 + v into v mod 2^16
                const uint32_t bx = (uint32_t)(rb - 4) * 0x00010001u;
                out[2 * k] = (bx + __byte_perm(D[k], 0x80u, 0x4140)) ^ 0x80008000u;
                out[2 * k + 1] = (bx + __byte_perm(D[k], 0x80u, 0x4342)) ^ 0x80008000u;
                rb += (int)(D[k] >> 24) - 4;
            }
            int16_t *dst = a.Mloc + a0 + o0;
            if (o0 + 16u <= tl) {
                reinterpret_cast<uint4 *>(dst)[0] = make_uint4(out[0], out[1], out[2], out[3]);
                reinterpret_cast<uint4 *>(dst)[1] = make_uint4(out[4], out[5], out[6], out[7]);
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (o0 + k < tl)
                        dst[k] = (int16_t)(out[k >> 1] >> (16 * (k & 1)));
            }
            if (want_mu) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const uint64_t y = t1 + o0 + k;
                    const uint32_t sh = 8u * (k & 3);
                    const int mu = (int)((pbs[k >> 2] >> sh) & 1u) - (int)((mbs[k >> 2] >> sh) & 1u);
                    if (o0 + k < tl && y >= a.mu_base && y <= a.mu_end)
                        a.mu_out[y - a.mu_base] = (int8_t)mu;
                }
            }
        }
        if (lane == 0)
            a.segsum[(a0 + so) >> kSegShift] = run;
    }
}

__global__ void __launch_bounds__(kSieveThreads, 1) mu_sieve_byte_kernel(ByteArgs a)
{
    extern __shared__ uint4 sb[];
    uint32_t *w = reinterpret_cast<uint32_t *>(sb);  // kByteWords words, four y each
    uint32_t *sq = w + kByteWords;                     // kByteSqWords words, 32 y each
    __shared__ uint32_t s_job;
    __shared__ uint4 s_jd[kByteJobsMax];
    __shared__ uint64_t s_mbar;
    const uint32_t a0 = blockIdx.x * (uint32_t)kByteTile;
    const uint64_t t1 = a.y1 + a0;
    const uint32_t tl = min(a.len - a0, (uint32_t)kByteTile);
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t jp = a.np_piece > 4 ? 8u * (a.np_piece - 4) : 0u;
    const uint32_t js = jp + (a.np_small - a.np_piece);  // small-prime jobs (<= kByteJobsMax)
    const uint32_t jobs = js + (a.np - a.np_small + 63u) / 64u;

    // prologue: small-prime job descriptors (a thread each), and the
    // pre-sieve pattern (bytes of 2, 3, 5, 7, square flags of 4, 9, 25, 49)
    uint32_t single = kNone;
    {
        // the tile's bytes: one bulk asynchronous copy of the pattern phase,
        // overlapped with the job descriptors and the square flags
        const uint32_t ph = (uint32_t)(t1 % kPatternPeriod);
        if (threadIdx.x == 0) {
            mbar_init(&s_mbar);
            fence_proxy_async_smem();
            mbar_arrive_expect(&s_mbar, (uint32_t)kByteTile + a.extra_tx);
            bulk_copy_g2s(sb, a.pat8 + (size_t)(ph & 15u) * (kPat8Len / 16) + (ph >> 4),
                          (uint32_t)kByteTile, &s_mbar);
            s_job = 0;
        }
        if (threadIdx.x < js)
            s_jd[threadIdx.x] = byte_small_desc(a, threadIdx.x, jp, a0, tl, &single);
        const uint32_t j0 = ph >> 5, s = ph & 31u;
        for (uint32_t i = threadIdx.x; i < (uint32_t)kByteSqWords; i += kSieveThreads)
            sq[i] = __funnelshift_r(a.patsq[j0 + i], a.patsq[j0 + i + 1], s);
    }
    __syncthreads();  // the mbarrier is initialised
    if (__syncthreads_or(!mbar_wait(&s_mbar, 0u))) {
        // the copy did not land in time: flag it, give it one more bounded
        // wait (it writes this CTA's shared memory), and leave the tile
        if (threadIdx.x == 0 && a.err)
            atomicOr(a.err, kErrTimeout);
        mbar_wait(&s_mbar, 0u);
        return;
    }
    if (single != kNone)
        atomicOr(&sq[single >> 5], 1u << (single & 31u));

    // jobs, largest first, handed out through a shared counter: small-prime
    // jobs (a warp over the multiples of one prime), then 64 primes >= 2048 at
    // a time (two per lane, the second one's loads in flight during the first)
    for (;;) {
        uint32_t job = 0;
        if (lane == 0)
            job = atomicAdd(&s_job, 1u);
        job = __shfl_sync(0xffffffffu, job, 0);
        if (job >= jobs)
            break;
        if (job < js) {
            byte_small_job(s_jd[job], w, sq, lane);
        } else {
            const uint32_t t0 = a.np_small + (job - js) * 64u + lane, t1p = t0 + 32u;
            uint4 q0 = make_uint4(0, 0, 0, 0), q1 = q0;
            uint32_t r0 = 0, r1 = 0;
            uint64_t r20 = 0, r21 = 0;
            if (t0 < a.np) {
                q0 = a.pq[t0];
                r0 = a.r[t0];
                r20 = a.r2[t0];
            }
            if (t1p < a.np) {
                q1 = a.pq[t1p];
                r1 = a.r[t1p];
                r21 = a.r2[t1p];
            }
            if (t0 < a.np)
                byte_large_prime(q0, r0, r20, w, sq, a0, tl);
            if (t1p < a.np)
                byte_large_prime(q1, r1, r21, w, sq, a0, tl);
        }
    }
    __syncthreads();

    byte_tile_decode(a, sb, sq, a0, t1, tl, lane, warp);
}

// ---------------------------------------------------------------------------
// a1 + a2, byte variant at weight scale 2 with the square flag in bit 7.
// Same method (Sec. 3 log sieve, then the prefix sum).  The byte of y holds
//     1 + sum over the distinct sieving primes p | y of w2(p),
// w2(p) the odd integer nearest 2 log2 p, plus 128 when a square of a
// sieving prime divides y.  The sum stays below 128 for y < 2^54
// (1 + 2 log2 y + E), so the square flag is set by atomicOr at any time and
// no add ever carries into it or out of the byte; the tile needs no separate
// square array, which lets two or three CTAs share an SM.
// Exactness: with A the weight sum, c = 1 gives A >= 2 log2 y - E and c > 1
// gives A <= 2 log2 y - 2 log2 P + E (E the summed rounding, at most the
// number of distinct prime factors), so the threshold T = 2 log2 y - log2 P
// separates them with log2 P - E units either side; the host takes this
// kernel only where that is at least 2.5, and then any integer threshold in
// [T - 2, T] is exact.  Tiles at y >= 2^26 take one even threshold thr per
// tile: W = (byte & 127) + 126 - thr puts A > thr into bit 7 of W and the
// count parity (xor 1) into bit 0, so mu = -1 exactly when they differ.
//
// Work of a tile:
//   * the pre-sieve pattern: primes 2, 3, 5, 7 with the base 1 and the flags
//     of 4, 9, 25, 49 (period 44100, one bulk asynchronous copy);
//   * primes 11 <= p < 1024: a warp over the multiples of one prime, largest
//     jobs first;
//   * primes p >= 1024: a lane per prime, four per lane, the hits of primes
//     below half the tile four at a time with loop-invariant shifted
//     weights; the square of a prime below 8192 per lane, those of larger
//     primes from a per-block list (at most sixteen multiples of p^2 per
//     prime in a block of up to 2^30 y).
// ---------------------------------------------------------------------------
struct T2Args {
    uint64_t y1;
    uint32_t len;          // <= 2^30
    uint32_t np;           // primes used (all p <= P)
    uint32_t np_lane;      // [4, np_lane): 11 <= p < 1024, a warp per prime
    uint32_t np_list;      // [np_list, np): p >= 8192, squares from the block's list
    float thr_half;        // log2 P
    const uint4 *pq;       // {p, m32(p), m32(p^2) or 0, s(p) | s(p^2) << 8 | w2(p) << 16}
    const uint4 *rec;      // per block, p >= 1024: {p, m32(p), y1 mod p, s(p) | w2(p) << 8}
    const uint2 *rec2;     // per block, 1024 <= p < 8192: {y1 mod p^2 | s(p^2) << 26, m32(p^2)}
    const uint32_t *r;     // y1 mod p
    const uint64_t *r2;    // y1 mod p^2
    const uint4 *pat;      // 16 phase copies of the 2, 3, 5, 7 pattern
    uint32_t *sqcnt;       // per tile: entries in the square list (cleared after use)
    const uint32_t *sqlist;// per tile: sqcap offsets of multiples of p^2, p >= 8192
    uint32_t sqcap;
    int16_t *Mloc;
    int32_t *segsum;
    int8_t *mu_out;
    uint64_t mu_base, mu_end;
    uint32_t extra_tx;     // bytes announced beyond the copy (0; tests of the bounded wait)
    uint32_t *err;         // kErrTimeout / kErrBucket
};

constexpr uint32_t kT2JobsMax = 192;          // descriptor jobs (168: the primes 11 .. 1021)
constexpr uint32_t kPat2Len = 142416;         // >= 44100 + 98304, multiple of 16
constexpr uint32_t kT2LaneMin = 1024;         // primes from here: a lane per prime
// a lane prime marks at most one multiple of its square per tile (98304 y)
static_assert(kT2LaneMin * kT2LaneMin > 98304u, "lane primes need p^2 above the tile");
constexpr uint32_t kT2ListMin = 8192;         // primes from here: squares from the list
constexpr uint64_t kT2MinTile = 65536;        // smallest tile (square-list scratch)
// Status bit: a bucket or a square list overflowed its capacity.
constexpr uint32_t kErrBucket = 4u;

// Per block: y1 mod p and y1 mod p^2 of every sieving prime, and the
// multiples of p^2 (p >= 8192, index >= list0) as offsets into per-tile lists.
__global__ void t2_block_prep_kernel(uint64_t y1, uint32_t np, const uint4 *__restrict__ pq,
                                     uint32_t *__restrict__ r, uint64_t *__restrict__ r2,
                                     uint32_t lane0, uint4 *__restrict__ rec,
                                     uint2 *__restrict__ rec2, uint32_t list0, uint32_t len,
                                     uint32_t tile, uint32_t *__restrict__ cnt,
                                     uint32_t *__restrict__ list, uint32_t cap,
                                     uint32_t *__restrict__ err)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np)
        return;
    const uint4 pr = pq[t];
    const uint64_t q = pr.x, q2 = q * q;
    const uint32_t rq = (uint32_t)(y1 % q);
    r[t] = rq;
    const uint64_t rem = y1 % q2;
    r2[t] = rem;
    if (t >= lane0) {
        rec[t] = make_uint4(pr.x, pr.y, rq, (pr.w & 255u) | ((pr.w >> 16) << 8));
        if (t < list0)  // q < 8192: q^2 < 2^26, its magic and shift
            rec2[t] = make_uint2((uint32_t)rem | (((pr.w >> 8) & 255u) << 26), pr.z);
    }
    if (t < list0)
        return;
    for (uint64_t o = rem ? q2 - rem : 0; o < len; o += q2) {
        const uint32_t ti = (uint32_t)(o / tile);
        const uint32_t slot = atomicAdd(&cnt[ti], 1u);
        if (slot < cap)
            list[(size_t)ti * cap + slot] = (uint32_t)(o - (uint64_t)ti * tile);
        else
            atomicOr(err, kErrBucket);
    }
}

// Descriptor job i of a tile of TILE y: {first multiple, tl, p | w2 << 16,
// first multiple of p^2 or kNone when p^2 > TILE}; *single = the one multiple
// of p^2 in the tile when p^2 > TILE.  Jobs: the primes 11 <= p < 1024 in
// order (index 4 + i), largest work first.
template <int TILE>
__device__ __forceinline__ uint4 t2_desc(const T2Args &a, uint32_t i, uint32_t a0,
                                         uint32_t tl, uint32_t *single)
{
    const uint32_t t = 4 + i, lo = 0, hi = tl;
    *single = kNone;
    const uint4 q = a.pq[t];
    const uint32_t p = q.x;
    const uint32_t v = a.r[t] + a0 + lo;  // < 2^31
    const uint32_t rem = v - div_magic32(v, q.y, q.w & 255u) * p;
    const uint32_t p2 = p * p;
    const uint32_t v2 = (uint32_t)a.r2[t] + a0 + lo;  // < 2^31
    const uint32_t rem2 = v2 - div_magic32(v2, q.z, (q.w >> 8) & 255u) * p2;
    uint32_t s2 = lo + (rem2 ? p2 - rem2 : 0u);
    if (p2 > (uint32_t)TILE) {
        *single = s2 < hi ? s2 : kNone;
        s2 = kNone;
    }
    return make_uint4(lo + (rem ? p - rem : 0u), hi, p | ((q.w >> 16) << 16), s2);
}

// Descriptor job: weights at the multiples of p in [first, hi), lanes over
// them (the step 32p is a multiple of 4, so a lane's shifted weight is
// loop-invariant; unrolled by hand, so no trip count is divided out), then
// the square flags at the multiples of p^2.
__device__ __forceinline__ void t2_desc_job(uint4 d, uint32_t *w, uint32_t lane)
{
    const uint32_t p = d.z & 0xffffu;
    const uint32_t yo = d.x + lane * p;
    if (yo < d.y) {
        const uint32_t wsh = (d.z >> 16) << ((yo & 3u) << 3);
        const uint32_t step = 8u * p;                      // words per 32 multiples
        const uint32_t end = (d.y + 3u - (yo & 3u)) >> 2;  // yo' < hi  <=>  yo' >> 2 < end
        uint32_t wi = yo >> 2;
        for (; wi + 3u * step < end; wi += 4u * step) {
            atomicAdd(&w[wi], wsh);
            atomicAdd(&w[wi + step], wsh);
            atomicAdd(&w[wi + 2u * step], wsh);
            atomicAdd(&w[wi + 3u * step], wsh);
        }
        for (; wi < end; wi += step)
            atomicAdd(&w[wi], wsh);
    }
    if (d.w != kNone) {
        const uint32_t p2 = p * p;
        for (uint32_t y2o = d.w + lane * p2; y2o < d.y; y2o += 32u * p2)
            atomicOr(&w[y2o >> 2], 0x80u << ((y2o & 3u) << 3));
    }
}

// One prime p >= 1024 over the whole tile (one lane): its weights, and its
// square when p < 8192 (p^2 > tile: at most one multiple).  Its per-block
// record q = {p, m32(p), y1 mod p, s(p) | w2(p) << 8} and, below 8192,
// e = {y1 mod p^2 | s(p^2) << 26, m32(p^2)} (see t2_block_prep_kernel).
template <int TILE>
__device__ __forceinline__ void t2_lane_prime(uint4 q, uint2 e, uint32_t *w, uint32_t a0,
                                              uint32_t tl)
{
    const uint32_t p = q.x;
    const uint32_t wt = q.w >> 8;
    const uint32_t v = q.z + a0;  // < 2^31
    const uint32_t rem = v - div_magic32(v, q.y, q.w & 255u) * p;
    uint32_t yo = rem ? p - rem : 0u;
    if (p < (uint32_t)TILE / 2u) {
        // four hits per round: p is odd, so the four byte positions of
        // yo, yo+p, yo+2p, yo+3p repeat every 4p
        const uint32_t w0 = wt << ((yo & 3u) << 3);
        const uint32_t w1 = wt << (((yo + p) & 3u) << 3);
        const uint32_t w2 = wt << (((yo + 2u * p) & 3u) << 3);
        const uint32_t w3 = wt << (((yo + 3u * p) & 3u) << 3);
        for (; yo + 3u * p < tl; yo += 4u * p) {
            atomicAdd(&w[yo >> 2], w0);
            atomicAdd(&w[(yo + p) >> 2], w1);
            atomicAdd(&w[(yo + 2u * p) >> 2], w2);
            atomicAdd(&w[(yo + 3u * p) >> 2], w3);
        }
        if (yo < tl) {
            atomicAdd(&w[yo >> 2], w0);
            if (yo + p < tl) {
                atomicAdd(&w[(yo + p) >> 2], w1);
                if (yo + 2u * p < tl)
                    atomicAdd(&w[(yo + 2u * p) >> 2], w2);
            }
        }
    } else if (p < (uint32_t)TILE) {
        for (; yo < tl; yo += p)
            atomicAdd(&w[yo >> 2], __funnelshift_l(0u, wt, yo << 3));
    } else if (yo < tl) {
        atomicAdd(&w[yo >> 2], __funnelshift_l(0u, wt, yo << 3));  // at most one multiple
    }
    if (p < kT2ListMin) {
        // p^2 < 2^26: the first multiple of p^2 at or after the tile start;
        // e.y = m32(p^2), its shift below 32 in the low bits of e.x's spare
        // room is not needed: y1 mod p^2 < 2^26 leaves e.x bits 26..31 for it
        const uint32_t p2 = p * p;
        const uint32_t v2 = (e.x & 0x3ffffffu) + a0;  // < 2^31
        const uint32_t rem2 = v2 - div_magic32(v2, e.y, e.x >> 26) * p2;
        const uint32_t o2 = rem2 ? p2 - rem2 : 0u;
        if (o2 < tl)
            atomicOr(&w[o2 >> 2], 0x80u << ((o2 & 3u) << 3));
    }
}

// mu of four y (one word of the tile) as the prefix word
//     D = byte j: 4 + sum of mu over bytes 0..j,
// from the square flags (bit 7 of each byte) and, with a tile threshold, the
// biased bytes W = (byte & 127) + bias: with nsq = 1 where no square divides
// and m = 1 where mu = -1 (nsq and bit 0 xor bit 7 of W), mu + 1 = 1 + nsq -
// 2m per byte, so D = (nsq - 2m) 0x01010101 + 0x04040404 (mod 2^32).  keep
// masks the bytes past the tile's end (mu = 0 there).
__device__ __forceinline__ uint32_t t2_word(uint32_t ws, uint32_t bias4, uint32_t keep,
                                            bool tile_thr, uint64_t y0, float thr_half,
                                            uint32_t *nsq_out, uint32_t *m_out)
{
    const uint32_t nsq = ~(ws >> 7) & 0x01010101u & keep;
    uint32_t m;
    if (tile_thr) {
        const uint32_t W = (ws & 0x7f7f7f7fu) + bias4;
        m = (W ^ (W >> 7)) & nsq;
    } else {
        m = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int A = (int)((ws >> (8 * j)) & 127u) - 1;
            const int th = (int)floorf(2.0f * __log2f(__ull2float_rn(y0 + j)) - thr_half);
            // count parity xor [c > 1]
            const uint32_t bit = ((uint32_t)A & 1u) ^ (A > th ? 0u : 1u);
            m |= bit << (8 * j);
        }
        m &= nsq;
    }
    *nsq_out = nsq;
    *m_out = m;
    return (nsq - 2u * m) * 0x01010101u + 0x04040404u;
}

// Decode + scan of one 2048-y segment of a scale-2 tile (one warp): a round
// covers 1024 y, each lane 16 y at 16 lane and 16 y at 512 + 16 lane (16-byte
// shared loads without bank conflicts), and one warp scan carries both
// halves' lane sums packed in one int32 (low and high 16-bit fields; every
// partial sum is within +-512).  kFast: the segment is whole, the tile takes
// one threshold and no mu is written, so none of the checks for those cases
// is issued.  Returns the segment's mu sum.
template <bool kFast>
__device__ int t2_segment(const T2Args &a, const uint4 *sb, uint32_t a0,
                          uint64_t t1, uint32_t tl, uint32_t so, uint32_t lane, uint32_t bias4,
                          bool tile_thr, bool want_mu)
{
    int run = 0;
#pragma unroll 1
    for (uint32_t r = 0; r < (uint32_t)kSegY / 1024u; ++r) {
        uint32_t D[8];
        int tot[2] = {0, 0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t o0 = so + r * 1024u + (uint32_t)h * 512u + lane * 16u;
            const uint4 q4 = sb[o0 >> 4];
            const uint32_t ws[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t ok = o0 + 4u * k;
                uint32_t nsq, m;
                if (kFast) {
                    nsq = ~(ws[k] >> 7) & 0x01010101u;
                    const uint32_t W = (ws[k] & 0x7f7f7f7fu) + bias4;
                    m = (W ^ (W >> 7)) & nsq;
                    D[4 * h + k] = (nsq - 2u * m) * 0x01010101u + 0x04040404u;
                } else {
                    const uint32_t keep =
                        ok + 4u <= tl ? 0xffffffffu
                                      : (ok >= tl ? 0u : 0xffffffffu >> (8u * (ok + 4u - tl)));
                    D[4 * h + k] = t2_word(ws[k], bias4, keep, tile_thr, t1 + ok, a.thr_half,
                                           &nsq, &m);
                    if (want_mu) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint64_t y = t1 + ok + j;
                            const int mu = (int)((nsq >> (8 * j)) & 1u) -
                                           2 * (int)((m >> (8 * j)) & 1u);
                            if (ok + j < tl && y >= a.mu_base && y <= a.mu_end)
                                a.mu_out[y - a.mu_base] = (int8_t)mu;
                        }
                    }
                }
                tot[h] += (int)(D[4 * h + k] >> 24) - 4;
            }
        }
        // packed inclusive scan of (tot[0], tot[1]) over the lanes
        int inc = tot[0] + tot[1] * 65536;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int nb = __shfl_up_sync(0xffffffffu, inc, o);
            if ((int)lane >= o)
                inc += nb;
        }
        const int all = __shfl_sync(0xffffffffu, inc, 31);
        const int incA = (int)(int16_t)(inc & 0xffff), incB = (inc - incA) >> 16;
        const int allA = (int)(int16_t)(all & 0xffff), allB = (all - allA) >> 16;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t o0 = so + r * 1024u + (uint32_t)h * 512u + lane * 16u;
            // M relative to the segment, before the lane's 16 y
            int rb = run + (h == 0 ? incA - tot[0] : allA + incB - tot[1]);
            uint32_t out[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t Dk = D[4 * h + k];
                // halfword = 0x8000 + value, so no borrow crosses halves; the
                // xor turns 0x8000 + v into v mod 2^16
                const uint32_t bx = (uint32_t)(rb - 4) * 0x00010001u;
                out[2 * k] = (bx + __byte_perm(Dk, 0x80u, 0x4140)) ^ 0x80008000u;
                out[2 * k + 1] = (bx + __byte_perm(Dk, 0x80u, 0x4342)) ^ 0x80008000u;
                rb += (int)(Dk >> 24) - 4;
            }
            int16_t *dst = a.Mloc + a0 + o0;
            if (kFast || o0 + 16u <= tl) {
                reinterpret_cast<uint4 *>(dst)[0] = make_uint4(out[0], out[1], out[2], out[3]);
                reinterpret_cast<uint4 *>(dst)[1] = make_uint4(out[4], out[5], out[6], out[7]);
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (o0 + k < tl)
                        dst[k] = (int16_t)(out[k >> 1] >> (16 * (k & 1)));
            }
        }
        run += allA + allB;
    }
    return run;
}

__device__ __forceinline__ int t2_segment_fast(const T2Args &a, const uint4 *sb, uint32_t a0,
                                               uint64_t t1, uint32_t tl, uint32_t so,
                                               uint32_t lane, uint32_t bias4)
{
    return t2_segment<true>(a, sb, a0, t1, tl, so, lane, bias4, true, false);
}

// The rare segments (a ragged end, thresholds per y, mu written) in a
// function of their own, so they hold no registers of the common path.
__device__ __noinline__ int t2_segment_general(const T2Args &a, const uint4 *sb, uint32_t a0,
                                               uint64_t t1, uint32_t tl, uint32_t so,
                                               uint32_t lane, uint32_t bias4, bool tile_thr,
                                               bool want_mu)
{
    return t2_segment<false>(a, sb, a0, t1, tl, so, lane, bias4, tile_thr, want_mu);
}

// Decode + scan of one scale-2 tile: each warp owns two 2048-y segments.
__device__ __forceinline__ void t2_tile_decode(const T2Args &a, const uint4 *sb, uint32_t a0,
                                               uint64_t t1, uint32_t tl, uint32_t lane,
                                               uint32_t warp)
{
    const bool tile_thr = t1 >= kByteTileThrMin;
    uint32_t bias4 = 0;
    if (tile_thr) {
        int thr = (int)floorf(2.0f * log2f(__ull2float_rn(t1)) - a.thr_half);
        thr &= ~1;
        bias4 = (uint32_t)(126 - thr) * 0x01010101u;
    }
    for (uint32_t sgi = 0; sgi < 2; ++sgi) {
        const uint32_t so = warp * (2u * kSegY) + sgi * kSegY;  // segment start in the tile
        if (so >= tl)
            break;
        const uint64_t ys = t1 + so;
        const bool want_mu = a.mu_out && ys <= a.mu_end && ys + (kSegY - 1) >= a.mu_base;
        const int run = (tile_thr && !want_mu && so + kSegY <= tl)
                            ? t2_segment_fast(a, sb, a0, t1, tl, so, lane, bias4)
                            : t2_segment_general(a, sb, a0, t1, tl, so, lane, bias4, tile_thr,
                                                 want_mu);
        if (lane == 0)
            a.segsum[(a0 + so) >> kSegShift] = run;
    }
}

template <int TILE, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) mu_sieve_t2_kernel(T2Args a)
{
    static_assert(TILE == THREADS * 128, "each warp decodes two 2048-y segments");
    static_assert(THREADS >= (int)kT2JobsMax, "one descriptor per thread");
    extern __shared__ uint4 sb[];
    uint32_t *w = reinterpret_cast<uint32_t *>(sb);  // TILE / 4 words, four y each
    __shared__ uint32_t s_job;
    __shared__ uint4 s_jd[kT2JobsMax];
    __shared__ uint64_t s_mbar;
    const uint32_t a0 = blockIdx.x * (uint32_t)TILE;
    const uint64_t t1 = a.y1 + a0;
    const uint32_t tl = min(a.len - a0, (uint32_t)TILE);
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t jd = a.np_lane - 4;  // descriptor jobs: primes 11 <= p < 1024
    const uint32_t jobs = jd + (a.np - a.np_lane + 127u) / 128u;
    const uint32_t nsq = min(a.sqcnt[blockIdx.x], a.sqcap);

    uint32_t single = kNone;
    {
        // the tile's bytes: one bulk asynchronous copy of the first pattern's
        // phase, overlapped with the job descriptors
        const uint32_t ph = (uint32_t)(t1 % kPatternPeriod);
        if (threadIdx.x == 0) {
            mbar_init(&s_mbar);
            fence_proxy_async_smem();
            mbar_arrive_expect(&s_mbar, (uint32_t)TILE + a.extra_tx);
            bulk_copy_g2s(sb, a.pat + (size_t)(ph & 15u) * (kPat2Len / 16) + (ph >> 4),
                          (uint32_t)TILE, &s_mbar);
            s_job = 0;
        }
        if (threadIdx.x < jd)
            s_jd[threadIdx.x] = t2_desc<TILE>(a, threadIdx.x, a0, tl, &single);
    }
    __syncthreads();  // the mbarrier is initialised; every thread has read sqcnt
    if (__syncthreads_or(!mbar_wait(&s_mbar, 0u))) {
        // the copy did not land in time: flag it, give it one more bounded
        // wait (it writes this CTA's shared memory), and leave the tile
        if (threadIdx.x == 0) {
            a.sqcnt[blockIdx.x] = 0;
            if (a.err)
                atomicOr(a.err, kErrTimeout);
        }
        mbar_wait(&s_mbar, 0u);
        return;
    }
    if (threadIdx.x == 0)
        a.sqcnt[blockIdx.x] = 0;  // read above; cleared for the next block
    if (single != kNone)
        atomicOr(&w[single >> 2], 0x80u << ((single & 3u) << 3));
    {
        const uint32_t *ls = a.sqlist + (size_t)blockIdx.x * a.sqcap;
        for (uint32_t i = threadIdx.x; i < nsq; i += THREADS) {
            const uint32_t o = ls[i];
            atomicOr(&w[o >> 2], 0x80u << ((o & 3u) << 3));
        }
    }

    // jobs, largest first, handed out through a shared counter: descriptor
    // jobs (a warp over the multiples of one prime), then 128 primes >= 1024
    // at a time (a lane takes primes i and 63 - i of each half of the job, so
    // the lanes' hit counts even out)
    for (;;) {
        uint32_t job = 0;
        if (lane == 0)
            job = atomicAdd(&s_job, 1u);
        job = __shfl_sync(0xffffffffu, job, 0);
        if (job >= jobs)
            break;
        if (job < jd) {
            t2_desc_job(s_jd[job], w, lane);
        } else {
            for (uint32_t hb = 0; hb < 128u; hb += 64u) {
            const uint32_t b0 = a.np_lane + (job - jd) * 128u + hb;
            const uint32_t t0 = b0 + lane, t1p = b0 + 63u - lane;
            uint4 q0 = make_uint4(0, 0, 0, 0), q1 = q0;
            uint2 e0 = make_uint2(0, 0), e1 = e0;
            if (t0 < a.np) {
                q0 = a.rec[t0];
                if (t0 < a.np_list)
                    e0 = a.rec2[t0];
            }
            if (t1p < a.np) {
                q1 = a.rec[t1p];
                if (t1p < a.np_list)
                    e1 = a.rec2[t1p];
            }
            if (t0 < a.np)
                t2_lane_prime<TILE>(q0, e0, w, a0, tl);
            if (t1p < a.np)
                t2_lane_prime<TILE>(q1, e1, w, a0, tl);
            }
        }
    }
    __syncthreads();

    t2_tile_decode(a, sb, a0, t1, tl, lane, warp);
}

// ---------------------------------------------------------------------------
// a1 + a2, persistent byte variant for blocks with many large primes.  One
// CTA per SM takes a contiguous range of tiles of the block and keeps, across
// its tiles:
//   * for every prime 2048 <= p < 2^17 (at most two tiles' worth of hits per
//     tile), the offset of its next multiple, in shared memory -- no division
//     per (prime, tile);
//   * for every prime p >= 2^17 (at most one hit per tile), a bucket entry in
//     the tile of its next multiple (Oliveira e Silva's bucket sieve, here per
//     CTA): a tile visits only the primes that hit it and forwards each to the
//     tile of its next multiple.
// Multiples of p^2 for p >= 2048 come from a bit array over the block made by
// square_bits_kernel; primes below 2048 are set up per tile as in the byte
// kernel.  The tile's bytes, decode and scan are those of the byte kernel.
// ---------------------------------------------------------------------------
constexpr uint32_t kMedMax = 12288;          // primes in [2048, 2^17): 11942
constexpr uint32_t kPersistTilesMax = 128;   // tiles per CTA (blocks <= 2^30 y, >= 64 CTAs)
constexpr uint32_t kBucketJob = 256;         // bucket entries per job (8 per lane)

__device__ __forceinline__ uint64_t bucket_entry(uint32_t p, uint32_t w, uint32_t off)
{
    return ((uint64_t)p << 24) | ((uint64_t)w << 17) | off;
}

// Bits of y (offset from the block start) with q^2 | y for a prime
// 2048 <= q <= P: one thread per prime walks its square multiples.
__global__ void square_bits_kernel(uint32_t len, uint32_t p0, uint32_t np,
                                   const uint32_t *__restrict__ p, const uint64_t *__restrict__ r2,
                                   uint32_t *__restrict__ bits)
{
    const uint32_t t = p0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np)
        return;
    const uint64_t q = p[t], q2 = q * q;
    const uint64_t rem = r2[t];
    for (uint64_t o = rem ? q2 - rem : 0; o < len; o += q2)
        atomicOr(&bits[o >> 5], 1u << (o & 31u));
}

__global__ void __launch_bounds__(kSieveThreads, 1) mu_sieve_persist_kernel(ByteArgs a)
{
    extern __shared__ uint4 sb[];
    uint32_t *w = reinterpret_cast<uint32_t *>(sb);  // kByteWords words, four y each
    uint32_t *sq = w + kByteWords;                     // kByteSqWords words, 32 y each
    uint32_t *moff = sq + kByteSqWords;                // kMedMax next offsets
    __shared__ uint32_t s_job;
    __shared__ uint4 s_jd[kByteJobsMax];
    __shared__ uint32_t s_cnt[kPersistTilesMax];
    __shared__ uint64_t s_mbar;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t ntiles = (a.len + kByteTile - 1) / kByteTile;
    const uint32_t tb = (uint32_t)((uint64_t)blockIdx.x * ntiles / gridDim.x);
    const uint32_t te = (uint32_t)((uint64_t)(blockIdx.x + 1) * ntiles / gridDim.x);
    const uint32_t T = te - tb;  // tiles of this CTA (the host keeps it <= kPersistTilesMax)
    if (T == 0)
        return;
    const uint32_t A0 = tb * (uint32_t)kByteTile;
    const uint32_t nmed = a.np_mid - a.np_small;

    // CTA prologue: next multiple of every medium prime, buckets of the large
    for (uint32_t i = threadIdx.x; i < kPersistTilesMax; i += kSieveThreads)
        s_cnt[i] = 0;
    if (threadIdx.x == 0) {
        mbar_init(&s_mbar);
        fence_proxy_async_smem();
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nmed; i += kSieveThreads) {
        const uint32_t t = a.np_small + i;
        const uint4 q = a.pq[t];
        const uint32_t v = a.r[t] + A0;  // < 2^31
        const uint32_t rem = v - div_magic32(v, q.y, q.w & 255u) * q.x;
        moff[i] = rem ? q.x - rem : 0u;
    }
    for (uint32_t t = a.np_mid + threadIdx.x; t < a.np; t += kSieveThreads) {
        const uint4 q = a.pq[t];
        const uint32_t v = a.r[t] + A0;  // < 2^31
        const uint32_t rem = v - div_magic32(v, q.y, q.w & 255u) * q.x;
        const uint32_t off = rem ? q.x - rem : 0u;  // < p < 2^27
        const uint32_t tr = off >> 17;
        if (tr < T) {
            const uint32_t slot = atomicAdd(&s_cnt[tr], 1u);
            if (slot < a.cap)
                a.bucket[(size_t)(tb + tr) * a.cap + slot] =
                    bucket_entry(q.x, q.w >> 16, off & (kByteTile - 1));
            else
                atomicOr(a.err, kErrBucket);
        }
    }
    __syncthreads();

    const uint32_t jp = a.np_piece > 4 ? 8u * (a.np_piece - 4) : 0u;
    const uint32_t js = jp + (a.np_small - a.np_piece);  // small-prime jobs
    const uint32_t jm = js + (nmed + 63u) / 64u;          // + medium jobs (64 primes)
    for (uint32_t tt = 0; tt < T; ++tt) {
        const uint32_t a0 = A0 + tt * (uint32_t)kByteTile;
        const uint64_t t1 = a.y1 + a0;
        const uint32_t tl = min(a.len - a0, (uint32_t)kByteTile);
        const uint32_t nb = min(s_cnt[tt], a.cap);  // final: appends go to later tiles
        const uint32_t jobs = jm + (nb + kBucketJob - 1) / kBucketJob;
        uint32_t single = kNone;
        {
            // bulk copy of the tile's pattern bytes (the previous tile's
            // readers are past the barrier that ended it), overlapped with
            // the descriptors and the square flags
            const uint32_t ph = (uint32_t)(t1 % kPatternPeriod);
            if (threadIdx.x == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect(&s_mbar, (uint32_t)kByteTile + a.extra_tx);
                bulk_copy_g2s(sb, a.pat8 + (size_t)(ph & 15u) * (kPat8Len / 16) + (ph >> 4),
                              (uint32_t)kByteTile, &s_mbar);
                s_job = 0;
            }
            if (threadIdx.x < js)
                s_jd[threadIdx.x] = byte_small_desc(a, threadIdx.x, jp, a0, tl, &single);
            const uint32_t j0 = ph >> 5, sh = ph & 31u;
            const uint32_t *gs = a.gsq + (a0 >> 5);
            for (uint32_t i = threadIdx.x; i < (uint32_t)kByteSqWords; i += kSieveThreads)
                sq[i] = __funnelshift_r(a.patsq[j0 + i], a.patsq[j0 + i + 1], sh) | gs[i];
        }
        if (__syncthreads_or(!mbar_wait(&s_mbar, tt & 1u))) {
            if (threadIdx.x == 0)
                atomicOr(a.err, kErrTimeout);
            mbar_wait(&s_mbar, tt & 1u);
            return;
        }
        if (single != kNone)
            atomicOr(&sq[single >> 5], 1u << (single & 31u));
        for (;;) {
            uint32_t job = 0;
            if (lane == 0)
                job = atomicAdd(&s_job, 1u);
            job = __shfl_sync(0xffffffffu, job, 0);
            if (job >= jobs)
                break;
            if (job < js) {
                byte_small_job(s_jd[job], w, sq, lane);
            } else if (job < jm) {
                // 64 medium primes, two per lane, both loads issued first;
                // offsets carried in shared memory
                const uint32_t i0 = (job - js) * 64u + lane, i1 = i0 + 32u;
                const uint32_t pw0 = i0 < nmed ? a.pw[a.np_small + i0] : 0u;
                const uint32_t pw1 = i1 < nmed ? a.pw[a.np_small + i1] : 0u;
                uint32_t o0 = i0 < nmed ? moff[i0] : 0xffffffffu;
                uint32_t o1 = i1 < nmed ? moff[i1] : 0xffffffffu;
                if (i0 < nmed) {
                    const uint32_t p = pw0 & 0xffffffu, wt = pw0 >> 24;
                    for (; o0 < tl; o0 += p)
                        atomicAdd(&w[o0 >> 2], __funnelshift_l(0u, wt, o0 << 3));
                    moff[i0] = o0 - (uint32_t)kByteTile;
                }
                if (i1 < nmed) {
                    const uint32_t p = pw1 & 0xffffffu, wt = pw1 >> 24;
                    for (; o1 < tl; o1 += p)
                        atomicAdd(&w[o1 >> 2], __funnelshift_l(0u, wt, o1 << 3));
                    moff[i1] = o1 - (uint32_t)kByteTile;
                }
            } else {
                // bucket entries of this tile: mark, forward to the tile of the
                // next multiple (warp-aggregated slot allocation)
                const uint32_t e0 = (job - jm) * kBucketJob;
                uint64_t *bk = a.bucket + (size_t)(tb + tt) * a.cap;
#pragma unroll 1
                for (uint32_t k = 0; k < kBucketJob / 32u; ++k) {
                    const uint32_t e = e0 + k * 32u + lane;
                    uint32_t nt = 0xffffffffu, fwd = 0;
                    uint64_t ent = 0;
                    if (e < nb) {
                        ent = bk[e];
                        const uint32_t off = (uint32_t)ent & (kByteTile - 1);
                        const uint32_t wt = (uint32_t)(ent >> 17) & 127u;
                        const uint32_t p = (uint32_t)(ent >> 24);
                        atomicAdd(&w[off >> 2], __funnelshift_l(0u, wt, off << 3));
                        const uint32_t nx = off + p;
                        if (tt + (nx >> 17) < T) {
                            nt = tt + (nx >> 17);
                            fwd = nx & (kByteTile - 1);
                        }
                    }
                    const uint32_t peers = __match_any_sync(0xffffffffu, nt);
                    if (nt != 0xffffffffu) {
                        const uint32_t leader = __ffs(peers) - 1u;
                        uint32_t base = 0;
                        if (lane == leader)
                            base = atomicAdd(&s_cnt[nt], (uint32_t)__popc(peers));
                        base = __shfl_sync(peers, base, leader);
                        const uint32_t slot = base + __popc(peers & ((1u << lane) - 1u));
                        if (slot < a.cap)
                            a.bucket[(size_t)(tb + nt) * a.cap + slot] =
                                (ent & ~(uint64_t)(kByteTile - 1)) | fwd;
                        else
                            atomicOr(a.err, kErrBucket);
                    }
                }
            }
        }
        __syncthreads();
        byte_tile_decode(a, sb, sq, a0, t1, tl, lane, warp);
        __syncthreads();  // the next tile reuses the shared arrays
    }
}

// a2 finish: segoff[s] = carry_in + sum of segsum[0..s) (int64), and
// carry_out = carry_in + all of them.  Each CTA scans 1024 segments and adds
// the sum of all segments before its range.
__global__ void __launch_bounds__(1024) seg_carry_kernel(const int32_t *__restrict__ segsum,
                                                         uint32_t nseg,
                                                         const int64_t *__restrict__ carry_in,
                                                         int64_t *__restrict__ segoff,
                                                         int64_t *__restrict__ carry_out)
{
    __shared__ int64_t sh[33];
    const uint32_t base = blockIdx.x * 1024u;
    int64_t before = 0;
    for (uint32_t i = threadIdx.x; i < base; i += 1024u)
        before += segsum[i];
    int64_t tb;
    block_excl_scan<int64_t>(before, sh, &tb);
    const uint32_t i = base + threadIdx.x;
    const int64_t v = i < nseg ? segsum[i] : 0;
    int64_t tot;
    const int64_t ex = block_excl_scan<int64_t>(v, sh, &tot);
    const int64_t c0 = *carry_in;
    if (i < nseg)
        segoff[i] = c0 + tb + ex;
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        *carry_out = c0 + tb + tot;
}

__global__ void expand_M_kernel(const int16_t *__restrict__ Mloc, const int64_t *__restrict__ segoff,
                                uint64_t len, int32_t *__restrict__ M, uint32_t *__restrict__ err)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const int64_t v = segoff[i >> kSegShift] + Mloc[i];
        if (v > INT32_MAX || v < INT32_MIN)
            atomicOr(err, kErrMOverflow);
        M[i] = (int32_t)v;
    }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
static std::vector<uint32_t> host_primes(uint64_t B)
{
    std::vector<uint8_t> comp(B + 1, 0);
    std::vector<uint32_t> out;
    for (uint64_t i = 2; i <= B; ++i) {
        if (comp[i])
            continue;
        out.push_back((uint32_t)i);
        for (uint64_t j = i * i; j <= B; j += i)
            comp[j] = 1;
    }
    return out;
}

static uint64_t isqrt_u64(uint64_t v)
{
    uint64_t r = (uint64_t)std::sqrt((double)v);
    while (r > 0 && r > v / r)
        --r;
    while ((r + 1) <= v / (r + 1))
        ++r;
    return r;
}

// Odd integer nearest S log2 p (ties upward).
static uint32_t byte_weight(uint32_t p, uint32_t S)
{
    const double x = S * std::log2((double)p);
    return 2u * (uint32_t)std::floor((x - 1.0) / 2.0 + 0.5) + 1u;
}

// Host copies of the byte sieve's pre-sieve tables for weight scale S (they
// depend on S only): built once per process and kept.
struct BytePatterns {
    std::vector<uint8_t> p8;     // 16 phase copies of the 2, 3, 5, 7 byte pattern
    std::vector<uint32_t> psq;   // square flags of 4, 9, 25, 49 as a bit string
};

static const BytePatterns &byte_patterns(uint32_t S)
{
    static std::mutex mu;
    static BytePatterns cache[5];
    std::lock_guard<std::mutex> lk(mu);
    BytePatterns &bp = cache[S < 5 ? S : 4];
    if (!bp.p8.empty())
        return bp;
    uint32_t w[4];
    const uint32_t small[4] = {2, 3, 5, 7};
    for (int q = 0; q < 4; ++q)
        w[q] = byte_weight(small[q], S);
    std::vector<uint8_t> pat(kPatternPeriod);
    std::vector<uint8_t> sqp(kPatternPeriod);
    for (uint32_t i = 0; i < kPatternPeriod; ++i) {
        uint32_t b = 0, f = 0;
        for (int q = 0; q < 4; ++q) {
            if (i % small[q] == 0)
                b += w[q];
            if (i % (small[q] * small[q]) == 0)
                f = 1;
        }
        pat[i] = (uint8_t)b;
        sqp[i] = (uint8_t)f;
    }
    bp.p8.resize((size_t)16 * kPat8Len);
    for (uint32_t k = 0; k < 16; ++k)
        for (uint32_t j = 0; j < kPat8Len; ++j)
            bp.p8[(size_t)k * kPat8Len + j] = pat[(k + j) % kPatternPeriod];
    bp.psq.assign(kPatSqWords, 0u);
    for (uint32_t j = 0; j < 32u * kPatSqWords; ++j)
        if (sqp[j % kPatternPeriod])
            bp.psq[j >> 5] |= 1u << (j & 31u);
    return bp;
}

// Host copy of the scale-2 byte pattern (see mu_sieve_t2_kernel), 16 phase
// copies (copy k starts at phase k), built once per process: 1 + the weights
// of 2, 3, 5, 7, plus 128 where 4, 9, 25 or 49 divides (period 44100).
struct T2Patterns {
    std::vector<uint8_t> a;
};

static const T2Patterns &t2_patterns()
{
    static std::mutex mu;
    static T2Patterns tp;
    std::lock_guard<std::mutex> lk(mu);
    if (!tp.a.empty())
        return tp;
    const uint32_t small[4] = {2, 3, 5, 7};
    std::vector<uint8_t> pat(kPatternPeriod);
    for (uint32_t i = 0; i < kPatternPeriod; ++i) {
        uint32_t b = 1;
        for (int q = 0; q < 4; ++q) {
            if (i % small[q] == 0)
                b += byte_weight(small[q], 2);
            if (i % (small[q] * small[q]) == 0)
                b |= 128u;
        }
        pat[i] = (uint8_t)b;
    }
    tp.a.resize((size_t)16 * kPat2Len);
    for (uint32_t k = 0; k < 16; ++k)
        for (uint32_t j = 0; j < kPat2Len; ++j)
            tp.a[(size_t)k * kPat2Len + j] = pat[(k + j) % kPatternPeriod];
    return tp;
}

// Tables of the byte sieve (see mu_sieve_byte_kernel).
static int byte_tables_create(PrimeTable *t, const std::vector<uint32_t> &pr, cudaStream_t s)
{
    const size_t np = pr.size();
    std::vector<uint4> pq(np);
    for (size_t i = 0; i < np; ++i) {
        const uint32_t p = pr[i];
        unsigned s1 = 0, s2 = 0;
        const uint32_t m1 = magic32_of(p, &s1);
        const uint64_t p2 = (uint64_t)p * p;
        const uint32_t m2 = p2 < (1ull << 30) ? magic32_of((uint32_t)p2, &s2) : 0u;
        pq[i] = make_uint4(p, m1, m2, s1 | (s2 << 8) | (byte_weight(p, t->byte_scale) << 16));
    }
    const BytePatterns &bp = byte_patterns(t->byte_scale);
    const std::vector<uint8_t> &p8 = bp.p8;
    const std::vector<uint32_t> &psq = bp.psq;
    // p | w << 24 for the primes below 2^17
    uint32_t nmid = 0;
    while (nmid < np && pr[nmid] < (1u << 17))
        ++nmid;
    t->np_mid = nmid;
    std::vector<uint32_t> pwv(nmid + 1, 0u);
    for (uint32_t i = 0; i < nmid; ++i)
        pwv[i] = pr[i] | (byte_weight(pr[i], t->byte_scale) << 24);
    t->pw = (uint32_t *)dev_alloc(t->al, (nmid + 1) * 4);
    if (!t->pw)
        return 2;
    cudaMemcpyAsync(t->pw, pwv.data(), (nmid + 1) * 4, cudaMemcpyHostToDevice, s);
    t->pq = (uint4 *)dev_alloc(t->al, np * sizeof(uint4));
    t->blk_r2 = (uint64_t *)dev_alloc(t->al, np * 8);
    t->pat8 = (uint4 *)dev_alloc(t->al, p8.size());
    t->patsq = (uint32_t *)dev_alloc(t->al, kPatSqWords * 4);
    if (!t->pq || !t->blk_r2 || !t->pat8 || !t->patsq)
        return 2;
    cudaMemcpyAsync(t->pq, pq.data(), np * sizeof(uint4), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(t->pat8, p8.data(), p8.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(t->patsq, psq.data(), kPatSqWords * 4, cudaMemcpyHostToDevice, s);
    // scale-2 records: the same constants with w2(p) in place of w(p)
    for (size_t i = 0; i < np; ++i)
        pq[i].w = (pq[i].w & 0xffffu) | (byte_weight(pr[i], 2) << 16);
    const T2Patterns &tp = t2_patterns();
    t->pq2 = (uint4 *)dev_alloc(t->al, np * sizeof(uint4));
    t->pat2 = (uint4 *)dev_alloc(t->al, tp.a.size());
    t->rec = (uint4 *)dev_alloc(t->al, np * sizeof(uint4));
    t->rec2 = (uint2 *)dev_alloc(t->al, np * sizeof(uint2));
    if (!t->pq2 || !t->pat2 || !t->rec || !t->rec2)
        return 2;
    cudaMemcpyAsync(t->pq2, pq.data(), np * sizeof(uint4), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(t->pat2, tp.a.data(), tp.a.size(), cudaMemcpyHostToDevice, s);
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return 3;
    return 0;
}

int prime_table_create(PrimeTable *t, const Allocator &al, uint64_t y_max, cudaStream_t s,
                       bool with_bytes)
{
    t->al = al;
    uint64_t B = isqrt_u64(y_max);
    if (B < 7)
        B = 7;
    if (B > 0xFFFFFFFFull)
        return 6;
    std::vector<uint32_t> pr = host_primes(B);
    const size_t np = pr.size();
    std::vector<uint32_t> lg(np);
    std::vector<uint64_t> mg(np);
    std::vector<uint8_t> sh(np);
    for (size_t i = 0; i < np; ++i) {
        lg[i] = (uint32_t)std::lround(kLogScale * std::log2((double)pr[i]));
        mg[i] = magic_of(pr[i]);
        sh[i] = (uint8_t)magic_shift(pr[i]);
    }
    // half-word pattern for 2,3,5,7 and 4,9,25,49, then the two word tables
    std::vector<uint32_t> pat16(kPatternPeriod, 0);
    const uint32_t small[4] = {2, 3, 5, 7};
    for (uint32_t i = 0; i < kPatternPeriod; ++i) {
        uint32_t h = 0;
        for (int q = 0; q < 4; ++q) {
            const uint32_t p = small[q];
            if (i % p == 0)
                h += lg[q] | kCountOne;
            if (i % (p * p) == 0)
                h |= kSquareBit;
        }
        pat16[i] = h;
    }
    std::vector<uint32_t> pe(kPatternWords), po(kPatternWords);
    for (uint32_t j = 0; j < kPatternWords; ++j) {
        pe[j] = pat16[2 * j] | (pat16[2 * j + 1] << 16);
        po[j] = pat16[2 * j + 1] | (pat16[(2 * j + 2) % kPatternPeriod] << 16);
    }
    t->np = (uint32_t)np;
    t->host_p = (uint32_t *)malloc(np * sizeof(uint32_t));
    if (!t->host_p)
        return 2;
    memcpy(t->host_p, pr.data(), np * sizeof(uint32_t));
    t->p = (uint32_t *)dev_alloc(al, np * 4);
    t->lg = (uint32_t *)dev_alloc(al, np * 4);
    t->m = (uint64_t *)dev_alloc(al, np * 8);
    t->l = (uint8_t *)dev_alloc(al, np);
    t->blk_r = (uint32_t *)dev_alloc(al, np * 4);
    t->blk_qm = (uint32_t *)dev_alloc(al, np * 4);
    t->pat_even = (uint32_t *)dev_alloc(al, kPatternWords * 4);
    t->pat_odd = (uint32_t *)dev_alloc(al, kPatternWords * 4);
    if (!t->p || !t->lg || !t->m || !t->l || !t->blk_r || !t->blk_qm || !t->pat_even ||
        !t->pat_odd)
        return 2;
    cudaMemcpyAsync(t->p, pr.data(), np * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(t->lg, lg.data(), np * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(t->m, mg.data(), np * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(t->l, sh.data(), np, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(t->pat_even, pe.data(), kPatternWords * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(t->pat_odd, po.data(), kPatternWords * 4, cudaMemcpyHostToDevice, s);
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return 3;
    // byte sieve tables: weight scale 4 below 2^42, 3 up to 2^54
    if (with_bytes && y_max < (1ull << 54)) {
        t->byte_scale = y_max < (1ull << 42) ? 4u : 3u;
        return byte_tables_create(t, pr, s);
    }
    return 0;
}

void prime_table_destroy(PrimeTable *t)
{
    const size_t np = t->np;
    dev_free(t->al, t->p, np * 4);
    dev_free(t->al, t->lg, np * 4);
    dev_free(t->al, t->m, np * 8);
    dev_free(t->al, t->l, np);
    dev_free(t->al, t->blk_r, np * 4);
    dev_free(t->al, t->blk_qm, np * 4);
    dev_free(t->al, t->pat_even, kPatternWords * 4);
    dev_free(t->al, t->pat_odd, kPatternWords * 4);
    dev_free(t->al, t->pq, np * sizeof(uint4));
    dev_free(t->al, t->blk_r2, np * 8);
    dev_free(t->al, t->pat8, (size_t)16 * kPat8Len);
    dev_free(t->al, t->patsq, kPatSqWords * 4);
    dev_free(t->al, t->pq2, np * sizeof(uint4));
    dev_free(t->al, t->pat2, (size_t)16 * kPat2Len);
    dev_free(t->al, t->rec, np * sizeof(uint4));
    dev_free(t->al, t->rec2, np * sizeof(uint2));
    if (t->pw)
        dev_free(t->al, t->pw, ((size_t)t->np_mid + 1) * 4);
    if (t->scratch_len) {
        const uint64_t ntiles = (t->scratch_len + kByteTile - 1) / kByteTile;
        dev_free(t->al, t->bucket, ntiles * t->bucket_cap * 8);
        dev_free(t->al, t->gsq, ntiles * (kByteTile / 8));
        dev_free(t->al, t->perr, 4);
        const uint64_t nt2 = (t->scratch_len + kT2MinTile - 1) / kT2MinTile;
        dev_free(t->al, t->sqcnt, nt2 * 4);
        dev_free(t->al, t->sqlist, nt2 * t->sq_cap * 4);
    }
    free(t->host_p);
    *t = PrimeTable();
}

uint32_t prime_count_upto(const PrimeTable *t, uint64_t b)
{
    uint32_t lo = 0, hi = t->np;  // first index with p > b
    while (lo < hi) {
        uint32_t mid = (lo + hi) / 2;
        if ((uint64_t)t->host_p[mid] <= b)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

int sieve_scratch_create(PrimeTable *t, uint64_t max_len)
{
    if (!t->pq || t->scratch_len || max_len == 0 || max_len > (1ull << 30))
        return 0;
    // entries of a tile: the primes p > 2^17 whose next multiple falls in it,
    // one with probability 2^17/p: mean mu, at most mu + 10 sqrt(mu) + 256
    double mu = 0;
    for (uint32_t i = t->np_mid; i < t->np; ++i)
        mu += (double)kByteTile / (double)t->host_p[i];
    uint32_t cap = (uint32_t)(mu + 10.0 * std::sqrt(mu) + 256.0);
    cap = (cap + 31u) & ~31u;
    const uint64_t ntiles = (max_len + kByteTile - 1) / kByteTile;
    t->bucket = (uint64_t *)dev_alloc(t->al, ntiles * cap * 8);
    t->gsq = (uint32_t *)dev_alloc(t->al, ntiles * (kByteTile / 8));
    t->perr = (uint32_t *)dev_alloc(t->al, 4);
    if (!t->bucket || !t->gsq || !t->perr) {
        dev_free(t->al, t->bucket, ntiles * cap * 8);
        dev_free(t->al, t->gsq, ntiles * (kByteTile / 8));
        dev_free(t->al, t->perr, 4);
        t->bucket = nullptr;
        t->gsq = nullptr;
        t->perr = nullptr;
        return 2;
    }
    // square lists of the scale-2 kernel: the primes 8192 <= q <= P put about
    // T / (8192 ln 8192) multiples of q^2 into a tile of T y (1.3 for 96 Ki
    // y); the kernel clears its tile's count after reading it, so the counts
    // start at zero once, here
    const uint64_t nt2 = (max_len + kT2MinTile - 1) / kT2MinTile;
    t->sq_cap = 64;
    t->sqcnt = (uint32_t *)dev_alloc(t->al, nt2 * 4);
    t->sqlist = (uint32_t *)dev_alloc(t->al, nt2 * t->sq_cap * 4);
    if (!t->sqcnt || !t->sqlist) {
        dev_free(t->al, t->sqcnt, nt2 * 4);
        dev_free(t->al, t->sqlist, nt2 * t->sq_cap * 4);
        t->sqcnt = nullptr;
        t->sqlist = nullptr;
        t->sq_cap = 0;
    } else {
        cudaMemset(t->sqcnt, 0, nt2 * 4);
    }
    cudaMemset(t->perr, 0, 4);
    t->bucket_cap = cap;
    t->scratch_len = max_len;
    return 0;
}

uint32_t sieve_scratch_status(PrimeTable *t)
{
    if (!t->perr)
        return 0;
    uint32_t v = 0;
    cudaMemcpy(&v, t->perr, 4, cudaMemcpyDeviceToHost);
    if (v)
        cudaMemset(t->perr, 0, 4);
    return v;
}

// Most distinct prime factors of any y' <= y (primorials).
static int omega_max(uint64_t y)
{
    static const uint64_t prim[15] = {2ull, 6ull, 30ull, 210ull, 2310ull, 30030ull, 510510ull,
                                      9699690ull, 223092870ull, 6469693230ull,
                                      200560490130ull, 7420738134810ull, 304250263527210ull,
                                      13082761331670030ull, 614889782588491410ull};
    int w = 0;
    while (w < 15 && prim[w] <= y)
        ++w;
    return w;
}

// The byte kernel is exact when all primes up to P >= 2^10 are sieved and,
// with E = the most distinct prime factors below y2 (the summed rounding
// error of the weights), the half gap (S/2) log2 P exceeds E + 2 (the tile
// threshold may sit up to 2 units low), the threshold S log2 y - (S/2) log2 P
// stays below 127 (bias B0 >= 0) and biased bytes stay below 2^8.  Blocks of
// at most 2^30 y keep its offsets within 31 bits.
static bool byte_path_ok(const PrimeTable *t, uint64_t y2, uint64_t P, uint64_t len)
{
    if (!t->pq || P < 1024 || y2 >= (1ull << 54) || len > (1ull << 30))
        return false;
    const double S = t->byte_scale;
    const double half = 0.5 * S * std::log2((double)P);
    const int E = omega_max(y2);
    const double thr = S * std::log2((double)y2) - half;
    return half >= E + 2.5 && thr < 126.0 && 127.0 + half + E + 3.0 < 255.0;
}

// The scale-2 kernel is exact when log2 P - E >= 2.5 (E as above); it also
// needs the biased bytes below 2^8 (1 + A + 126 - thr, A <= 2 log2 y2 + E),
// the sums below 2^7 (bit 7 is the square flag), thr < 126, P >= 2^10 and
// blocks of at most 2^30 y; and its scratch (square lists, status word).
static bool t2_path_ok(const PrimeTable *t, uint64_t y2, uint64_t P, uint64_t len)
{
    if (!t->pq2 || !t->sqcnt || !t->perr || P < 1024 || y2 >= (1ull << 54) ||
        len > (1ull << 30) || len > t->scratch_len)
        return false;
    const double half = std::log2((double)P);
    const int E = omega_max(y2);
    const double thr = 2.0 * std::log2((double)y2) - half;
    const double amax = 2.0 * std::log2((double)y2) + E;
    return half >= E + 2.5 && thr < 124.0 && 1.0 + amax < 127.0 &&
           amax - (thr - 2.0) + 127.0 < 255.0;
}

template <int TILE, int THREADS, int MINB>
static int t2_launch(const PrimeTable *t, const SieveLaunch &L, uint32_t np, uint64_t P,
                     cudaStream_t s)
{
    static std::atomic<uint64_t> attr_devs{0};
    const uint64_t dbit = device_bit();
    if (attrs_needed(attr_devs, dbit)) {
        cudaFuncSetAttribute(mu_sieve_t2_kernel<TILE, THREADS, MINB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, TILE);
        attrs_done(attr_devs, dbit);
    }
    const uint32_t tiles = (uint32_t)((L.len + TILE - 1) / TILE);
    T2Args a{};
    a.y1 = L.y1;
    a.len = (uint32_t)L.len;
    a.np = np;
    a.np_lane = std::min(prime_count_upto(t, kT2LaneMin - 1), np);
    a.np_list = std::min(prime_count_upto(t, kT2ListMin - 1), np);
    a.thr_half = (float)std::log2((double)P);
    a.pq = t->pq2;
    a.r = t->blk_r;
    a.r2 = t->blk_r2;
    a.rec = t->rec;
    a.rec2 = t->rec2;
    a.pat = t->pat2;
    a.sqcnt = t->sqcnt;
    a.sqlist = t->sqlist;
    a.sqcap = t->sq_cap;
    a.Mloc = L.Mloc;
    a.segsum = L.segsum;
    a.mu_out = L.mu_out;
    a.mu_base = L.mu_base;
    a.mu_end = L.mu_end;
    a.err = t->perr;
    a.extra_tx = getenv("MERTENS_TEST_STALL_COPY") ? 16u : 0u;
    t2_block_prep_kernel<<<(np + 255) / 256, 256, 0, s>>>(
        L.y1, np, t->pq2, t->blk_r, t->blk_r2, a.np_lane, t->rec, t->rec2, a.np_list, a.len,
        (uint32_t)TILE, t->sqcnt, t->sqlist, t->sq_cap, t->perr);
    mu_sieve_t2_kernel<TILE, THREADS, MINB><<<tiles, THREADS, TILE, s>>>(a);
    return 2;
}

int sieve_block_enqueue(const PrimeTable *t, const SieveLaunch &L, cudaStream_t s)
{
    static std::atomic<uint64_t> attr_devs{0};
    const uint64_t dbit = device_bit();
    if (attrs_needed(attr_devs, dbit)) {
        cudaFuncSetAttribute(mu_sieve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSieveWords * 4);
        cudaFuncSetAttribute(mu_sieve_byte_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kByteTile + kByteSqWords * 4);
        cudaFuncSetAttribute(mu_sieve_persist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kByteTile + kByteSqWords * 4 + kMedMax * 4);
        attrs_done(attr_devs, dbit);
    }
    const uint64_t y2 = L.y1 + L.len - 1;
    uint64_t P = isqrt_u64(y2);
    if (P < 7)
        P = 7;
    const uint32_t np = prime_count_upto(t, P);
    const uint32_t np_small = prime_count_upto(t, 2047);
    const bool bytes = byte_path_ok(t, y2, P, L.len) && getenv("MERTENS_SIEVE16") == nullptr;
    int launches = 0;
    // the scale-2 kernel where it is exact and the bucketed kernel does not
    // pay (MERTENS_SIEVE_BYTE4 / MERTENS_SIEVE_TILES keep the scale-4/3 per-tile
    // kernel, MERTENS_SIEVE_BUCKETS the bucketed one, MERTENS_SIEVE16 the
    // 16-bit one; MERTENS_T2_TILE=64 takes 64 Ki-y tiles)
    {
        const uint32_t nmid = std::min(t->np_mid, np);
        const bool persist = bytes && t->bucket && L.len <= t->scratch_len && np_small < np &&
                             (np - nmid > 3u * (nmid - std::min(np_small, nmid)) ||
                              getenv("MERTENS_SIEVE_BUCKETS") != nullptr) &&
                             getenv("MERTENS_SIEVE_TILES") == nullptr;
        const bool t2 = bytes && !persist && t2_path_ok(t, y2, P, L.len) &&
                        getenv("MERTENS_SIEVE_BYTE4") == nullptr &&
                        getenv("MERTENS_SIEVE_TILES") == nullptr;
        if (t2) {
            const char *tt = getenv("MERTENS_T2_TILE");
            launches += (tt && tt[0] == '6') ? t2_launch<65536, 512, 3>(t, L, np, P, s)
                                             : t2_launch<98304, 768, 2>(t, L, np, P, s);
            if (L.mid)
                cudaEventRecord(L.mid, s);
            if (L.mid2)
                cudaEventRecord(L.mid2, s);
            const uint32_t nseg = (uint32_t)sieve_segments(L.len);
            seg_carry_kernel<<<(nseg + 1023) / 1024, 1024, 0, s>>>(L.segsum, nseg, L.carry_in,
                                                                  L.segoff, L.carry_out);
            ++launches;
            return cudaGetLastError() == cudaSuccess ? launches : -1;
        }
    }
    if (np > 4) {
        sieve_block_prep_kernel<<<(np + 255) / 256, 256, 0, s>>>(
            L.y1, np, t->p, t->blk_r, t->blk_qm, bytes ? t->blk_r2 : nullptr);
        ++launches;
    }
    if (bytes) {
        ByteArgs b{};
        b.y1 = L.y1;
        b.len = (uint32_t)L.len;
        b.np = np;
        b.np_small = np_small < np ? np_small : np;
        const uint32_t np_p = prime_count_upto(t, 127);
        b.np_piece = np_p < b.np_small ? np_p : b.np_small;
        b.scale = (float)t->byte_scale;
        b.thr_half = (float)(0.5 * t->byte_scale * std::log2((double)P));
        b.pq = t->pq;
        b.r = t->blk_r;
        b.r2 = t->blk_r2;
        b.pat8 = t->pat8;
        b.patsq = t->patsq;
        b.Mloc = L.Mloc;
        b.segsum = L.segsum;
        b.mu_out = L.mu_out;
        b.mu_base = L.mu_base;
        b.mu_end = L.mu_end;
        b.err = t->perr;  // bounded-wait status (null without scratch)
        // MERTENS_TEST_STALL_COPY: announce 16 bytes that never come, so the
        // bounded wait runs out (the test of that error path)
        b.extra_tx = (getenv("MERTENS_TEST_STALL_COPY") && t->perr) ? 16u : 0u;
        const uint32_t btiles = (uint32_t)((L.len + kByteTile - 1) / kByteTile);
        // the bucketed kernel pays once the primes above 2^17 outnumber the
        // medium ones (2048 <= p < 2^17) more than 3:1 (measured crossover
        // near y = 4e11); MERTENS_SIEVE_TILES / MERTENS_SIEVE_BUCKETS force
        // one kernel (tests)
        const uint32_t nmid = std::min(t->np_mid, np);
        bool persist = np - nmid > 3u * (nmid - std::min(np_small, nmid));
        if (getenv("MERTENS_SIEVE_BUCKETS"))
            persist = true;
        if (getenv("MERTENS_SIEVE_TILES"))
            persist = false;
        persist = persist && t->bucket && L.len <= t->scratch_len && np_small < np;
        if (persist) {
            int dev = 0, sms = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            // at least 64 CTAs keep a CTA's tiles within kPersistTilesMax
            const uint32_t grid = std::min<uint32_t>((uint32_t)std::max(sms, 64), btiles);
            b.np_mid = std::min(t->np_mid, np);
            b.cap = t->bucket_cap;
            b.pw = t->pw;
            b.gsq = t->gsq;
            b.bucket = t->bucket;
            b.err = t->perr;
            cudaMemsetAsync(t->gsq, 0, (size_t)btiles * (kByteTile / 8), s);
            const uint32_t nsq = np - b.np_small;
            square_bits_kernel<<<(nsq + 255) / 256, 256, 0, s>>>((uint32_t)L.len, b.np_small, np,
                                                              t->p, t->blk_r2, t->gsq);
            mu_sieve_persist_kernel<<<grid, kSieveThreads,
                                      kByteTile + kByteSqWords * 4 + kMedMax * 4, s>>>(b);
            launches += 2;
        } else {
            mu_sieve_byte_kernel<<<btiles, kSieveThreads, kByteTile + kByteSqWords * 4, s>>>(b);
            ++launches;
        }
    }
    const uint32_t tiles = bytes ? 0u : (uint32_t)((L.len + kSieveTile - 1) / kSieveTile);
    SieveArgs a;
    a.y1 = L.y1;
    a.len = L.len;
    a.np = np;
    a.np_small = np_small < np ? np_small : np;
    const uint32_t np_q = prime_count_upto(t, 127);
    a.np_quarter = np_q < a.np_small ? np_q : a.np_small;
    a.thr_bias = (float)(0.5 * kLogScale * std::log2((double)P));
    a.p = t->p;
    a.lg = t->lg;
    a.r = t->blk_r;
    a.qm = t->blk_qm;
    a.pat_even = t->pat_even;
    a.pat_odd = t->pat_odd;
    a.m = t->m;
    a.l = t->l;
    a.Mloc = L.Mloc;
    a.segsum = L.segsum;
    a.mu_out = L.mu_out;
    a.mu_base = L.mu_base;
    a.mu_end = L.mu_end;
    if (tiles) {
        mu_sieve_kernel<<<tiles, kSieveThreads, kSieveWords * 4, s>>>(a);
        ++launches;
    }
    if (L.mid)
        cudaEventRecord(L.mid, s);
    if (L.mid2)
        cudaEventRecord(L.mid2, s);
    const uint32_t nseg = (uint32_t)sieve_segments(L.len);
    seg_carry_kernel<<<(nseg + 1023) / 1024, 1024, 0, s>>>(L.segsum, nseg, L.carry_in, L.segoff,
                                                          L.carry_out);
    ++launches;
    if (cudaGetLastError() != cudaSuccess)
        return -1;
    return launches;
}

int expand_M_enqueue(const int16_t *Mloc, const int64_t *segoff, uint64_t len, int32_t *M,
                     uint32_t *err, cudaStream_t s)
{
    uint64_t blocks = (len + 255) / 256;
    if (blocks > 152 * 32)
        blocks = 152 * 32;
    expand_M_kernel<<<(unsigned)blocks, 256, 0, s>>>(Mloc, segoff, len, M, err);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace mert
