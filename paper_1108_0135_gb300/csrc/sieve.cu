// Steps a1 (mu_sieve) and a2 (m_scan) of the isolated-value Mertens method:
// mu(y) for a block of y by a segmented log sieve, then M(y) by prefix sum
// with the carry of the previous block (arXiv:1108.0135, Sec. 3).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace mert {

// ---------------------------------------------------------------------------
// a1: per-block remainders of the sieving primes.
// ---------------------------------------------------------------------------
__global__ void sieve_block_prep_kernel(uint64_t y1, uint32_t np, const uint32_t *__restrict__ p,
                                        uint32_t *__restrict__ r, uint32_t *__restrict__ qm)
{
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np)
        return;
    uint64_t pp = p[t];
    r[t] = (uint32_t)(y1 % pp);
    qm[t] = (uint32_t)((y1 / pp) % pp);
}

struct SieveArgs {
    uint64_t y1, len;
    uint32_t np, np_small;      // primes used; [4, np_small) sieved warp-cooperatively
    float thr_bias;             // 8 * log2(P), P = largest value all of whose primes are sieved
    const uint32_t *p, *lg, *r, *qm, *pattern;
    const uint64_t *m;
    const uint8_t *l;
    int8_t *mu;
    int8_t *mu_aux;
    uint64_t aux_end;
    int32_t *tile_sum;
};

// First multiple of p at or after t1 = y1 + a0, as an offset `off` into the
// tile, and c = (that multiple / p) mod p, which is 0 exactly when p^2 divides
// the multiple.  Uses y1 mod p and floor(y1/p) mod p of the block.
__device__ __forceinline__ void first_multiple(const SieveArgs &a, uint32_t t, uint64_t a0,
                                               uint32_t &p, uint32_t &off, uint32_t &c)
{
    p = a.p[t];
    const uint64_t m = a.m[t];
    const unsigned l = a.l[t];
    const uint64_t v = (uint64_t)a.r[t] + a0;       // (t1 - floor(y1/p)*p)
    const uint64_t qv = div_magic(v << 1, m, l);     // floor(v / p)
    const uint32_t off0 = (uint32_t)(v - qv * p);    // t1 mod p
    off = off0 ? p - off0 : 0u;
    const uint64_t c0 = (uint64_t)a.qm[t] + qv + (off0 ? 1u : 0u);
    c = (uint32_t)(c0 - div_magic(c0 << 1, m, l) * p);
}

// mu(y) for one tile of kSieveTile y values.  Each y owns one 32-bit shared
// word; every sieving prime p adds round(16 log2 p) plus one to the prime
// count at its multiples, and one to the square count at multiples of p^2
// (shared-memory atomics).  Primes 2, 3, 5, 7 and their squares come from a
// periodic pattern.  Decoding (exact; proof in the design notes): with all
// primes <= P sieved and (P+1)^2 > y, the unsieved cofactor c of y is 1 or a
// prime > P; the log sum A is within 7.5 units of 16 log2 y when c = 1 and at
// least 16 log2 P - 7 units below it otherwise, so "A > 16 log2 y - 8 log2 P"
// decides c = 1.  mu = 0 if a square divides y, else (-1)^(count + [c > 1]).
__global__ void __launch_bounds__(kSieveThreads) mu_sieve_kernel(SieveArgs a)
{
    extern __shared__ uint32_t w[];
    __shared__ int red[33];
    const uint64_t a0 = (uint64_t)blockIdx.x * kSieveTile;
    const uint64_t t1 = a.y1 + a0;
    const uint32_t tl = (uint32_t)((a.len - a0) < (uint64_t)kSieveTile ? (a.len - a0) : kSieveTile);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;

    // pattern of primes 2,3,5,7 (period 44100 > tile, so at most one wrap)
    {
        const uint32_t ph = (uint32_t)(t1 % kPatternPeriod);
        for (uint32_t i = threadIdx.x; i < (uint32_t)kSieveTile; i += blockDim.x) {
            uint32_t idx = ph + i;
            if (idx >= kPatternPeriod)
                idx -= kPatternPeriod;
            w[i] = a.pattern[idx];
        }
    }
    __syncthreads();

    // small primes: a warp per prime, lanes over its multiples
    for (uint32_t t = 4 + warp; t < a.np_small; t += nwarp) {
        uint32_t p, off, c;
        first_multiple(a, t, a0, p, off, c);
        const uint32_t add = a.lg[t] | kCountOne;
        uint32_t ci = (c + (uint32_t)lane) % p;
        const uint32_t inc = 32u % p;
        for (uint32_t yo = off + (uint32_t)lane * p; yo < tl; yo += 32u * p) {
            atomicAdd(&w[yo], add + (ci == 0 ? kSquareOne : 0u));
            ci += inc;
            if (ci >= p)
                ci -= p;
        }
    }
    // large primes: a thread per prime
    for (uint32_t t = (a.np_small > 4 ? a.np_small : 4) + threadIdx.x; t < a.np; t += blockDim.x) {
        uint32_t p, off, c;
        first_multiple(a, t, a0, p, off, c);
        const uint32_t add = a.lg[t] | kCountOne;
        for (uint32_t yo = off; yo < tl; yo += p) {
            atomicAdd(&w[yo], add + (c == 0 ? kSquareOne : 0u));
            c = (c + 1 == p) ? 0u : c + 1;
        }
    }
    __syncthreads();

    // decode 16 consecutive y per step, 16-byte stores
    int sum = 0;
    const uint32_t ngroups = (tl + 15) / 16;
    for (uint32_t g = threadIdx.x; g < ngroups; g += blockDim.x) {
        const uint32_t i0 = g * 16;
        const uint64_t y0 = t1 + i0;
        const float base = (float)kLogScale * __log2f(__ull2float_rn(y0)) - a.thr_bias;
        int8_t v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const uint32_t word = w[(i0 + k) < (uint32_t)kSieveTile ? i0 + k : 0];
            const uint64_t y = y0 + k;
            float thr = base;
            if (y0 < 4096)
                thr = (float)kLogScale * __log2f((float)y) - a.thr_bias;
            const int A = (int)(word & 2047u);
            const int cnt = (int)((word >> 11) & 31u);
            const int fully = (float)A > thr ? 1 : 0;
            int mu = ((cnt + (fully ^ 1)) & 1) ? -1 : 1;
            if (word >> 16)
                mu = 0;
            v[k] = (int8_t)((i0 + k) < tl ? mu : 0);
            sum += v[k];
        }
        int8_t *dst = a.mu + a0 + i0;
        if (i0 + 16 <= tl) {
            int4 pack;
            memcpy(&pack, v, 16);
            *reinterpret_cast<int4 *>(dst) = pack;
        } else {
            for (uint32_t k = 0; i0 + k < tl; ++k)
                dst[k] = v[k];
        }
        if (a.mu_aux && y0 <= a.aux_end) {
            for (int k = 0; k < 16; ++k) {
                const uint64_t y = y0 + k;
                if (i0 + k < tl && y <= a.aux_end)
                    a.mu_aux[y - 1] = v[k];
            }
        }
    }
    int tot;
    block_excl_scan<int>(sum, red, &tot);
    if (threadIdx.x == 0 && a.tile_sum)
        a.tile_sum[blockIdx.x] = tot;
}

// ---------------------------------------------------------------------------
// a2: carries of the tiles, then M(y) of each tile.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) tile_carry_kernel(const int32_t *__restrict__ tile_sum,
                                                          uint32_t ntiles,
                                                          int64_t *__restrict__ tile_off,
                                                          int64_t *__restrict__ carry)
{
    __shared__ int64_t sh[33];
    const uint32_t per = (ntiles + blockDim.x - 1) / blockDim.x;
    const uint32_t b = threadIdx.x * per, e = min(ntiles, b + per);
    int64_t s = 0;
    for (uint32_t i = b; i < e; ++i)
        s += tile_sum[i];
    int64_t tot;
    int64_t ex = block_excl_scan<int64_t>(s, sh, &tot);
    const int64_t base = *carry;
    __syncthreads();
    int64_t run = base + ex;
    for (uint32_t i = b; i < e; ++i) {
        tile_off[i] = run;
        run += tile_sum[i];
    }
    if (threadIdx.x == 0)
        *carry = base + tot;
}

// M(y) = carry + prefix sum of mu over one tile: 1024 threads x 32 y, then a
// padded shared-memory transpose for coalesced int32 stores.
__global__ void __launch_bounds__(1024) m_scan_kernel(const int8_t *__restrict__ mu, uint64_t len,
                                                      const int64_t *__restrict__ tile_off,
                                                      int32_t *__restrict__ M,
                                                      uint32_t *__restrict__ err)
{
    extern __shared__ int32_t buf[];  // kSieveTile + kSieveTile/32 words
    __shared__ int32_t sh[33];
    const uint64_t a0 = (uint64_t)blockIdx.x * kSieveTile;
    const uint32_t tl = (uint32_t)((len - a0) < (uint64_t)kSieveTile ? (len - a0) : kSieveTile);
    const uint32_t i0 = threadIdx.x * 32;
    int8_t v[32];
    if (i0 + 32 <= tl) {
        const int4 *src = reinterpret_cast<const int4 *>(mu + a0 + i0);
        int4 x0 = src[0], x1 = src[1];
        memcpy(v, &x0, 16);
        memcpy(v + 16, &x1, 16);
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k)
            v[k] = (i0 + k < tl) ? mu[a0 + i0 + k] : 0;
    }
    int run = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k)
        run += v[k];
    int tot;
    const int ex = block_excl_scan<int>(run, sh, &tot);
    int64_t mv = tile_off[blockIdx.x] + ex;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        mv += v[k];
        bad |= (mv > INT32_MAX) || (mv < INT32_MIN);
        const uint32_t e = i0 + k;
        buf[e + (e >> 5)] = (int32_t)mv;
    }
    if (bad)
        atomicOr(err, kErrMOverflow);
    __syncthreads();
    for (uint32_t e = threadIdx.x; e < tl; e += blockDim.x)
        M[a0 + e] = buf[e + (e >> 5)];
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
    while (r * r > v)
        --r;
    while ((r + 1) * (r + 1) <= v)
        ++r;
    return r;
}

int prime_table_create(PrimeTable *t, const Allocator &al, uint64_t y_max, cudaStream_t s)
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
    // pattern for 2,3,5,7 and 4,9,25,49
    std::vector<uint32_t> pat(kPatternPeriod, 0);
    const uint32_t small[4] = {2, 3, 5, 7};
    for (uint32_t i = 0; i < kPatternPeriod; ++i) {
        uint32_t wv = 0;
        for (int q = 0; q < 4; ++q) {
            const uint32_t p = small[q];
            if (i % p == 0)
                wv += lg[q] | kCountOne;
            if (i % (p * p) == 0)
                wv += kSquareOne;
        }
        pat[i] = wv;
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
    t->pattern = (uint32_t *)dev_alloc(al, kPatternPeriod * 4);
    if (!t->p || !t->lg || !t->m || !t->l || !t->blk_r || !t->blk_qm || !t->pattern)
        return 2;
    cudaMemcpyAsync(t->p, pr.data(), np * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(t->lg, lg.data(), np * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(t->m, mg.data(), np * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(t->l, sh.data(), np, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(t->pattern, pat.data(), kPatternPeriod * 4, cudaMemcpyHostToDevice, s);
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return 3;
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
    dev_free(t->al, t->pattern, kPatternPeriod * 4);
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

int sieve_block_enqueue(const PrimeTable *t, const SieveLaunch &L, cudaStream_t s)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(mu_sieve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSieveTile * 4);
        cudaFuncSetAttribute(m_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (kSieveTile + kSieveTile / 32) * 4);
        attr_set = true;
    }
    const uint64_t y2 = L.y1 + L.len - 1;
    uint64_t P = isqrt_u64(y2);
    if (P < 7)
        P = 7;
    const uint32_t np = prime_count_upto(t, P);
    const uint32_t np_small = prime_count_upto(t, 1023);
    int launches = 0;
    const uint32_t tiles = (uint32_t)sieve_tiles(L.len);
    if (np > 4) {
        sieve_block_prep_kernel<<<(np + 255) / 256, 256, 0, s>>>(L.y1, np, t->p, t->blk_r,
                                                                 t->blk_qm);
        ++launches;
    }
    SieveArgs a;
    a.y1 = L.y1;
    a.len = L.len;
    a.np = np;
    a.np_small = np_small < np ? np_small : np;
    a.thr_bias = (float)(8.0 * std::log2((double)P));
    a.p = t->p;
    a.lg = t->lg;
    a.r = t->blk_r;
    a.qm = t->blk_qm;
    a.pattern = t->pattern;
    a.m = t->m;
    a.l = t->l;
    a.mu = L.mu;
    a.mu_aux = L.mu_aux;
    a.aux_end = L.aux_end;
    a.tile_sum = L.tile_sum;
    mu_sieve_kernel<<<tiles, kSieveThreads, kSieveTile * 4, s>>>(a);
    ++launches;
    if (L.mid)
        cudaEventRecord(L.mid, s);
    if (L.mid2)
        cudaEventRecord(L.mid2, s);
    if (L.M) {
        tile_carry_kernel<<<1, 1024, 0, s>>>(L.tile_sum, tiles, L.tile_off, L.carry);
        m_scan_kernel<<<tiles, 1024, (kSieveTile + kSieveTile / 32) * 4, s>>>(
            L.mu, L.len, L.tile_off, L.M, L.err);
        launches += 2;
    }
    if (cudaGetLastError() != cudaSuccess)
        return -1;
    return launches;
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scan of uint32 (three passes, no inter-CTA waits).
// ---------------------------------------------------------------------------
constexpr int kScanPer = 2048;  // values per CTA (256 threads x 8)

__global__ void __launch_bounds__(256) scan_reduce_kernel(const uint32_t *__restrict__ in, size_t n,
                                                          uint32_t *__restrict__ part)
{
    __shared__ uint32_t sh[33];
    const size_t b = (size_t)blockIdx.x * kScanPer;
    uint32_t s = 0;
    for (int k = 0; k < 8; ++k) {
        size_t i = b + (size_t)k * 256 + threadIdx.x;
        if (i < n)
            s += in[i];
    }
    uint32_t tot;
    block_excl_scan<uint32_t>(s, sh, &tot);
    if (threadIdx.x == 0)
        part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) scan_parts_kernel(uint32_t *__restrict__ part, uint32_t nparts,
                                                          uint32_t *__restrict__ total_out)
{
    __shared__ uint32_t sh[33];
    const uint32_t per = (nparts + blockDim.x - 1) / blockDim.x;
    const uint32_t b = threadIdx.x * per, e = min(nparts, b + per);
    uint32_t s = 0;
    for (uint32_t i = b; i < e; ++i)
        s += part[i];
    uint32_t tot;
    uint32_t run = block_excl_scan<uint32_t>(s, sh, &tot);
    for (uint32_t i = b; i < e; ++i) {
        uint32_t v = part[i];
        part[i] = run;
        run += v;
    }
    if (threadIdx.x == 0)
        *total_out = tot;
}

__global__ void __launch_bounds__(256) scan_down_kernel(const uint32_t *__restrict__ in, size_t n,
                                                        const uint32_t *__restrict__ part,
                                                        uint32_t *__restrict__ out)
{
    __shared__ uint32_t sh[33];
    const size_t b = (size_t)blockIdx.x * kScanPer + (size_t)threadIdx.x * 8;
    uint32_t v[8], s = 0;
    for (int k = 0; k < 8; ++k) {
        size_t i = b + k;
        v[k] = i < n ? in[i] : 0u;
        s += v[k];
    }
    uint32_t tot;
    uint32_t run = block_excl_scan<uint32_t>(s, sh, &tot) + part[blockIdx.x];
    for (int k = 0; k < 8; ++k) {
        size_t i = b + k;
        if (i < n)
            out[i] = run;
        run += v[k];
    }
}

size_t scan_scratch_words(size_t n)
{
    return (n + kScanPer - 1) / kScanPer + 1;
}

int exclusive_scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *scratch,
                       cudaStream_t s)
{
    const uint32_t nparts = (uint32_t)((n + kScanPer - 1) / kScanPer);
    if (nparts == 0) {
        cudaMemsetAsync(out, 0, 4, s);
        return 1;
    }
    scan_reduce_kernel<<<nparts, 256, 0, s>>>(in, n, scratch);
    scan_parts_kernel<<<1, 1024, 0, s>>>(scratch, nparts, out + n);
    scan_down_kernel<<<nparts, 256, 0, s>>>(in, n, scratch, out);
    if (cudaGetLastError() != cudaSuccess)
        return -1;
    return 3;
}

}  // namespace mert
