// Step a3 (mertens_update) and step a4 (resolve) of the isolated-value
// Mertens method (arXiv:1108.0135, Sec. 2-3).
//
// Entry x of a target n has k = floor(n/x) and s = floor(sqrt(k)).  By the
// split formula of Sec. 2 (taken at t = s+1) its array value is
//   M(k) = 1 - sum_{j=2}^{floor(k/(s+1))} M(floor(k/j))
//            - sum_{y=1}^{s} M(y) (floor(k/y) - floor(k/(y+1))).
// The terms with j <= floor(k/u) are other array entries (added in resolve);
// the rest -- direct terms y <= s and gathered terms j in
// [floor(k/u)+1, floor(k/(s+1))] -- are accumulated into S[x] by the update.
//
// The update covers y in [1, yc] for a cut-off yc >= s (a "dense" range, the
// paper's regions 1 and 1', Sec. 3) with the coefficient form
//   sum_{y<=yc} M(y)(q(y) - q(y+1)) = sum_{y<=yc} mu(y) q(y) - M(yc) q(yc+1),
// q(y) = floor(k/y) (summation by parts), which needs mu(y) and one quotient
// per squarefree y; and it covers y > yc with the gathered form, one term
// M(floor(k/j)) for each j in [floor(k/u)+1, floor(k/(yc+1))] (regions 2-4).
// Both forms count every j >= floor(k/u)+1 exactly once, so the sum is the
// same for any yc in [s, floor(k/(floor(k/u)+1)) - 1].
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "update.h"

namespace mert {

// ---------------------------------------------------------------------------
// Tables.
// ---------------------------------------------------------------------------
// MG[d] = division magic of d, d = 1..nd (MG[0] unused).
__global__ void magic_table_kernel(uint64_t *__restrict__ MG, uint64_t nd)
{
    for (uint64_t d = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; d <= nd;
         d += (uint64_t)gridDim.x * blockDim.x)
        MG[d] = magic_of(d);
}

// Squarefree list of one chunk of kChunk y values (y <= ydense): the magics
// and offsets y - chunk start, in increasing y, in four parts -- mu = +1 and
// odd y, +1 and even y, -1 and odd y, -1 and even y -- each from an even
// index; dl_cnt = {n0 | n1 << 16, n2 | n3 << 16}.  256 threads x 16 y.
__device__ __forceinline__ uint32_t even_up(uint32_t v) { return (v + 1u) & ~1u; }

__global__ void __launch_bounds__(256) dense_list_kernel(const int8_t *__restrict__ mu_aux,
                                                         uint64_t ydense,
                                                         const uint64_t *__restrict__ MG,
                                                         uint64_t *__restrict__ dl_m,
                                                         uint16_t *__restrict__ dl_yo,
                                                         uint2 *__restrict__ dl_cnt)
{
    __shared__ uint32_t sh[33];
    const uint64_t c = blockIdx.x;
    const uint64_t cb = c * kChunk;
    int8_t mv[16];
    uint32_t cp = 0, cm = 0;  // per thread: counts of the parts, 16-bit fields (odd | even << 16)
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint64_t y = cb + threadIdx.x * 16 + k;
        mv[k] = (y >= 1 && y <= ydense) ? mu_aux[y - 1] : (int8_t)0;
        const uint32_t f = (k & 1) ? 1u : 65536u;  // y even when k is (cb and 16 t are even)
        cp += mv[k] > 0 ? f : 0u;
        cm += mv[k] < 0 ? f : 0u;
    }
    uint32_t totp, totm;
    const uint32_t ip = block_scan_u32(cp, sh, &totp);  // no field exceeds 2048
    const uint32_t im = block_scan_u32(cm, sh, &totm);
    const uint32_t n0 = totp & 0xffffu, n1 = totp >> 16, n2 = totm & 0xffffu;
    const uint32_t b1 = even_up(n0), b2 = b1 + even_up(n1), b3 = b2 + even_up(n2);
    uint32_t i0 = ip & 0xffffu, i1 = b1 + (ip >> 16), i2 = b2 + (im & 0xffffu),
             i3 = b3 + (im >> 16);
    uint64_t *dm = dl_m + c * kChunkCapPad;
    uint16_t *dy = dl_yo + c * kChunkCapPad;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint32_t o = threadIdx.x * 16 + k;
        const uint64_t y = cb + o;
        if (mv[k] != 0) {
            const uint32_t i = mv[k] > 0 ? ((k & 1) ? i0++ : i1++) : ((k & 1) ? i2++ : i3++);
            dm[i] = MG[y];
            dy[i] = (uint16_t)o;
        }
    }
    if (threadIdx.x == 0)
        dl_cnt[c] = make_uint2(totp, totm);
}

// ---------------------------------------------------------------------------
// Dense update: lanes = 32 array entries of one group, all reading the same
// squarefree y (shared-memory broadcast); S[x] += sum mu(y) floor(k/y).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t upper_bound_u16(const uint16_t *a, uint32_t n, uint32_t v)
{
    uint32_t lo = 0, hi = n;  // first index with a[i] > v
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (a[mid] <= v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Sum of floor(k/y) over a staged list with the chunk's uniform shift l.
__device__ __forceinline__ uint64_t quot_sum_uniform(uint64_t k2, const uint64_t *mp, uint32_t n,
                                                     unsigned l)
{
    uint64_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    uint32_t i = 0;
    const ulonglong2 *m2 = reinterpret_cast<const ulonglong2 *>(mp);
    for (; i + 4 <= n; i += 4) {
        const ulonglong2 u = m2[i >> 1];
        const ulonglong2 v = m2[(i >> 1) + 1];
        a0 += div_magic(k2, u.x, l);
        a1 += div_magic(k2, u.y, l);
        a2 += div_magic(k2, v.x, l);
        a3 += div_magic(k2, v.y, l);
    }
    for (; i < n; ++i)
        a0 += div_magic(k2, mp[i], l);
    return (a0 + a1) + (a2 + a3);
}

// The same over mp[s0 .. s0 + n): a first odd element alone, then from an
// even index (mp itself starts at an even index).
__device__ __forceinline__ uint64_t quot_sum_uniform_at(uint64_t k2, const uint64_t *mp,
                                                        uint32_t s0, uint32_t n, unsigned l)
{
    uint64_t a = 0;
    if ((s0 & 1u) && n) {
        a = div_magic(k2, mp[s0], l);
        ++s0;
        --n;
    }
    return a + quot_sum_uniform(k2, mp + s0, n, l);
}

// Same with a per-term shift (chunk 0) and/or a per-lane cut-off y <= ycl.
__device__ __forceinline__ uint64_t quot_sum_general(uint64_t k2, const uint64_t *mp,
                                                     const uint16_t *yp, uint32_t n, uint64_t cb,
                                                     unsigned l, bool var_shift, uint64_t ycl)
{
    uint64_t a = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const uint64_t y = cb + yp[i];
        const unsigned li = var_shift ? magic_shift(y) : l;
        const uint64_t q = div_magic(k2, mp[i], li);
        a += (y <= ycl) ? q : 0ull;
    }
    return a;
}

__global__ void __launch_bounds__(kDenseThreads) dense_update_kernel(DenseArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint64_t *s_m = reinterpret_cast<uint64_t *>(smem);
    uint16_t *s_yo = reinterpret_cast<uint16_t *>(s_m + kDenseChunks * kChunkCapPad);
    __shared__ uint32_t s_item;
    __shared__ uint2 s_cnt[kDenseChunks];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(a.counter, 1u);
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= a.nitems)
            break;
        const DenseItem d = a.items[it];
        for (uint32_t c = d.c0; c < d.c1; ++c) {
            const uint2 cnt = a.dl_cnt[c];
            const uint32_t tot = even_up(cnt.x & 0xffffu) + even_up(cnt.x >> 16) +
                                 even_up(cnt.y & 0xffffu) + (cnt.y >> 16);
            const uint64_t *src = a.dl_m + (uint64_t)c * kChunkCapPad;
            const uint16_t *ysrc = a.dl_yo + (uint64_t)c * kChunkCapPad;
            uint64_t *dst = s_m + (c - d.c0) * kChunkCapPad;
            uint16_t *ydst = s_yo + (c - d.c0) * kChunkCapPad;
            for (uint32_t i = threadIdx.x; i < tot; i += blockDim.x) {
                dst[i] = src[i];
                ydst[i] = ysrc[i];
            }
            if (threadIdx.x == 0)
                s_cnt[c - d.c0] = cnt;
        }
        __syncthreads();
        for (uint32_t g = d.g0 + warp; g < d.g1; g += nwarp) {
            const Group G = a.groups[g];
            const bool act = (uint32_t)lane < G.count;
            const uint64_t e = (uint64_t)G.first + (uint64_t)G.stride * lane;
            const uint64_t k2 = act ? (a.K[e] << 1) : 0ull;
            const uint64_t ycl = G.pred ? (act ? a.YCE[e] : 0ull) : G.yc;
            uint64_t acc_o = 0, acc_e = 0;  // odd-y and even-y parts, mod 2^64
            for (uint32_t c = d.c0; c < d.c1; ++c) {
                const uint64_t cb = (uint64_t)c * kChunk;
                if (cb > G.yc)
                    break;
                const uint2 cnt = s_cnt[c - d.c0];
                // parts: [lo, hi) index ranges of +odd, +even, -odd, -even
                uint32_t n[4] = {cnt.x & 0xffffu, cnt.x >> 16, cnt.y & 0xffffu, cnt.y >> 16};
                uint32_t base[4];
                base[0] = 0;
                base[1] = even_up(n[0]);
                base[2] = base[1] + even_up(n[1]);
                base[3] = base[2] + even_up(n[2]);
                const uint64_t *mp = s_m + (c - d.c0) * kChunkCapPad;
                const uint16_t *yp = s_yo + (c - d.c0) * kChunkCapPad;
                if (cb + kChunk - 1 > G.yc) {
                    const uint32_t lim = (uint32_t)(G.yc - cb);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        n[q] = upper_bound_u16(yp + base[q], n[q], lim);
                }
                // odd y <= olo come from entry x/2 (the group's lower bound)
                uint32_t skip[4] = {0, 0, 0, 0};
                if (G.olo >= cb) {
                    if (G.olo >= cb + kChunk - 1) {
                        skip[0] = n[0];
                        skip[2] = n[2];
                    } else {
                        const uint32_t lo = (uint32_t)(G.olo - cb);
                        skip[0] = upper_bound_u16(yp + base[0], n[0], lo);
                        skip[2] = upper_bound_u16(yp + base[2], n[2], lo);
                    }
                }
                const unsigned l = magic_shift((c + 1) * (uint64_t)kChunk - 1);
                uint64_t part[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t s0 = skip[q], cntq = n[q] > s0 ? n[q] - s0 : 0u;
                    if (c == 0 || G.pred)
                        part[q] = quot_sum_general(k2, mp + base[q] + s0, yp + base[q] + s0, cntq,
                                                   cb, l, c == 0, ycl);
                    else
                        part[q] = quot_sum_uniform_at(k2, mp + base[q], s0, cntq, l);
                }
                acc_o += part[0] - part[2];
                acc_e += part[1] - part[3];
            }
            if (act) {
                atomicAdd(reinterpret_cast<unsigned long long *>(a.S + e),
                          (unsigned long long)(acc_o + acc_e));
                if ((G.emit >> lane) & 1u) {
                    // entry 2x: its odd y' = y/2 terms are minus these
                    const uint64_t x = (uint64_t)G.x0 + (uint64_t)G.stride * lane;
                    atomicAdd(reinterpret_cast<unsigned long long *>(a.S + e + x),
                              (unsigned long long)(0ull - acc_e));
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Gathered terms of one sieve block [y1, y2].
// ---------------------------------------------------------------------------
// Entries with at most this many gathered terms in a tile or block are
// handled by one lane; more, by a whole warp.
constexpr uint64_t kLaneTerms = 48;

// M(y) of the current block from its segment offsets and int16 values.
__device__ __forceinline__ int64_t block_M(const int64_t *segoff, const int16_t *Mloc,
                                           uint64_t i)
{
    return segoff[i >> kSegShift] + (int64_t)Mloc[i];
}

// Gathered terms shared along chains x, 2x, 4x, 8x, 16x of one target:
// since floor(floor(n/x)/(2^s j')) = floor(floor(n/(2^s x))/j'), entry x's
// term at j = 2^s j' is entry 2^s x's term at j'.  The plan gives each entry
// of a chain after its first only the j above half of the previous entry's
// top (its own range starts there; the part below is the previous entries'
// terms), and every entry adds, for s = 1 .. L, the sum of its own terms at
// j = 0 mod 2^s to entry 2^s x.  EMIT[e] = x | L << 29 (L <= 4; 0: none).
// Results are unchanged; the plan states which chains are valid.
static_assert(kShareLevels >= 1 && kShareLevels <= 4, "level sums come from the c-bit butterfly");
constexpr uint32_t kShareShift = 29;

// Warp sum of v where lane l holds terms j = top - l - 32 i (so all of one
// residue c = (top - l) mod 32): a butterfly over the bits of c from the
// highest down.  After the step on bit 2^s every lane holds the sum over the
// c' that agree with its c below bit s, so the lane with c = 0 holds the sum
// over j = 0 mod 2^s: h[s - 1] (s = 4 .. 1, valid in that lane only).  The
// last step gives the total (every lane).
__device__ __forceinline__ int64_t warp_sum_levels(int64_t v, uint32_t top, uint32_t lane,
                                                   int64_t h[kShareLevels])
{
    const uint32_t c = (top - lane) & 31u;
#pragma unroll
    for (int s = 4; s >= 1; --s) {
        v += __shfl_sync(0xffffffffu, v, (int)((top - (c ^ (1u << s))) & 31u));
        if (s <= (int)kShareLevels)
            h[s - 1] = v;
    }
    return v + __shfl_sync(0xffffffffu, v, (int)((top - (c ^ 1u)) & 31u));
}

// Adds entry e's level sums over its own j in [lo, hi] (1 <= lo) to the
// entries 2^s x it feeds; base is added once per term (the tile kernels'
// staged values are relative to it).
__device__ __forceinline__ void emit_levels(uint64_t *S, uint64_t e, uint32_t em, uint64_t lo,
                                            uint64_t hi, const int64_t h[kShareLevels],
                                            int64_t base)
{
    const uint32_t L = em >> kShareShift;
    const uint64_t x = em & ((1u << kShareShift) - 1u);
#pragma unroll
    for (uint32_t s = 1; s <= kShareLevels; ++s) {
        if (s > L)
            break;
        const uint64_t c = (hi >> s) - ((lo - 1u) >> s);  // multiples of 2^s in [lo, hi]
        if (c)
            atomicAdd(reinterpret_cast<unsigned long long *>(S + e + ((1ull << s) - 1u) * x),
                      (unsigned long long)(h[s - 1] + (int64_t)c * base));
    }
}

// M(floor(k/j)) of the block for four j at once: the four magic loads, then
// the four M loads, so eight loads per lane are in flight instead of a chain.
// h[s - 1] gets the part over j = 0 mod 2^s.
__device__ __forceinline__ int64_t block_M4(const SparseArgs &a, uint64_t k2, uint64_t y1,
                                            const uint32_t j[4], const bool ok[4],
                                            int64_t h[kShareLevels])
{
    uint64_t m[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
        m[u] = ok[u] ? a.MG[j[u]] : 0ull;
    uint64_t i[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
        i[u] = ok[u] ? div_magic(k2, m[u], 32u - __clz(j[u] - 1u)) - y1 : 0ull;
    int64_t s = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (ok[u]) {
            const int64_t v = block_M(a.segoff, a.Mloc, i[u]);
            s += v;
#pragma unroll
            for (uint32_t l = 0; l < kShareLevels; ++l)
                h[l] += (j[u] & ((2u << l) - 1u)) ? 0 : v;
        }
    return s;
}

// Global-memory part [y_lo, y2] of block [y1, y2], one lane per entry (those
// with k < kmax; the others take the block's shared-memory tiles): the
// entry's j-range, j in [max(jlo, floor(k/(y2+1))+1), min(jc0, floor(k/y_lo))]
// (so floor(k/j) lies in it; every earlier block's range ends above it).
// Entries with at most kLaneTerms terms are summed here, four terms at a time;
// heavier ones are posted as chunks of kSparseItem consecutive j (a
// warp-aggregated slot count) for sparse_chunk_kernel.  Also adds the
// boundary term -M(yc) floor(k/(yc+1)) of the dense form when yc is in the
// block.
__global__ void __launch_bounds__(256) sparse_range_kernel(SparseBlockArgs b, SparseArgs a)
{
    const uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u;
    const bool act = e < a.nent;
    const uint64_t k = act ? a.K[e] : 0ull;
    const uint64_t k2 = k << 1;
    uint64_t jtop = 0, jbot = 1;
    if (k2 && k < a.kmax) {
        const uint64_t q1 = div_magic(k2, a.m_ylo, a.l_ylo);    // floor(k / y_lo)
        const uint64_t q2 = div_magic(k2, b.m_y2p1, b.l_y2p1);  // floor(k / (y2+1))
        const uint64_t jc = a.JC0[e], jlo = a.JLO[e];
        jtop = jc < q1 ? jc : q1;
        jbot = (q2 + 1) > jlo ? (q2 + 1) : jlo;
    }
    const uint64_t cnt = jtop >= jbot ? jtop - jbot + 1 : 0;
    int64_t add = 0;
    if (cnt && cnt <= kLaneTerms) {
        // j < 2^32 here (j <= sqrt(k))
        int64_t h[kShareLevels] = {};
        for (uint32_t j0 = (uint32_t)jbot; j0 <= (uint32_t)jtop; j0 += 4u) {
            const uint32_t j[4] = {j0, j0 + 1u, j0 + 2u, j0 + 3u};
            const bool ok[4] = {true, j0 + 1u <= (uint32_t)jtop, j0 + 2u <= (uint32_t)jtop,
                                j0 + 3u <= (uint32_t)jtop};
            add += block_M4(a, k2, b.y1, j, ok, h);
        }
        if (jtop >= 2u) {
            const uint32_t em = a.EMIT[e];
            if (em)
                emit_levels(a.S, e, em, jbot, jtop, h, 0);
        }
    }
    if (k2) {
        const uint64_t yc = a.YCE[e];
        if (yc >= b.y1 && yc <= b.y2) {
            const int64_t Myc = block_M(a.segoff, a.Mloc, yc - b.y1);
            add -= (int64_t)((uint64_t)Myc * a.JC0[e]);
        }
    }
    if (add)
        atomicAdd(reinterpret_cast<unsigned long long *>(a.S + e), (unsigned long long)add);
    // heavy entries: ceil(cnt / kSparseItem) chunk records, slots taken with
    // one atomic per warp
    const uint32_t nch = cnt > kLaneTerms ? (uint32_t)((cnt + kSparseItem - 1) / kSparseItem) : 0u;
    uint32_t incl = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t nb = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o)
            incl += nb;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0)
        return;
    uint32_t base = 0;
    if (lane == 31)
        base = atomicAdd(a.qlen, total);
    base = __shfl_sync(0xffffffffu, base, 31);
    uint32_t slot = base + incl - nch;
    for (uint32_t c = 0; c < nch; ++c, ++slot) {
        const uint64_t jt = jtop - (uint64_t)c * kSparseItem;
        const uint64_t n = jt - jbot + 1 < (uint64_t)kSparseItem ? jt - jbot + 1 : kSparseItem;
        if (slot < a.qcap)
            a.queue[slot] = make_uint4((uint32_t)e, (uint32_t)jt, (uint32_t)(jt >> 32),
                                       (uint32_t)n);
        else
            atomicOr(a.err, kErrQueue);
    }
}

// The posted chunks, one warp per chunk (grid-stride): lanes over its j,
// four terms per lane per round (sixteen loads in flight per lane).
__global__ void __launch_bounds__(256) sparse_chunk_kernel(SparseBlockArgs b, SparseArgs a)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t q = *a.qlen;
    const uint32_t total = q < a.qcap ? q : a.qcap;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nw) {
        const uint4 r = a.queue[w];
        const uint64_t e = r.x;
        const uint64_t jt = (uint64_t)r.y | ((uint64_t)r.z << 32);
        const uint32_t n = r.w;  // terms j = jt - n + 1 .. jt; jt <= sqrt(k) < 2^32
        const uint64_t k2 = a.K[e] << 1;
        int64_t acc = 0, h[kShareLevels] = {};
        for (uint32_t i = lane; i < n; i += 128u) {
            const uint32_t j[4] = {(uint32_t)jt - i, (uint32_t)jt - i - 32u, (uint32_t)jt - i - 64u,
                                   (uint32_t)jt - i - 96u};
            const bool ok[4] = {true, i + 32u < n, i + 64u < n, i + 96u < n};
            acc += block_M4(a, k2, b.y1, j, ok, h);
        }
        // a lane's j share one residue mod 32: the level sums fall out of the
        // reduction (the per-lane ones are not needed)
        acc = warp_sum_levels(acc, (uint32_t)jt, lane, h);
        if (lane == ((uint32_t)jt & 31u)) {
            atomicAdd(reinterpret_cast<unsigned long long *>(a.S + e), (unsigned long long)acc);
            const uint32_t em = a.EMIT[e];
            if (em)
                emit_levels(a.S, e, em, jt - n + 1, jt, h, 0);
        }
    }
}

// Quotient of a gathered term inside a tile.  With R = k - t1 j, the term's
// y - t1 = floor(R / j) and 0 <= R < len j, len <= 2^15, so the quotient Q is
// below 2^15.  The float path estimates it without any conversion unit (on
// this part the 64-bit integer -> float conversion runs on the FP64 pipe):
// R and j come from float_of (exact 16- and 23-bit pieces, two roundings:
// relative error <= 2^-23) at the start of a lane's run and are then stepped
// with one fused multiply-add each from the run's start (R_i = R_0 + i dR,
// j_i = j_0 + i dj, one rounding each, so the error stays within 2^-22 of the
// current value, or, where R falls, within 2^-22 R_0); 1/j is rcp.approx
// (<= 1 ulp).  So R (1/j) is within 1/40 of Q (relative errors near 2^-21 on
// values below 2^15), and rounding R (1/j) - 17/32 to an integer (adding
// 1.5 2^23 makes the float addition round to an integer, read back from the
// bits) gives floor(Q) or floor(Q) - 1; the exact remainder R - q j, in
// [0, 2j), decides the step.  kQuotF32 takes the remainder in 32 bits (every
// j < 2^31, so 2j < 2^32), kQuotF64 in 64.  The result is clamped to
// lim = len - 1, which keeps the shared-memory index inside the tile whatever
// the estimate.  kQuotMagic keeps the 64-bit multiply-high path.
constexpr int kQuotMagic = 0, kQuotF32 = 1, kQuotF64 = 2;
static_assert(kGatherTile <= 32768, "the quotient bound needs tiles of at most 2^15 y");

// v (< 2^55) as a float with relative error at most 2^-23, from exact pieces:
// a 23-bit integer p is the float with bits 0x4B000000 | p, less 2^23.
__device__ __forceinline__ float float_of(uint64_t v)
{
    const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
    const float fh = __int_as_float(0x4B000000 | hi) - 8388608.0f;
    const float fa = __int_as_float(0x4B000000 | (lo >> 16)) - 8388608.0f;
    const float fb = __int_as_float(0x4B000000 | (lo & 0xffffu)) - 8388608.0f;
    return __fmaf_rn(fh, 4294967296.0f, __fmaf_rn(fa, 65536.0f, fb));
}

template <int kQuot>
__device__ __forceinline__ uint32_t tile_quot(float Rf, float jf, uint64_t R, uint32_t j,
                                              uint32_t lim)
{
    float rj;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rj) : "f"(jf));
    const float t = __fadd_rn(__fmaf_rn(Rf, rj, -0.53125f), 12582912.0f);
    const int32_t qs = __float_as_int(t) - 0x4B400000;  // floor(Q) or floor(Q) - 1 (>= -1)
    uint32_t q = (uint32_t)qs;
    if (kQuot == kQuotF32) {
        const uint32_t rem = (uint32_t)R - q * j;
        q += rem >= j ? 1u : 0u;
    } else {
        const uint64_t rem = R - (uint64_t)((int64_t)qs * (int64_t)j);
        q += rem >= j ? 1u : 0u;
    }
    return q < lim ? q : lim;
}

// The lane-per-entry part of the tile kernel: entry e's cnt (<= kLaneTerms)
// terms j = j0 .. j0 + cnt - 1 in the staged tile, one lane, and its level
// sums for the entries 2^s x it feeds.
template <int kQuot>
__device__ __forceinline__ void tile_lane_entry(uint64_t *S, const uint32_t *EMIT, const uint64_t *MG,
                                             uint64_t t1, uint32_t lim, int64_t base, uint32_t e,
                                             uint64_t k2, uint32_t j0, uint32_t cnt)
{
    extern __shared__ int16_t Mt[];
    // acc: the sum; h[s - 1]: the part over j = 0 mod 2^s (for the entries
    // 2^s x this one feeds)
    int acc = 0, h[kShareLevels] = {};
    if (kQuot == kQuotMagic) {
        const uint32_t t1lo = (uint32_t)t1;
        for (uint32_t i = 0; i < cnt; ++i) {
            const uint32_t j = j0 + i;
            const uint64_t y = div_magic(k2, MG[j], 32u - __clz(j - 1u));
            const int v = Mt[(uint32_t)y - t1lo];
            acc += v;
#pragma unroll
            for (uint32_t l = 0; l < kShareLevels; ++l)
                h[l] += (j & ((2u << l) - 1u)) ? 0 : v;
        }
    } else {
        // R = k - t1 j falls by t1 per step of j
        uint64_t R = (k2 >> 1) - t1 * (uint64_t)j0;
        const float Rf0 = float_of(R), jf0 = float_of(j0), t1f = float_of(t1);
        float fi = 0.0f;
        for (uint32_t i = 0; i < cnt; ++i, R -= t1, fi += 1.0f) {
            const float Rf = __fmaf_rn(fi, -t1f, Rf0), jf = __fadd_rn(jf0, fi);
            const uint32_t j = j0 + i;
            const int v = Mt[tile_quot<kQuot>(Rf, jf, R, j, lim)];
            acc += v;
#pragma unroll
            for (uint32_t l = 0; l < kShareLevels; ++l)
                h[l] += (j & ((2u << l) - 1u)) ? 0 : v;
        }
    }
    atomicAdd(reinterpret_cast<unsigned long long *>(S + e),
              (unsigned long long)((int64_t)acc + (int64_t)cnt * base));
    const uint32_t jl = j0 + cnt - 1u;
    const uint32_t em = jl >= 2u ? EMIT[e] : 0u;
    if (em) {
        int64_t hl[kShareLevels];
#pragma unroll
        for (uint32_t l = 0; l < kShareLevels; ++l)
            hl[l] = h[l];
        emit_levels(S, e, em, j0, jl, hl, base);
    }
}

// The end of the warp-per-entry loop for an entry that feeds entries 2^s x:
// a lane's j share one residue mod 32 (lanes idle past cns add zero), so the
// level sums fall out of the reduction in the lane whose j are 0 mod 32.
__device__ __forceinline__ void tile_warp_emit(uint64_t *S, uint32_t e, uint32_t em, int64_t acc,
                                            uint32_t jts, uint32_t cns, uint32_t lane,
                                            int64_t base)
{
    int64_t h[kShareLevels];
    const int64_t tot = warp_sum_levels(acc, jts, lane, h);
    if (lane == (jts & 31u)) {
        atomicAdd(reinterpret_cast<unsigned long long *>(S + e),
                  (unsigned long long)(tot + (int64_t)cns * base));
        emit_levels(S, e, em, jts - cns + 1u, jts, h, base);
    }
}

// Shared-memory gather path for the low, dense part of a block.  A work item
// is one tile [t1, t1+len) of y and a range of entries of one target.  The
// tile's M(y) - M(t1-1) is staged in shared memory as int16 (|value| <= 3/4
// of the tile); every entry with gathered terms in the tile -- j in
// [max(jlo, floor(k/(t1+len))+1), min(jcur, floor(k/t1))] -- adds
// sum_j M(floor(k/j)) = sum_j (staged value) + count * M(t1-1).  Warps take
// 32 entries at a time (lane per entry for the range), then each entry with
// terms in turn, lanes over its j.
// Three 512-thread CTAs per SM (64 KiB of tile each): registers capped to fit.
// kQuot picks how a term's quotient is taken (tile_quot above).
template <int kQuot>
__global__ void __launch_bounds__(512, 3) gather_tile_kernel(GatherArgs a)
{
    extern __shared__ int16_t Mt[];  // kGatherTile
    __shared__ uint32_t s_item;
    __shared__ int64_t s_base;
    __shared__ int32_t s_delta[kGatherTile / kSegY];
    __shared__ uint64_t s_mbar;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    uint32_t staged = 0xffffffffu, phase = 0;
    if (threadIdx.x == 0) {
        mbar_init(&s_mbar);
        fence_proxy_async_smem();
    }
    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(a.counter, 1u);
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= a.nitems)
            break;
        const GatherItem I = a.items[it];
        const GatherTile T = a.tiles[I.tile];
        if (I.tile != staged) {
            // stage M(y) - M(t1 - 1) of the tile: one bulk asynchronous copy
            // of the block's int16 values (whole 16-byte units; the buffer is
            // padded), then each 2048-y segment's offset added in place
            const uint64_t o1 = T.t1 - a.y1;  // a multiple of the tile length
            const uint32_t n8 = (T.len + 7u) & ~7u;
            if (threadIdx.x == 0) {
                fence_proxy_async_smem();  // earlier readers of Mt passed the barrier
                mbar_arrive_expect(&s_mbar, n8 * 2u);
                bulk_copy_g2s(Mt, a.Mloc + o1, n8 * 2u, &s_mbar);
                s_base = (o1 == 0) ? a.segoff[0] : block_M(a.segoff, a.Mloc, o1 - 1);
            }
            __syncthreads();
            const uint32_t nseg = (T.len + kSegY - 1) / kSegY;
            if (threadIdx.x < nseg)
                s_delta[threadIdx.x] =
                    (int32_t)(a.segoff[(o1 >> kSegShift) + threadIdx.x] - s_base);
            if (__syncthreads_or(!mbar_wait(&s_mbar, phase & 1u))) {
                if (threadIdx.x == 0)
                    atomicOr(a.err, kErrTimeout);
                mbar_wait(&s_mbar, phase & 1u);
                return;
            }
            ++phase;
            uint32_t *Mw = reinterpret_cast<uint32_t *>(Mt);
            for (uint32_t i = threadIdx.x; i < n8 / 2u; i += blockDim.x) {
                const uint32_t v = Mw[i];
                const int32_t d = s_delta[(2u * i) >> kSegShift];
                const uint32_t lo = (uint32_t)((int32_t)(int16_t)(v & 0xffffu) + d) & 0xffffu;
                const uint32_t hi = (uint32_t)((int32_t)(int16_t)(v >> 16) + d);
                Mw[i] = lo | (hi << 16);
            }
            staged = I.tile;
        }
        __syncthreads();
        const int64_t base = s_base;
        for (uint32_t eb = I.e0 + (uint32_t)warp * 32u; eb < I.e1; eb += (uint32_t)nwarp * 32u) {
            const uint32_t e = eb + (uint32_t)lane;
            uint64_t k2 = 0, jt = 0, jb = 1;
            if (e < I.e1) {
                k2 = a.K[e] << 1;
                const uint64_t jc = a.JCUR[e], jlo = a.JLO[e];
                const uint64_t q1 = div_magic(k2, T.m1, T.l1);  // floor(k / t1)
                const uint64_t q2 = div_magic(k2, T.m2, T.l2);  // floor(k / (t1+len))
                jt = jc < q1 ? jc : q1;
                jb = (q2 + 1) > jlo ? (q2 + 1) : jlo;
            }
            // j < 2^32 (j <= sqrt(k) < 2^32) and y - t1 < 2^15: 32-bit loop
            // counters and offsets
            const uint32_t cnt = jt >= jb ? (uint32_t)(jt - jb + 1) : 0u;
            const uint32_t t1lo = (uint32_t)T.t1, lim = T.len - 1u;
            // entries with few terms: one lane each, serially
            if (cnt > 0 && cnt <= kLaneTerms)
                tile_lane_entry<kQuot>(a.S, a.EMIT, a.MG, T.t1, lim, base, e, k2, (uint32_t)jb,
                                       cnt);
            // entries with many terms: the whole warp, lanes over j
            uint32_t mask = __ballot_sync(0xffffffffu, cnt > kLaneTerms);
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                const uint32_t jts = (uint32_t)__shfl_sync(0xffffffffu, jt, src);
                const uint32_t cns = __shfl_sync(0xffffffffu, cnt, src);
                const uint64_t k2s = __shfl_sync(0xffffffffu, k2, src);
                int acc = 0;
                if ((uint32_t)lane < cns) {
                    // lanes over j descending, 32 apart
                    uint32_t j = jts - (uint32_t)lane;
                    if (kQuot == kQuotMagic) {
                        // the magic pointer is walked rather than indexed
                        // (measured faster)
                        const uint64_t *mp = a.MG + j;
                        for (uint32_t i = (uint32_t)lane; i < cns; i += 32u, j -= 32u, mp -= 32) {
                            const uint64_t y = div_magic(k2s, *mp, 32u - __clz(j - 1u));
                            acc += Mt[(uint32_t)y - t1lo];
                        }
                    } else {
                        // R = k - t1 j rises by 32 t1 per step, j falls by 32
                        uint64_t R = (k2s >> 1) - T.t1 * (uint64_t)j;
                        const uint64_t dR = T.t1 << 5;
                        const float Rf0 = float_of(R), jf0 = float_of(j), dRf = float_of(dR);
                        float fi = 0.0f;
                        for (uint32_t i = (uint32_t)lane; i < cns;
                             i += 32u, j -= 32u, R += dR, fi += 1.0f) {
                            const float Rf = __fmaf_rn(fi, dRf, Rf0);
                            const float jf = __fmaf_rn(fi, -32.0f, jf0);
                            acc += Mt[tile_quot<kQuot>(Rf, jf, R, j, lim)];
                        }
                    }
                }
                // the entry's sum; if it feeds entries 2^s x, also its level
                // sums (tile_warp_emit)
                const uint32_t ems = a.EMIT[eb + src];  // one address: warp-uniform
                if (ems) {
                    tile_warp_emit(a.S, eb + src, ems, (int64_t)acc, jts, cns, (uint32_t)lane,
                                   base);
                } else {
                    const int64_t tot = warp_sum_i64((int64_t)acc);
                    if (lane == 0)
                        atomicAdd(reinterpret_cast<unsigned long long *>(a.S + eb + src),
                                  (unsigned long long)(tot + (int64_t)cns * base));
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Resolve (Sec. 2): for x = X down to 1,
//   M[x] = 1 - S[x] - sum_{j=2}^{floor(X/x)} M[x j]   (mod 2^64),
// in three phases, one CTA per target, r = min(floor(sqrt(X)), kResolveSmall):
//  A. x > r level by level: all x with the same q = floor(X/x) only read
//     entries of smaller q (parallel over the x of a level);
//  B. for x <= r, the part of the sum with x j > r (all known after A),
//     parallel over x;
//  C. x = r down to 1, the remaining sum over x j <= r from shared memory.
// ---------------------------------------------------------------------------
constexpr int kResolveSmall = 4096;

__global__ void __launch_bounds__(1024) resolve_kernel(const QueryDev *__restrict__ qs,
                                                       const uint64_t *__restrict__ S,
                                                       const uint64_t *__restrict__ K,
                                                       uint64_t *__restrict__ R)
{
    __shared__ uint64_t Tsm[kResolveSmall + 1];  // phase B sums, then phase C values
    const QueryDev Q = qs[blockIdx.x];
    const uint64_t X = Q.X, base = Q.off;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    uint64_t r = (uint64_t)sqrt((double)X);
    while (r * r > X)
        --r;
    while ((r + 1) * (r + 1) <= X)
        ++r;
    if (r > (uint64_t)kResolveSmall)
        r = kResolveSmall;
    // A
    uint64_t xhi = X;
    while (xhi > r) {
        const uint64_t qv = X / xhi;
        uint64_t xlo = X / (qv + 1) + 1;
        if (xlo <= r)
            xlo = r + 1;
        const uint64_t size = xhi - xlo + 1;
        if (size >= blockDim.x || qv <= 8) {
            for (uint64_t x = xlo + threadIdx.x; x <= xhi; x += blockDim.x) {
                uint64_t acc = 0;
                for (uint64_t j = 2; j <= qv; ++j)
                    acc += R[base + x * j - 1];
                const uint64_t e = base + x - 1;
                R[e] = (K[e] == 1) ? 1ull : 1ull - S[e] - acc;
            }
        } else {
            for (uint64_t x = xlo + warp; x <= xhi; x += nwarp) {
                uint64_t acc = 0;
                for (uint64_t j = 2 + lane; j <= qv; j += 32)
                    acc += R[base + x * j - 1];
                acc = warp_sum_u64(acc);
                if (lane == 0) {
                    const uint64_t e = base + x - 1;
                    R[e] = (K[e] == 1) ? 1ull : 1ull - S[e] - acc;
                }
            }
        }
        __syncthreads();
        xhi = xlo - 1;
    }
    // B: Tsm[x] = 1 - S[x] - sum_{j >= 2, x j > r} M[x j]
    for (uint64_t x = 1 + warp; x <= r; x += nwarp) {
        const uint64_t jmax = X / x;
        uint64_t j0 = r / x + 1;
        if (j0 < 2)
            j0 = 2;
        uint64_t acc = 0;
        for (uint64_t j = j0 + lane; j <= jmax; j += 32)
            acc += R[base + x * j - 1];
        acc = warp_sum_u64(acc);
        if (lane == 0) {
            const uint64_t e = base + x - 1;
            Tsm[x] = (K[e] == 1) ? 1ull : 1ull - S[e] - acc;
        }
    }
    __syncthreads();
    // C: the rest, x j <= r, in decreasing x (one warp, values in Tsm)
    if (warp == 0) {
        for (uint64_t x = r; x >= 1; --x) {
            const uint64_t e = base + x - 1;
            uint64_t acc = 0;
            if (K[e] != 1) {
                const uint64_t jmax = r / x;
                for (uint64_t j = 2 + lane; j <= jmax; j += 32)
                    acc += Tsm[x * j];
                acc = warp_sum_u64(acc);
            }
            const uint64_t v = Tsm[x] - acc;
            __syncwarp();
            if (lane == 0) {
                Tsm[x] = v;
                R[e] = v;
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// Exchange of window sums (Sec. 2-3: a window's contributions are affine in
// its carry C = M(y_first - 1)).  An exchange buffer holds every entry's
// 64-bit sum as two int64 words, its low and its high 32-bit half, so that
// element-wise sums of such buffers over up to 2^31 windows never overflow
// a signed 64-bit word, whatever adds them.
// ---------------------------------------------------------------------------
// halves[2i] += low, halves[2i+1] += high half of S_loc[i] + C coef[i] (mod 2^64).
__global__ void window_accumulate_kernel(const uint64_t *__restrict__ S,
                                         const uint64_t *__restrict__ coef, uint64_t C,
                                         uint64_t X, int64_t *__restrict__ halves)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < X;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = S[i] + C * coef[i];
        halves[2 * i] += (int64_t)(v & 0xffffffffull);
        halves[2 * i + 1] += (int64_t)(v >> 32);
    }
}

// S[i] = halves[2i] + 2^32 halves[2i+1] (mod 2^64).
__global__ void halves_to_sums_kernel(const int64_t *__restrict__ halves, uint64_t X,
                                      uint64_t *__restrict__ S)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < X;
         i += (uint64_t)gridDim.x * blockDim.x)
        S[i] = (uint64_t)halves[2 * i] + ((uint64_t)halves[2 * i + 1] << 32);
}

static unsigned grid_for(uint64_t n)
{
    const uint64_t b = (n + 255) / 256;
    return (unsigned)(b < 152 * 16 ? (b ? b : 1) : 152 * 16);
}

int window_accumulate_enqueue(const uint64_t *S, const uint64_t *coef, uint64_t C, uint64_t X,
                              int64_t *halves, cudaStream_t s)
{
    if (X == 0)
        return 0;
    window_accumulate_kernel<<<grid_for(X), 256, 0, s>>>(S, coef, C, X, halves);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int halves_to_sums_enqueue(const int64_t *halves, uint64_t X, uint64_t *S, cudaStream_t s)
{
    if (X == 0)
        return 0;
    halves_to_sums_kernel<<<grid_for(X), 256, 0, s>>>(halves, X, S);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
int magic_table_enqueue(uint64_t *MG, uint64_t nd, cudaStream_t s)
{
    if (nd == 0)
        return 0;
    uint64_t blocks = (nd + 255) / 256;
    if (blocks > 152 * 64)
        blocks = 152 * 64;
    magic_table_kernel<<<(unsigned)blocks, 256, 0, s>>>(MG, nd);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int dense_list_enqueue(const int8_t *mu_aux, uint64_t ydense, const uint64_t *MG, uint64_t *dl_m,
                       uint16_t *dl_yo, uint2 *dl_cnt, cudaStream_t s)
{
    const uint64_t nchunks = ydense / kChunk + 1;
    dense_list_kernel<<<(unsigned)nchunks, 256, 0, s>>>(mu_aux, ydense, MG, dl_m, dl_yo, dl_cnt);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int dense_update_enqueue(const DenseArgs &a, cudaStream_t s)
{
    static std::atomic<uint64_t> attr_devs{0};
    const size_t smem = (size_t)kDenseChunks * kChunkCapPad * (8 + 2);
    const uint64_t dbit = device_bit();
    if (attrs_needed(attr_devs, dbit)) {
        cudaFuncSetAttribute(dense_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        attrs_done(attr_devs, dbit);
    }
    if (a.nitems == 0)
        return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, dense_update_kernel, kDenseThreads, smem);
    if (per < 1)
        per = 1;
    if (a.ctas_per_sm && (int)a.ctas_per_sm < per)
        per = (int)a.ctas_per_sm;
    uint32_t grid = (uint32_t)(sms * per);
    if (grid > a.nitems)
        grid = a.nitems;
    cudaMemsetAsync(a.counter, 0, 4, s);
    dense_update_kernel<<<grid, kDenseThreads, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int sparse_block_enqueue(const SparseBlockArgs &b, const SparseArgs &a, cudaStream_t s)
{
    const unsigned pb = (unsigned)((a.nent + 255) / 256);
    cudaMemsetAsync(a.qlen, 0, 4, s);
    sparse_range_kernel<<<pb, 256, 0, s>>>(b, a);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sparse_chunk_kernel<<<sms * 8, 256, 0, s>>>(b, a);
    return cudaGetLastError() == cudaSuccess ? 2 : -1;
}

// ---------------------------------------------------------------------------
// Entries with k >= 2^63 (one CTA row per entry, grid.y = entries): the
// block's direct terms y in [y1, min(y2, s)] and gathered terms j in
// [max(jlo, floor(k/(y2+1))+1), min(jhi, floor(k/y1))], numbered as one unit
// range; each thread takes kWidePer consecutive units.  Quotients are exact
// 128-by-64 divisions; sums are mod 2^64 (the direct differences are taken
// on the low words, which is the same mod 2^64).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kWideThreads) wide_update_kernel(WideArgs a)
{
    __shared__ uint64_t red[kWideThreads / 32];
    const WideEntry W = a.W[blockIdx.y];
    const unsigned __int128 k = ((unsigned __int128)W.k_hi << 64) | W.k_lo;
    uint64_t nd, ja, ng;
    wide_ranges(W, a.y1, a.y2, &nd, &ja, &ng);
    const uint64_t units = nd + ng;
    const uint64_t u0 = (uint64_t)blockIdx.x * kWideUnitsPerCta + (uint64_t)threadIdx.x * kWidePer;
    const uint64_t u1 = u0 + kWidePer < units ? u0 + kWidePer : units;
    uint64_t acc = 0;
    uint64_t u = u0;
    if (u < u1 && u < nd) {
        // direct: y = y1 + u, consecutive; q = floor(k/y) carried along
        uint64_t y = a.y1 + u;
        uint64_t q = (uint64_t)(k / y);
        const uint64_t ue = u1 < nd ? u1 : nd;
        for (; u < ue; ++u, ++y) {
            const uint64_t qn = (uint64_t)(k / ((unsigned __int128)y + 1));
            const uint64_t i = y - a.y1;
            const int64_t M = a.segoff[i >> kSegShift] + (int64_t)a.Mloc[i];
            acc += (uint64_t)M * (q - qn);
            q = qn;
        }
    }
    for (; u < u1; ++u) {
        // gathered: y = floor(k/j) in [y1, y2]
        const uint64_t j = ja + (u - nd);
        const uint64_t i = (uint64_t)(k / j) - a.y1;
        acc += (uint64_t)(a.segoff[i >> kSegShift] + (int64_t)a.Mloc[i]);
    }
    acc = warp_sum_u64(acc);
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int w = 0; w < kWideThreads / 32; ++w)
            t += red[w];
        if (t)
            atomicAdd(reinterpret_cast<unsigned long long *>(a.S + W.e), (unsigned long long)t);
    }
}

__global__ void table_lookup_kernel(const uint64_t *__restrict__ pairs, uint32_t count,
                                    const int16_t *__restrict__ Mloc,
                                    const int64_t *__restrict__ segoff, uint64_t *__restrict__ R)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count)
        return;
    const uint64_t y = pairs[2 * i + 1];
    R[pairs[2 * i]] = (uint64_t)(segoff[(y - 1) >> kSegShift] + (int64_t)Mloc[y - 1]);
}

__global__ void carry_from_table_kernel(const int16_t *__restrict__ Mloc,
                                        const int64_t *__restrict__ segoff, uint64_t y,
                                        int64_t *__restrict__ out)
{
    *out = segoff[(y - 1) >> kSegShift] + (int64_t)Mloc[y - 1];
}

int carry_from_table_enqueue(const int16_t *Mloc, const int64_t *segoff, uint64_t y,
                             int64_t *out, cudaStream_t s)
{
    carry_from_table_kernel<<<1, 1, 0, s>>>(Mloc, segoff, y, out);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int table_lookup_enqueue(const uint64_t *pairs, uint32_t count, const int16_t *Mloc,
                         const int64_t *segoff, uint64_t *R, cudaStream_t s)
{
    if (count == 0)
        return 0;
    table_lookup_kernel<<<(count + 255) / 256, 256, 0, s>>>(pairs, count, Mloc, segoff, R);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int wide_update_enqueue(const WideArgs &a, uint32_t nw, uint32_t grid_x, cudaStream_t s)
{
    if (nw == 0 || grid_x == 0)
        return 0;
    wide_update_kernel<<<dim3(grid_x, nw), kWideThreads, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int gather_tiles_enqueue(const GatherArgs &a, cudaStream_t s)
{
    static std::atomic<uint64_t> attr_devs{0};
    const int smem = kGatherTile * 2;
    const uint64_t dbit = device_bit();
    if (attrs_needed(attr_devs, dbit)) {
        cudaFuncSetAttribute(gather_tile_kernel<kQuotMagic>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(gather_tile_kernel<kQuotF32>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(gather_tile_kernel<kQuotF64>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attrs_done(attr_devs, dbit);
    }
    if (a.nitems == 0)
        return 0;
    void (*kern)(GatherArgs) = a.quot == kQuotF32   ? gather_tile_kernel<kQuotF32>
                               : a.quot == kQuotF64 ? gather_tile_kernel<kQuotF64>
                                                    : gather_tile_kernel<kQuotMagic>;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = a.threads == 256 ? 256 : 512;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem);
    if (per < 1)
        per = 1;
    if (a.ctas_per_sm && (int)a.ctas_per_sm < per)
        per = (int)a.ctas_per_sm;
    uint32_t grid = (uint32_t)(sms * per);
    if (grid > a.nitems)
        grid = a.nitems;
    cudaMemsetAsync(a.counter, 0, 4, s);
    kern<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int resolve_enqueue(const QueryDev *qs, uint32_t nq, const uint64_t *S, const uint64_t *K,
                    uint64_t *R, cudaStream_t s)
{
    resolve_kernel<<<nq, 1024, 0, s>>>(qs, S, K, R);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace mert
