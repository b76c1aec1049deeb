// Interval scan: M(y) for every y of [y_first, y_last] from a known
// M(y_first - 1), by the sieve and prefix scan (steps a1 + a2, Sec. 3), and
// the extremes of M(y) and of M(y)/sqrt(y) over the interval -- the search
// that Sec. 6 of the paper runs around its candidate to find the new extreme
// value of M(n)/sqrt(n).  Ratios are compared exactly: for M1, M2 >= 0,
// M1/sqrt(y1) > M2/sqrt(y2) iff M1^2 y2 > M2^2 y1 (128-bit products).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/libmertens.h"
#include "common.cuh"
#include "internal.h"

using namespace mert;

namespace {

typedef unsigned __int128 u128;

// Running extremes; ties go to the smaller y.
struct Ext {
    int64_t mx, mn;    // largest and smallest M(y)
    uint64_t ymx, ymn;
    int64_t rpM, rnM;  // M at the largest and smallest M(y)/sqrt(y)
    uint64_t rpy, rny;
};

// a/sqrt(ya) > b/sqrt(yb) exactly
__host__ __device__ inline bool ratio_gt(int64_t a, uint64_t ya, int64_t b, uint64_t yb)
{
    if ((a >= 0) != (b >= 0))
        return a >= 0;
    const u128 aa = (u128)(uint64_t)(a >= 0 ? a : -a), bb = (u128)(uint64_t)(b >= 0 ? b : -b);
    const u128 l = aa * aa * yb, r = bb * bb * ya;
    return a >= 0 ? l > r : l < r;
}

__host__ __device__ inline void ext_init(Ext &e)
{
    e.mx = INT64_MIN;
    e.mn = INT64_MAX;
    e.ymx = e.ymn = e.rpy = e.rny = UINT64_MAX;
    e.rpM = e.rnM = 0;
}

__host__ __device__ inline void ext_point(Ext &e, int64_t M, uint64_t y)
{
    if (M > e.mx || (M == e.mx && y < e.ymx)) {
        e.mx = M;
        e.ymx = y;
    }
    if (M < e.mn || (M == e.mn && y < e.ymn)) {
        e.mn = M;
        e.ymn = y;
    }
    if (e.rpy == UINT64_MAX || ratio_gt(M, y, e.rpM, e.rpy) ||
        (!ratio_gt(e.rpM, e.rpy, M, y) && y < e.rpy)) {
        e.rpM = M;
        e.rpy = y;
    }
    if (e.rny == UINT64_MAX || ratio_gt(e.rnM, e.rny, M, y) ||
        (!ratio_gt(M, y, e.rnM, e.rny) && y < e.rny)) {
        e.rnM = M;
        e.rny = y;
    }
}

__host__ __device__ inline void ext_merge(Ext &e, const Ext &o)
{
    if (o.ymx != UINT64_MAX && (o.mx > e.mx || (o.mx == e.mx && o.ymx < e.ymx))) {
        e.mx = o.mx;
        e.ymx = o.ymx;
    }
    if (o.ymn != UINT64_MAX && (o.mn < e.mn || (o.mn == e.mn && o.ymn < e.ymn))) {
        e.mn = o.mn;
        e.ymn = o.ymn;
    }
    if (o.rpy != UINT64_MAX &&
        (e.rpy == UINT64_MAX || ratio_gt(o.rpM, o.rpy, e.rpM, e.rpy) ||
         (!ratio_gt(e.rpM, e.rpy, o.rpM, o.rpy) && o.rpy < e.rpy))) {
        e.rpM = o.rpM;
        e.rpy = o.rpy;
    }
    if (o.rny != UINT64_MAX &&
        (e.rny == UINT64_MAX || ratio_gt(e.rnM, e.rny, o.rnM, o.rny) ||
         (!ratio_gt(o.rnM, o.rny, e.rnM, e.rny) && o.rny < e.rny))) {
        e.rnM = o.rnM;
        e.rny = o.rny;
    }
}

constexpr int kExtThreads = 256;
constexpr uint32_t kExtPer = 64;  // y per thread

__device__ inline Ext ext_shfl(const Ext &e, int src)
{
    Ext o;
    o.mx = __shfl_down_sync(0xffffffffu, e.mx, src);
    o.mn = __shfl_down_sync(0xffffffffu, e.mn, src);
    o.ymx = __shfl_down_sync(0xffffffffu, e.ymx, src);
    o.ymn = __shfl_down_sync(0xffffffffu, e.ymn, src);
    o.rpM = __shfl_down_sync(0xffffffffu, e.rpM, src);
    o.rnM = __shfl_down_sync(0xffffffffu, e.rnM, src);
    o.rpy = __shfl_down_sync(0xffffffffu, e.rpy, src);
    o.rny = __shfl_down_sync(0xffffffffu, e.rny, src);
    return o;
}

// One block of M(y): every CTA reduces kExtThreads * kExtPer consecutive y to
// one record in part[blockIdx.x].
__global__ void __launch_bounds__(kExtThreads) block_extremes_kernel(
    uint64_t y1, uint64_t len, const int16_t *__restrict__ Mloc,
    const int64_t *__restrict__ segoff, Ext *__restrict__ part)
{
    __shared__ Ext sh[kExtThreads / 32];
    Ext e;
    ext_init(e);
    const uint64_t i0 = ((uint64_t)blockIdx.x * kExtThreads + threadIdx.x) * kExtPer;
    const uint64_t i1 = i0 + kExtPer < len ? i0 + kExtPer : len;
    for (uint64_t i = i0; i < i1; ++i)
        ext_point(e, segoff[i >> kSegShift] + (int64_t)Mloc[i], y1 + i);
    for (int o = 16; o > 0; o >>= 1) {
        const Ext q = ext_shfl(e, o);
        ext_merge(e, q);
    }
    if ((threadIdx.x & 31) == 0)
        sh[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kExtThreads / 32; ++w)
            ext_merge(e, sh[w]);
        part[blockIdx.x] = e;
    }
}

// All partial records into part[0] (one CTA, strided then a serial pass).
__global__ void __launch_bounds__(kExtThreads) merge_extremes_kernel(Ext *part, uint32_t n)
{
    __shared__ Ext sh[kExtThreads];
    Ext e;
    ext_init(e);
    for (uint32_t i = threadIdx.x; i < n; i += kExtThreads)
        ext_merge(e, part[i]);
    sh[threadIdx.x] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 1; t < kExtThreads; ++t)
            ext_merge(e, sh[t]);
        part[0] = e;
    }
}

}  // namespace

extern "C" {

int mertens_scan_extremes(uint64_t y_first, uint64_t y_last, int64_t carry,
                          mertens_extremes *out, void *stream)
{
    if (!out || y_first == 0 || y_last < y_first || y_last >= (1ull << 62)) {
        set_last_error("mertens_scan_extremes: need 1 <= y_first <= y_last < 2^62 and an output");
        return MERTENS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const Allocator al = current_allocator();
    const uint64_t span = y_last - y_first + 1;
    const uint64_t L = std::min<uint64_t>(1ull << 30, ((span + kSegY - 1) / kSegY) * kSegY);
    const uint64_t nblocks = (span + L - 1) / L;
    const uint64_t per_cta = (uint64_t)kExtThreads * kExtPer;
    const uint64_t ctas = (L + per_cta - 1) / per_cta;
    const uint64_t nparts = nblocks * ctas;
    if (nparts >= (1ull << 32)) {
        set_last_error("mertens_scan_extremes: interval too long");
        return MERTENS_ENOTSUP;
    }
    PrimeTable pt;
    int rc = MERTENS_OK;
    int prc = prime_table_create(&pt, al, y_last, s);
    if (prc == 0)
        prc = sieve_scratch_create(&pt, L);
    if (prc != 0)
        rc = prc == 6 ? MERTENS_ENOTSUP : (prc == 2 ? MERTENS_ENOMEM : MERTENS_ECUDA);
    const uint64_t nseg = sieve_segments(L);
    int16_t *ml = (int16_t *)dev_alloc(al, (L + 2) * 2);
    int32_t *ss = (int32_t *)dev_alloc(al, nseg * 4);
    int64_t *so = (int64_t *)dev_alloc(al, nseg * 8);
    int64_t *cy = (int64_t *)dev_alloc(al, (nblocks + 1) * 8);
    Ext *part = (Ext *)dev_alloc(al, nparts * sizeof(Ext));
    if (rc == MERTENS_OK && (!ml || !ss || !so || !cy || !part))
        rc = MERTENS_ENOMEM;
    if (rc == MERTENS_OK) {
        cudaMemcpyAsync(cy, &carry, 8, cudaMemcpyHostToDevice, s);
        for (uint64_t b = 0; b < nblocks && rc == MERTENS_OK; ++b) {
            SieveLaunch Lc;
            Lc.y1 = y_first + b * L;
            Lc.len = std::min(L, y_last - Lc.y1 + 1);
            Lc.Mloc = ml;
            Lc.segsum = ss;
            Lc.segoff = so;
            Lc.carry_in = cy + b;
            Lc.carry_out = cy + b + 1;
            if (sieve_block_enqueue(&pt, Lc, s) < 0)
                rc = MERTENS_ECUDA;
            // every block launches all `ctas` CTAs; those past a short last
            // block write empty records
            block_extremes_kernel<<<(unsigned)ctas, kExtThreads, 0, s>>>(Lc.y1, Lc.len, ml, so,
                                                                        part + b * ctas);
            if (cudaGetLastError() != cudaSuccess)
                rc = MERTENS_ECUDA;
        }
        if (rc == MERTENS_OK)
            merge_extremes_kernel<<<1, kExtThreads, 0, s>>>(part, (uint32_t)nparts);
        Ext e;
        int64_t last = 0;
        if (rc == MERTENS_OK &&
            (cudaMemcpyAsync(&e, part, sizeof(Ext), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
             cudaMemcpyAsync(&last, cy + nblocks, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
             cudaStreamSynchronize(s) != cudaSuccess))
            rc = MERTENS_ECUDA;
        if (rc == MERTENS_OK) {
            const uint32_t st = sieve_scratch_status(&pt);
            if (st) {
                set_last_error("mertens_scan_extremes: %s", sieve_status_text(st));
                rc = sieve_status_code(st);
            }
        }
        if (rc == MERTENS_OK) {
            out->M_last = last;
            out->M_max = e.mx;
            out->y_M_max = e.ymx;
            out->M_min = e.mn;
            out->y_M_min = e.ymn;
            out->R_max_M = e.rpM;
            out->y_R_max = e.rpy;
            out->R_min_M = e.rnM;
            out->y_R_min = e.rny;
            out->R_max = (double)e.rpM / std::sqrt((double)e.rpy);
            out->R_min = (double)e.rnM / std::sqrt((double)e.rny);
        }
    }
    if (rc == MERTENS_ECUDA)
        set_last_error("mertens_scan_extremes: %s", cudaGetErrorString(cudaGetLastError()));
    dev_free(al, ml, (L + 2) * 2);
    dev_free(al, ss, nseg * 4);
    dev_free(al, so, nseg * 8);
    dev_free(al, cy, (nblocks + 1) * 8);
    dev_free(al, part, nparts * sizeof(Ext));
    if (pt.np)
        prime_table_destroy(&pt);
    return rc;
}

}  // extern "C"
