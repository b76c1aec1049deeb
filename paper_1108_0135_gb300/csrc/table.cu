// Resident M(y) table: the sieve (steps a1 + a2) run once over [1, y_max]
// and kept in device memory, together with the parts of the update that do
// not depend on the target (the divisor magics and the squarefree dense
// list).  Plans made on a table (mertens_plan_on_table) read M(y) from it and
// run only the update and resolve.  The paper sieves per target (Sec. 3);
// keeping the sieve's output resident is what lets many queries share it.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/libmertens.h"
#include "common.cuh"
#include "internal.h"
#include "update.h"

namespace mert {
double plan_dense_factor();
}  // namespace mert

using namespace mert;

namespace {

typedef unsigned __int128 u128;

uint64_t isqrt_u128(u128 v)
{
    u128 r = (u128)std::sqrt((double)v);
    if (r > 0)
        r = (r + v / r) / 2;
    while (r * r > v)
        --r;
    while ((r + 1) * (r + 1) <= v)
        ++r;
    return (uint64_t)r;
}

template <typename T>
T *table_alloc(mertens_table_s *t, size_t count)
{
    const size_t bytes = count * sizeof(T);
    void *p = dev_alloc(t->al, bytes);
    if (p) {
        t->allocs.push_back({p, bytes});
        t->bytes += bytes;
    }
    return (T *)p;
}

}  // namespace

extern "C" {

int mertens_table_create(mertens_table_t *out, uint64_t y_max, mertens_u128 n_max, void *stream)
{
    if (!out)
        return MERTENS_EINVAL;
    *out = nullptr;
    if (y_max == 0 || y_max >= (1ull << 40) || (n_max.lo == 0 && n_max.hi == 0) ||
        n_max.hi >= (1ull << 63)) {
        set_last_error("mertens_table_create: need 1 <= y_max < 2^40 and 1 <= n_max < 2^127");
        return MERTENS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    mertens_table_s *t = new (std::nothrow) mertens_table_s();
    if (!t)
        return MERTENS_ENOMEM;
    t->al = current_allocator();
    cudaGetDevice(&t->device);
    t->y_max = y_max;
    t->n_max_lo = n_max.lo;
    t->n_max_hi = n_max.hi;
    const u128 nm = ((u128)n_max.hi << 64) | n_max.lo;
    const uint64_t r = isqrt_u128(nm);
    // the planner's dense cut-offs stay below the chunk-aligned dc sqrt(n)
    // (or sqrt(n) itself); their quotients k/(yc+1) below sqrt(n)
    const double dc = plan_dense_factor();
    uint64_t yd = (uint64_t)(std::max(dc, 1.0) * std::sqrt((double)nm)) + 2 * kChunk;
    yd = ((yd + kChunk - 1) / kChunk) * kChunk - 1;
    t->ydense = std::min(yd, y_max);
    t->mg_n = std::max(t->ydense, r) + 2;

    const uint64_t nseg = sieve_segments(y_max);
    const uint64_t nchunks = dense_chunks(t->ydense);
    t->Mloc = table_alloc<int16_t>(t, y_max + 16);  // gather tiles copy whole 16-byte units
    t->segoff = table_alloc<int64_t>(t, nseg);
    t->MG = table_alloc<uint64_t>(t, t->mg_n + 1);
    t->dl_m = table_alloc<uint64_t>(t, nchunks * kChunkCapPad);
    t->dl_yo = table_alloc<uint16_t>(t, nchunks * kChunkCapPad);
    t->dl_cnt = table_alloc<uint2>(t, nchunks);
    // scratch of the build
    const uint64_t L = std::min<uint64_t>(1ull << 30, ((y_max + kSegY - 1) / kSegY) * kSegY);
    const uint64_t nblocks = (y_max + L - 1) / L;
    int8_t *mu = (int8_t *)dev_alloc(t->al, t->ydense + 16);
    int32_t *segsum = (int32_t *)dev_alloc(t->al, sieve_segments(L) * 4);
    int64_t *carry = (int64_t *)dev_alloc(t->al, (nblocks + 1) * 8);
    int rc = MERTENS_OK;
    if (!t->Mloc || !t->segoff || !t->MG || !t->dl_m || !t->dl_yo || !t->dl_cnt || !mu ||
        !segsum || !carry)
        rc = MERTENS_ENOMEM;
    PrimeTable pt;
    if (rc == MERTENS_OK) {
        int prc = prime_table_create(&pt, t->al, y_max, s);
        if (prc == 0)
            prc = sieve_scratch_create(&pt, L);
        if (prc != 0)
            rc = prc == 2 ? MERTENS_ENOMEM : MERTENS_ECUDA;
    }
    if (rc == MERTENS_OK) {
        cudaMemsetAsync(carry, 0, (nblocks + 1) * 8, s);
        cudaMemsetAsync(mu, 0, t->ydense + 16, s);
        for (uint64_t b = 0; b < nblocks && rc == MERTENS_OK; ++b) {
            const uint64_t y1 = 1 + b * L;
            const uint64_t y2 = std::min(y1 + L - 1, y_max);
            SieveLaunch Lc;
            Lc.y1 = y1;
            Lc.len = y2 - y1 + 1;
            Lc.Mloc = t->Mloc + (y1 - 1);
            Lc.segsum = segsum;
            Lc.segoff = t->segoff + ((y1 - 1) >> kSegShift);
            Lc.carry_in = carry + b;
            Lc.carry_out = carry + b + 1;
            Lc.mu_out = y1 <= t->ydense ? mu : nullptr;
            Lc.mu_base = 1;
            Lc.mu_end = t->ydense;
            if (sieve_block_enqueue(&pt, Lc, s) < 0)
                rc = MERTENS_ECUDA;
        }
        if (rc == MERTENS_OK && (magic_table_enqueue(t->MG, t->mg_n, s) < 0 ||
                                 dense_list_enqueue(mu, t->ydense, t->MG, t->dl_m, t->dl_yo,
                                                    t->dl_cnt, s) < 0))
            rc = MERTENS_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess)
            rc = MERTENS_ECUDA;
        if (rc == MERTENS_OK) {
            const uint32_t st = sieve_scratch_status(&pt);
            if (st) {
                set_last_error("mertens_table_create: %s", sieve_status_text(st));
                rc = sieve_status_code(st);
            }
        }
    }
    if (rc == MERTENS_ECUDA)
        set_last_error("mertens_table_create: %s", cudaGetErrorString(cudaGetLastError()));
    else if (rc == MERTENS_ENOMEM)
        set_last_error("mertens_table_create: device allocation failed");
    if (pt.np)
        prime_table_destroy(&pt);
    dev_free(t->al, mu, t->ydense + 16);
    dev_free(t->al, segsum, sieve_segments(L) * 4);
    dev_free(t->al, carry, (nblocks + 1) * 8);
    if (rc != MERTENS_OK) {
        mertens_table_destroy(t);
        return rc;
    }
    *out = t;
    return MERTENS_OK;
}

int mertens_table_info(mertens_table_t t, uint64_t *y_max, mertens_u128 *n_max, size_t *bytes)
{
    if (!t)
        return MERTENS_EINVAL;
    if (y_max)
        *y_max = t->y_max;
    if (n_max) {
        n_max->lo = t->n_max_lo;
        n_max->hi = t->n_max_hi;
    }
    if (bytes)
        *bytes = t->bytes;
    return MERTENS_OK;
}

void mertens_table_destroy(mertens_table_t t)
{
    if (!t)
        return;
    cudaDeviceSynchronize();
    for (auto &a : t->allocs)
        dev_free(t->al, a.first, a.second);
    delete t;
}

}  // extern "C"
