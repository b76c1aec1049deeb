// mertens_sieve_M_noalloc: the window sieve and prefix scan of
// mertens_sieve_M with every scratch buffer in one file-scope device array,
// so the call itself allocates no device (or host heap) memory.
//
// The array lives on every GPU that loads this library until the process
// exits.  Its device address is looked up once per device, on the first call
// made while that device is current; that first call should therefore come
// before any stream capture on that device.  All calls share the array and
// it keeps the last call's contents: calls that overlap on the GPU (two
// streams, or two host threads each with a stream) race on it and must be
// serialised by the caller.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/libmertens.h"
#include "common.cuh"
#include "internal.h"

namespace mert {

// Limits of the allocation-free variant: windows of at most 2^21 y that end
// below 2^40 (so the sieving primes are below 2^20: pi(2^20) = 82025).
constexpr uint64_t kNaMaxLen = 1ull << 21;
constexpr uint64_t kNaMaxY = 1ull << 40;
constexpr uint32_t kNaMaxPrimeBound = 1u << 20;
constexpr uint32_t kNaMaxPrimes = 82100;

// Byte layout of the scratch array (each part 256-byte aligned).
constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t kNaOffP = 0;
constexpr size_t kNaOffLg = align256(kNaOffP + 4ull * kNaMaxPrimes);
constexpr size_t kNaOffM = align256(kNaOffLg + 4ull * kNaMaxPrimes);
constexpr size_t kNaOffL = align256(kNaOffM + 8ull * kNaMaxPrimes);
constexpr size_t kNaOffR = align256(kNaOffL + 1ull * kNaMaxPrimes);
constexpr size_t kNaOffQm = align256(kNaOffR + 4ull * kNaMaxPrimes);
constexpr size_t kNaOffPatE = align256(kNaOffQm + 4ull * kNaMaxPrimes);
constexpr size_t kNaOffPatO = align256(kNaOffPatE + 4ull * kPatternWords);
constexpr size_t kNaOffMloc = align256(kNaOffPatO + 4ull * kPatternWords);
constexpr size_t kNaSegs = kNaMaxLen / kSegY;
constexpr size_t kNaOffSegsum = align256(kNaOffMloc + 2ull * (kNaMaxLen + 2));
constexpr size_t kNaOffSegoff = align256(kNaOffSegsum + 4ull * kNaSegs);
constexpr size_t kNaOffCarry = align256(kNaOffSegoff + 8ull * kNaSegs);
constexpr size_t kNaOffErr = align256(kNaOffCarry + 16);
constexpr size_t kNaBytes = align256(kNaOffErr + 4);  // about 6.2 MB

static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

// Host state: the device address of the array per device (looked up once),
// and the prime table of the last window (host side, static storage).
static std::mutex g_na_mu;
constexpr int kNaMaxDevices = 64;
static unsigned char *g_na_dev_ptr[kNaMaxDevices];
static uint8_t g_na_composite[kNaMaxPrimeBound + 1];
static uint32_t g_na_p[kNaMaxPrimes];
static uint32_t g_na_lg[kNaMaxPrimes];
static uint64_t g_na_m[kNaMaxPrimes];
static uint8_t g_na_l[kNaMaxPrimes];
static uint32_t g_na_pat16[kPatternPeriod];
static uint32_t g_na_pat_e[kPatternWords];
static uint32_t g_na_pat_o[kPatternWords];
static uint32_t g_na_np = 0;       // primes currently in the host table
static uint32_t g_na_bound = 0;    // they are all primes <= g_na_bound

static int na_device_ptr(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
        set_last_error("mertens_sieve_M_noalloc: no usable current device");
        return MERTENS_ECUDA;
    }
    if (!g_na_dev_ptr[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_na_scratch);
        if (e != cudaSuccess || !ptr) {
            set_last_error("mertens_sieve_M_noalloc: cudaGetSymbolAddress failed: %s",
                           cudaGetErrorString(e));
            return MERTENS_ECUDA;
        }
        g_na_dev_ptr[dev] = (unsigned char *)ptr;
    }
    *out = g_na_dev_ptr[dev];
    return MERTENS_OK;
}

// Primes up to B (7 <= B <= 2^20) with their log weights and division
// magics, and the pre-sieve pattern, in the static host arrays.
static void na_host_primes(uint32_t B)
{
    if (B <= g_na_bound && g_na_np)
        return;
    memset(g_na_composite, 0, (size_t)B + 1);
    uint32_t np = 0;
    for (uint64_t i = 2; i <= B; ++i) {
        if (g_na_composite[i])
            continue;
        g_na_p[np] = (uint32_t)i;
        g_na_lg[np] = (uint32_t)std::lround(kLogScale * std::log2((double)i));
        g_na_m[np] = magic_of(i);
        g_na_l[np] = (uint8_t)magic_shift(i);
        ++np;
        for (uint64_t j = i * i; j <= B; j += i)
            g_na_composite[j] = 1;
    }
    for (uint32_t i = 0; i < kPatternPeriod; ++i) {
        uint32_t h = 0;
        const uint32_t small[4] = {2, 3, 5, 7};
        for (int q = 0; q < 4; ++q) {
            if (i % small[q] == 0)
                h += g_na_lg[q] | kCountOne;
            if (i % (small[q] * small[q]) == 0)
                h |= kSquareBit;
        }
        g_na_pat16[i] = h;
    }
    for (uint32_t j = 0; j < kPatternWords; ++j) {
        g_na_pat_e[j] = g_na_pat16[2 * j] | (g_na_pat16[2 * j + 1] << 16);
        g_na_pat_o[j] = g_na_pat16[2 * j + 1] | (g_na_pat16[(2 * j + 2) % kPatternPeriod] << 16);
    }
    g_na_np = np;
    g_na_bound = B;
}

}  // namespace mert

using namespace mert;

extern "C" int mertens_sieve_M_noalloc(uint64_t y1, uint64_t len, int64_t carry, int32_t *M_dev,
                                       void *stream)
{
    if (!M_dev || ((uintptr_t)M_dev & 3u)) {
        set_last_error("mertens_sieve_M_noalloc: M_dev must be a 4-byte aligned device pointer");
        return MERTENS_EINVAL;
    }
    if (y1 == 0 || len == 0) {
        set_last_error("mertens_sieve_M_noalloc: need y1 >= 1 and len >= 1");
        return MERTENS_EINVAL;
    }
    if (len > kNaMaxLen || y1 > kNaMaxY || y1 + len - 1 >= kNaMaxY) {
        set_last_error("mertens_sieve_M_noalloc: window too large: need len <= 2^21 and "
                       "y1 + len - 1 < 2^40 (got y1 = %llu, len = %llu)",
                       (unsigned long long)y1, (unsigned long long)len);
        return MERTENS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    unsigned char *base = nullptr;
    int rc = na_device_ptr(&base);
    if (rc != MERTENS_OK)
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t y2 = y1 + len - 1;
    uint64_t B = (uint64_t)std::sqrt((double)y2);
    while (B * B > y2)
        --B;
    while ((B + 1) * (B + 1) <= y2)
        ++B;
    if (B < 7)
        B = 7;
    na_host_primes((uint32_t)B);

    PrimeTable pt;
    pt.np = g_na_np;
    pt.p = (uint32_t *)(base + kNaOffP);
    pt.lg = (uint32_t *)(base + kNaOffLg);
    pt.m = (uint64_t *)(base + kNaOffM);
    pt.l = (uint8_t *)(base + kNaOffL);
    pt.blk_r = (uint32_t *)(base + kNaOffR);
    pt.blk_qm = (uint32_t *)(base + kNaOffQm);
    pt.pat_even = (uint32_t *)(base + kNaOffPatE);
    pt.pat_odd = (uint32_t *)(base + kNaOffPatO);
    pt.host_p = g_na_p;
    const size_t np = g_na_np;
    cudaMemcpyAsync(pt.p, g_na_p, np * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(pt.lg, g_na_lg, np * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(pt.m, g_na_m, np * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(pt.l, g_na_l, np, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(pt.pat_even, g_na_pat_e, kPatternWords * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(pt.pat_odd, g_na_pat_o, kPatternWords * 4, cudaMemcpyHostToDevice, s);

    int64_t *cy = (int64_t *)(base + kNaOffCarry);
    uint32_t *er = (uint32_t *)(base + kNaOffErr);
    cudaMemcpyAsync(cy, &carry, 8, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(er, 0, 4, s);  // the error word must start at zero every call

    SieveLaunch L;
    L.y1 = y1;
    L.len = len;
    L.Mloc = (int16_t *)(base + kNaOffMloc);
    L.segsum = (int32_t *)(base + kNaOffSegsum);
    L.segoff = (int64_t *)(base + kNaOffSegoff);
    L.carry_in = cy;
    L.carry_out = cy + 1;
    if (sieve_block_enqueue(&pt, L, s) < 0 ||
        expand_M_enqueue(L.Mloc, L.segoff, len, M_dev, er, s) < 0) {
        set_last_error("mertens_sieve_M_noalloc: launch failed: %s",
                       cudaGetErrorString(cudaGetLastError()));
        return MERTENS_ECUDA;
    }
    uint32_t e = 0;
    if (cudaMemcpyAsync(&e, er, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        set_last_error("mertens_sieve_M_noalloc: %s", cudaGetErrorString(cudaGetLastError()));
        return MERTENS_ECUDA;
    }
    if (e & kErrMOverflow) {
        set_last_error("mertens_sieve_M_noalloc: some |M(y)| >= 2^31");
        return MERTENS_EOVERFLOW;
    }
    return MERTENS_OK;
}
