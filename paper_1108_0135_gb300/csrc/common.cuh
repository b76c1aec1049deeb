// Device helpers shared by the libmertens kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mert {

// Sieve tile: y values per CTA of the fused mu_sieve / m_scan kernel.  Each
// y owns a 16-bit half of a 32-bit shared word (two y per word).
constexpr int kSieveTile = 65536;
constexpr int kSieveWords = kSieveTile / 2;
constexpr int kSieveThreads = 1024;
// M(y) is stored as an int16 relative to M(segment start - 1), one int64
// offset per segment of kSegY y (|relative M| <= 3/4 kSegY < 2^15).  A
// segment is the 2048 y one warp of the sieve decodes.
constexpr int kSegShift = 11;
constexpr int kSegY = 1 << kSegShift;
// Dense chunk: y values per chunk of the squarefree list used by the dense
// update, and the largest number of squarefree y a chunk can hold (one y in
// four is a multiple of 4, so at most 3/4 of any 4096 consecutive y).
constexpr int kChunk = 4096;
constexpr int kChunkCap = 3072;
// Gathered terms per warp work item of the global-memory gather path.
constexpr int kSparseItem = 1024;
// y values per shared-memory tile of the gather path (int16 relative M).
constexpr int kGatherTile = 32768;

// Fixed-point scale of the log sieve: lg(p) = round(8 * log2 p).
constexpr int kLogScale = 8;
// Half-word layout of the log sieve: bits 0..9 sum of lg(p) over the distinct
// sieving primes of y, bits 10..13 their number, bit 15 set when the square
// of a sieving prime divides y (atomicOr, so it never carries).
constexpr uint32_t kCountOne = 1u << 10;
constexpr uint32_t kSquareBit = 1u << 15;
// Pre-sieve pattern: primes 2,3,5,7 and their squares, period 4*9*25*49.
constexpr uint32_t kPatternPeriod = 44100;
constexpr uint32_t kPatternWords = kPatternPeriod / 2;

// Byte sieve (the fast variant of a1 + a2): one byte per y holding the sum of
// odd weights w(p) = the odd integer nearest S log2 p (so its parity is the
// parity of the prime count), and one bit per y set when a prime square
// divides y.  S = 4 while y < 2^42, else 3 (up to 2^54).  A tile of kByteTile
// y takes 128 KiB + 16 KiB of shared memory.
constexpr int kByteTile = 131072;
constexpr int kByteWords = kByteTile / 4;
constexpr int kByteSqWords = kByteTile / 32;
// Pre-sieve tables of the byte sieve: 16 copies of the byte pattern of
// 2, 3, 5, 7, copy k starting at phase k, each long enough for any phase plus
// one tile (so a tile is one 16-byte aligned copy), and the square flags of
// 4, 9, 25, 49 as one long bit string read with a funnel shift.
constexpr uint32_t kPat8Len = 175184;   // >= 44100 + 131072, multiple of 16
constexpr uint32_t kPatSqWords = 5480;  // > (44100 + 131072 + 64) / 32
// Tiles whose first y is at least this take one decision threshold for the
// whole tile (4 log2 y moves by < 0.012 over a tile); lower tiles decide
// with a threshold per y.
constexpr uint64_t kByteTileThrMin = 1ull << 26;

// Error bits of the plan's device status word.
constexpr uint32_t kErrMOverflow = 1u;   // |M(y)| did not fit int32

// Bit length of v (0 for v = 0).
__host__ __device__ __forceinline__ unsigned bitlen64(uint64_t v)
{
#ifdef __CUDA_ARCH__
    return 64u - (unsigned)__clzll((long long)v);
#else
    return v ? 64u - (unsigned)__builtin_clzll(v) : 0u;
#endif
}

// Division by an invariant divisor d (Granlund & Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994, Sec. 4): with
// l = ceil(log2 d) and m = floor(2^(63+l)/d) + 1 (so m < 2^64), every k < 2^63
// has floor(k/d) = floor(m*k / 2^(63+l)) = floor(mulhi64(m, 2k) / 2^l).
__host__ __device__ __forceinline__ unsigned magic_shift(uint64_t d)
{
    return bitlen64(d - 1);
}

// m = floor(2^(63+l)/d) + 1: on the device by restoring long division of the
// 128-bit numerator 2^(63+l) (high word 2^(l-1), low word 0) by d (the high
// word is below d, so the quotient fits 64 bits), on the host by one 128-bit
// division.  d = 1 gives 2^63 + 1.
__host__ __device__ inline uint64_t magic_of(uint64_t d)
{
    unsigned l = magic_shift(d);
    if (l == 0)
        return (1ull << 63) + 1ull;
#ifndef __CUDA_ARCH__
    // on the host, one 128-by-64 division of 2^(63+l)
    return (uint64_t)((((unsigned __int128)1) << (63 + l)) / d) + 1ull;
#endif
    uint64_t r = 1ull << (l - 1);  // running remainder, always < d
    uint64_t q = 0;
    for (int i = 63; i >= 0; --i) {
        // r = 2r (next numerator bit is 0); r < 2d < 2^39, no overflow
        r <<= 1;
        q <<= 1;
        if (r >= d) {
            r -= d;
            q |= 1ull;
        }
    }
    return q + 1ull;
}

__device__ __forceinline__ uint64_t div_magic(uint64_t k2, uint64_t m, unsigned l)
{
    return __umul64hi(k2, m) >> l;
}

// The same theorem with 31-bit numerators: for 2 <= d < 2^31, l = ceil(log2 d)
// and m = floor(2^(31+l)/d) + 1 < 2^32, every v < 2^31 has
// floor(v/d) = floor(mulhi32(m, v) / 2^(l-1)).  Returns m; *s = l - 1.
__host__ __device__ inline uint32_t magic32_of(uint32_t d, unsigned *s)
{
    const unsigned l = bitlen64((uint64_t)d - 1);
    *s = l - 1;
    return (uint32_t)(((1ull << (31 + l)) / d) + 1ull);
}

__device__ __forceinline__ uint32_t div_magic32(uint32_t v, uint32_t m, unsigned s)
{
    return __umulhi(v, m) >> s;
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies global -> shared (cp.async.bulk, completing on an
// mbarrier in shared memory) with bounded waits.
// ---------------------------------------------------------------------------
constexpr uint32_t kErrTimeout = 8u;       // a bounded wait gave up
constexpr uint32_t kBulkWaitLimit = 1u << 20;  // tries of at most ~1 us each

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// One arrival expected (the thread that issues the copies).
__device__ __forceinline__ void mbar_init(uint64_t *mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)) : "memory");
}

// Orders this thread's earlier shared-memory accesses (and an mbarrier init)
// before later asynchronous-proxy accesses.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The issuing thread's arrival, announcing `bytes` to come (< 2^20).
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)),
                 "r"(bytes)
                 : "memory");
}

// dst (shared) <- src (global), `bytes` a multiple of 16, both 16-byte aligned.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(mbar))
        : "memory");
}

// Waits (bounded) for phase `parity` of the mbarrier to complete; false when
// the limit was reached first.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity)
{
    for (uint32_t it = 0; it < kBulkWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(mbar)), "r"(parity)
            : "memory");
        if (done)
            return true;
    }
    return false;
}

// Warp-wide sum of a 64-bit value (mod 2^64).
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int64_t warp_sum_i64(int64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Block-wide scans (warp shuffles, then a pass over the warp totals).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += n;
    }
    return v;
}

// Exclusive scan over the CTA; returns the thread's exclusive prefix and
// writes the CTA total to *total.  `sh` holds 33 values of T.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T *sh, T *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31)
        sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? sh[lane] : T(0);
        T wi = warp_incl_scan(w);
        if (lane < nw)
            sh[lane] = wi - w;
        if (lane == nw - 1)
            sh[32] = wi;
    }
    __syncthreads();
    T res = sh[warp] + inc - v;
    *total = sh[32];
    __syncthreads();
    return res;
}

__device__ __forceinline__ uint32_t block_scan_u32(uint32_t v, uint32_t *sh, uint32_t *total)
{
    return block_excl_scan<uint32_t>(v, sh, total);
}

}  // namespace mert
