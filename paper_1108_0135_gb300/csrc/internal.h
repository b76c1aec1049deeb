// Host-side declarations shared by the libmertens translation units.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <utility>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/libmertens.h"
#include "common.cuh"

namespace mert {

// Device-memory hook captured by a plan (null alloc = cudaMalloc/cudaFree).
struct Allocator {
    mertens_alloc_fn alloc = nullptr;
    mertens_free_fn release = nullptr;
    void *ctx = nullptr;
};
Allocator current_allocator();
void *dev_alloc(const Allocator &a, size_t bytes);
void dev_free(const Allocator &a, void *p, size_t bytes);

// Prime table of a plan (device arrays, index 0..np-1, primes ascending,
// the first four are 2, 3, 5, 7 which the pre-sieve pattern covers).
struct PrimeTable {
    uint32_t np = 0;              // primes in the table
    uint32_t *p = nullptr;        // prime
    uint32_t *lg = nullptr;       // round(8 * log2 p)
    uint64_t *m = nullptr;        // division magic of p
    uint8_t *l = nullptr;         // division shift of p
    uint32_t *blk_r = nullptr;    // per block: y1 mod p
    uint32_t *blk_qm = nullptr;   // per block: floor(y1 / p) mod p
    uint32_t *pat_even = nullptr; // pre-sieve pattern words for an even phase
    uint32_t *pat_odd = nullptr;  // ... and for an odd phase
    // byte sieve (null when the table was built without it), weight scale S
    uint32_t byte_scale = 0;
    uint4 *pq = nullptr;          // {p, m32(p), m32(p^2) or 0, s(p) | s(p^2) << 8 | w(p) << 16}
    uint64_t *blk_r2 = nullptr;   // per block: y1 mod p^2
    uint4 *pat8 = nullptr;        // 16 phase copies of the byte pattern
    uint32_t *patsq = nullptr;    // square flags of 4, 9, 25, 49 as a long bit string
    // persistent byte sieve: p | w(p) << 24 for p < 2^17, and scratch for
    // blocks of up to scratch_len y (sieve_scratch_create)
    uint32_t np_mid = 0;          // primes below 2^17
    uint32_t *pw = nullptr;
    uint64_t scratch_len = 0;
    uint32_t bucket_cap = 0;      // entries per tile
    uint64_t *bucket = nullptr;   // tiles x bucket_cap
    uint32_t *gsq = nullptr;      // one bit per y of a block, whole tiles
    uint32_t *perr = nullptr;     // status bits of the persistent kernel
    // byte sieve at weight scale 2 (square flag in bit 7): its prime records
    // (as pq, with w2(p) = the odd integer nearest 2 log2 p), its pattern, and
    // per-tile lists of the multiples of p^2 (p >= 8192) of a block
    uint4 *pq2 = nullptr;
    uint4 *pat2 = nullptr;        // 16 phase copies: 2, 3, 5, 7 (base 1, flags of their squares)
    uint4 *rec = nullptr;         // per block, p >= 512: {p, m32(p), y1 mod p, s(p) | w2 << 8}
    uint2 *rec2 = nullptr;        // per block, 512 <= p < 8192: {y1 mod p^2 | s << 26, m32(p^2)}
    uint32_t sq_cap = 0;          // list entries per tile
    uint32_t *sqcnt = nullptr;    // tiles of scratch_len
    uint32_t *sqlist = nullptr;   // tiles x sq_cap
    // host copy of the primes (for counting primes <= a bound)
    uint32_t *host_p = nullptr;
    Allocator al;
};

// Arguments of one sieve block (steps a1 + a2, fused).  Results:
//   M(y) = segoff[(y - y1) >> kSegShift] + Mloc[y - y1],  y in [y1, y1+len).
struct SieveLaunch {
    uint64_t y1 = 0;             // first y of the block (>= 1)
    uint64_t len = 0;            // y values in the block
    int16_t *Mloc = nullptr;     // [len + 1] M relative to its segment
    int32_t *segsum = nullptr;   // [segments] scratch: mu sum per segment
    int64_t *segoff = nullptr;   // [segments] M(segment start - 1)
    const int64_t *carry_in = nullptr;  // device M(y1 - 1)
    int64_t *carry_out = nullptr;       // device M(y1 + len - 1)
    int8_t *mu_out = nullptr;    // optional: mu_out[y - mu_base] for y <= mu_end
    uint64_t mu_base = 0, mu_end = 0;
    cudaEvent_t mid = nullptr;   // if set: recorded after a1 ...
    cudaEvent_t mid2 = nullptr;  // ... and this one before a2 (profiling)
};

// Builds the prime table for sieving up to y_max (host + device upload);
// with_bytes adds the tables of the byte sieve.
int prime_table_create(PrimeTable *t, const Allocator &al, uint64_t y_max, cudaStream_t s,
                       bool with_bytes = true);
void prime_table_destroy(PrimeTable *t);
// Scratch of the persistent byte sieve for blocks of up to max_len y (bucket
// storage sized from the table's primes above 2^17, and the square bit
// array).  Optional: without it blocks take the per-tile byte kernel.
int sieve_scratch_create(PrimeTable *t, uint64_t max_len);
// Status bits the persistent sieve left since the last call (and clears them):
// kErrBucket when a bucket overflowed (the block's M(y) is then wrong).
uint32_t sieve_scratch_status(PrimeTable *t);
// The status code and the text for those bits: a bounded wait that gave up
// (MERTENS_ETIMEOUT) or an overflowed bucket (MERTENS_EOVERFLOW).
inline int sieve_status_code(uint32_t st)
{
    return (st & kErrTimeout) ? MERTENS_ETIMEOUT : MERTENS_EOVERFLOW;
}
inline const char *sieve_status_text(uint32_t st)
{
    return (st & kErrTimeout) ? "a bounded wait for a bulk copy in the sieve gave up"
                              : "a sieve bucket overflowed its capacity";
}
// Number of primes in the table that are <= b.
uint32_t prime_count_upto(const PrimeTable *t, uint64_t b);
// Enqueues the fused steps a1 + a2 for one block.  Returns the number of
// kernels launched, or -1 on a launch error.
int sieve_block_enqueue(const PrimeTable *t, const SieveLaunch &L, cudaStream_t s);
// Segments of a block of `len` y values.
inline uint64_t sieve_segments(uint64_t len) { return (len + kSegY - 1) / kSegY; }

// A kernel's attributes belong to each device's copy of it: the launch sites
// that raise a dynamic shared-memory limit keep one bit per device in an
// atomic word, set after the attributes (a race only repeats the setting).
inline uint64_t device_bit()
{
    int dev = 0;
    cudaGetDevice(&dev);
    return 1ull << (dev & 63);
}
inline bool attrs_needed(const std::atomic<uint64_t> &done, uint64_t bit)
{
    return (done.load(std::memory_order_acquire) & bit) == 0;
}
inline void attrs_done(std::atomic<uint64_t> &done, uint64_t bit)
{
    done.fetch_or(bit, std::memory_order_release);
}
// M(y) of a window as int32 (the step-level entry point); sets *err bit 1 on
// an int32 overflow.
int expand_M_enqueue(const int16_t *Mloc, const int64_t *segoff, uint64_t len, int32_t *M,
                     uint32_t *err, cudaStream_t s);

// Thread-local last-error text.
void set_last_error(const char *fmt, ...);

// Device bytes of the Granlund-Montgomery magic table and of the dense
// squarefree list (update.cu) for a dense limit ydense.
inline uint64_t dense_chunks(uint64_t ydense) { return ydense / kChunk + 1; }

}  // namespace mert

// A resident M(y) table (mertens_table_create): M(y) for 1 <= y <= y_max in
// the sieve's block layout (int16 relative to the 2048-y segment, int64
// segment offsets, both indexed from y = 1), and the query-independent parts
// of the update for targets up to n_max: divisor magics for d < mg_n and the
// squarefree dense list for y <= ydense.
struct mertens_table_s {
    mert::Allocator al;
    int device = 0;
    uint64_t y_max = 0;
    uint64_t n_max_lo = 0, n_max_hi = 0;
    uint64_t ydense = 0, mg_n = 0;
    int16_t *Mloc = nullptr;
    int64_t *segoff = nullptr;
    uint64_t *MG = nullptr, *dl_m = nullptr;
    uint16_t *dl_yo = nullptr;
    uint2 *dl_cnt = nullptr;
    size_t bytes = 0;
    std::vector<std::pair<void *, size_t>> allocs;
};

namespace mert {

}  // namespace mert
