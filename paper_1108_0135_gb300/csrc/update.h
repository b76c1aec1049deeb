// Argument blocks of the update (a3) and resolve (a4) kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mert {

// Chunks staged per dense work item, threads per dense CTA, and the padded
// per-chunk capacity of the squarefree list (four parts -- mu = +1 odd y,
// +1 even, -1 odd, -1 even -- each starting at an even index so that they
// can be read 16 bytes at a time; at most 3072 squarefree y per chunk).
constexpr int kDenseChunks = 2;
constexpr int kDenseThreads = 256;
constexpr int kChunkCapPad = 3076;

// Gathered terms are shared along chains x, 2x, ..., 2^kShareLevels x of
// one target (update.cu): the level sums the kernels produce per entry.
constexpr uint32_t kShareLevels = 4;

// Up to 32 entries of one target, e = first + stride * lane (x = x0 +
// stride * lane), sharing one dense cut-off yc (pred = 0), or with a cut-off
// per entry in YCE (pred = 1; yc = their maximum).  Odd y <= olo are left
// out of their sums (0: none): those terms come from the entries x/2, whose
// lanes in `emit` add minus their even-y sums to entry 2x (update.cu).
struct Group {
    uint32_t first;
    uint32_t count;   // entries in the group (1..32)
    uint32_t pred;
    uint32_t emit;    // lanes that add their even-y sum to entry 2x
    uint64_t yc;
    uint64_t olo;
    uint32_t x0;
    uint32_t stride;  // 1 or 2
};

// Dense work item: chunks [c0, c1) for the groups [g0, g1) of the sorted
// group list.
struct DenseItem {
    uint32_t c0, c1, g0, g1;
};

struct DenseArgs {
    const DenseItem *items;
    uint32_t nitems;
    uint32_t *counter;
    const Group *groups;
    const uint64_t *K;    // k = floor(n/x) per entry
    const uint64_t *YCE;  // dense cut-off per entry
    const uint64_t *dl_m;
    const uint16_t *dl_yo;
    const uint2 *dl_cnt;
    uint64_t *S;
    uint32_t ctas_per_sm;  // 0: as many as fit; else at most this many per SM
};

// Invariant-divisor constants of one block [y1, y2].
struct SparseBlockArgs {
    uint64_t y1, y2;
    uint64_t m_y1, m_y2p1;
    uint32_t l_y1, l_y2p1;
};

// M(y) of the current block: segoff[(y - y1) >> kSegShift] + Mloc[y - y1].
// Chunks of heavy entries go to `queue` ({entry, j_top low, j_top high,
// terms}, qlen of them, at most qcap; beyond that kErrQueue in *err).
struct SparseArgs {
    uint64_t nent;
    uint64_t y_lo;  // first y of the block handled by the global-memory path
    uint64_t kmax;  // entries with k >= kmax have their terms in the block's tiles
    uint64_t m_ylo;
    uint32_t l_ylo;
    uint32_t qcap;
    const uint64_t *K, *JLO, *JC0, *YCE, *MG;
    const uint32_t *EMIT;  // x | L << 29: the entries 2^s x (s <= L) it feeds (update.cu)
    uint64_t *S;
    uint4 *queue;
    uint32_t *qlen;
    uint32_t *err;
    const int16_t *Mloc;
    const int64_t *segoff;
};

// Status bit of a plan: the global gather's chunk queue overflowed.
constexpr uint32_t kErrQueue = 16u;

struct QueryDev {
    uint64_t X;    // entries of the target
    uint64_t off;  // global index of its entry x = 1
};

// Shared-memory gather path: one tile of kGatherTile y (or fewer) and the
// division constants of its first y and of its last y + 1.
struct GatherTile {
    uint64_t t1;
    uint64_t m1, m2;
    uint32_t len;
    uint32_t l1, l2;
    uint32_t pad;
};

// Work item: entries [e0, e1) (global indices, one target) for one tile.
struct GatherItem {
    uint32_t tile, e0, e1, pad;
};

struct GatherArgs {
    uint64_t y1;  // block start (index base of Mloc / segoff)
    const GatherTile *tiles;
    const GatherItem *items;
    uint32_t nitems;
    uint32_t *counter;
    const int16_t *Mloc;
    const int64_t *segoff;
    const uint64_t *K, *JLO, *JCUR, *MG;
    const uint32_t *EMIT;  // x | L << 29: the entries 2^s x (s <= L) it feeds (update.cu)
    uint64_t *S;
    uint32_t threads;      // 256 or 512 per CTA
    uint32_t ctas_per_sm;  // 0: as many as fit; else at most this many per SM
    uint32_t *err;         // status word: kErrTimeout when a bounded wait gave up
    uint32_t quot;         // 0: multiply-high magics; 1: float estimate, 32-bit
                           // remainder (every j < 2^31); 2: float, 64-bit
};

// Array entry with k = floor(n/x) >= 2^63 (targets n >= 2^63 only): its k
// needs two words, so it takes the paper's split form directly -- direct terms
// M(y)(floor(k/y) - floor(k/(y+1))) for y <= s and gathered terms
// M(floor(k/j)) for j in [jlo, jhi] -- with 128-bit quotients, in its own
// kernel.  The 64-bit kernels see such an entry as k = 0 (no terms).
struct WideEntry {
    uint64_t k_lo, k_hi;  // k
    uint64_t s;           // floor(sqrt(k))
    uint64_t jlo, jhi;    // floor(X/x) + 1, floor(k/(s+1))
    uint64_t e;           // global entry index
};

struct WideArgs {
    const WideEntry *W;
    uint64_t y1, y2;  // the block
    const int16_t *Mloc;
    const int64_t *segoff;
    uint64_t *S;
};

// Units (terms) per CTA of the wide kernel, and the units of entry W in the
// block [y1, y2] (host and device).
constexpr int kWideThreads = 256;
constexpr int kWidePer = 16;
constexpr uint64_t kWideUnitsPerCta = (uint64_t)kWideThreads * kWidePer;

__host__ __device__ inline void wide_ranges(const WideEntry &W, uint64_t y1, uint64_t y2,
                                            uint64_t *nd, uint64_t *ja, uint64_t *ng)
{
    const unsigned __int128 k = ((unsigned __int128)W.k_hi << 64) | W.k_lo;
    const uint64_t dl = y2 < W.s ? y2 : W.s;
    *nd = y1 <= dl ? dl - y1 + 1 : 0;
    // j with floor(k/j) in [y1, y2]: floor(k/(y2+1)) < j <= floor(k/y1)
    const unsigned __int128 q2 = k / ((unsigned __int128)y2 + 1) + 1;
    const unsigned __int128 q1 = k / y1;
    const unsigned __int128 a = q2 > W.jlo ? q2 : (unsigned __int128)W.jlo;
    const unsigned __int128 b = q1 < W.jhi ? q1 : (unsigned __int128)W.jhi;
    *ja = (uint64_t)a;
    *ng = b >= a ? (uint64_t)(b - a + 1) : 0;
}

int magic_table_enqueue(uint64_t *MG, uint64_t nd, cudaStream_t s);
// R[pairs[2i]] = M(pairs[2i+1]) from a resident table (i < count).
int table_lookup_enqueue(const uint64_t *pairs, uint32_t count, const int16_t *Mloc,
                         const int64_t *segoff, uint64_t *R, cudaStream_t s);
// *out = M(y) from a resident table (1 <= y <= its y_max).
int carry_from_table_enqueue(const int16_t *Mloc, const int64_t *segoff, uint64_t y,
                             int64_t *out, cudaStream_t s);
int wide_update_enqueue(const WideArgs &a, uint32_t nw, uint32_t grid_x, cudaStream_t s);
int dense_list_enqueue(const int8_t *mu_aux, uint64_t ydense, const uint64_t *MG, uint64_t *dl_m,
                       uint16_t *dl_yo, uint2 *dl_cnt, cudaStream_t s);
int dense_update_enqueue(const DenseArgs &a, cudaStream_t s);
int sparse_block_enqueue(const SparseBlockArgs &b, const SparseArgs &a, cudaStream_t s);
int gather_tiles_enqueue(const GatherArgs &a, cudaStream_t s);
// Exchange buffers (two int64 words per entry: the low and the high 32-bit
// half of its 64-bit sum): add S_loc + C coef of a window; turn one back into
// 64-bit sums.
int window_accumulate_enqueue(const uint64_t *S, const uint64_t *coef, uint64_t C, uint64_t X,
                              int64_t *halves, cudaStream_t s);
int halves_to_sums_enqueue(const int64_t *halves, uint64_t X, uint64_t *S, cudaStream_t s);
int resolve_enqueue(const QueryDev *qs, uint32_t nq, const uint64_t *S, const uint64_t *K,
                    uint64_t *R, cudaStream_t s);

}  // namespace mert
