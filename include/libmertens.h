/*
 * libmertens -- exact isolated values of the Mertens function on one GB300.
 *
 * The method is the one of "Computing the Mertens function on a GPU"
 * (arXiv:1108.0135), Sec. 2-3: pick a sieve limit u > sqrt(n), keep an array
 * of X = floor(n/u) entries that end up holding M(floor(n/x)), x = 1..X, sieve
 * M(y) for y < u block by block, add every block's contributions to the array,
 * and resolve the array at the end.  M(y) = sum_{m <= y} mu(m) (Sec. 1).
 *
 * All entry points are plain C.  Pointers are host pointers unless the
 * argument name ends in _dev (device memory of the current CUDA device).
 * `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 * stream).  Every function returns an int status (MERTENS_OK = 0 or one of the
 * codes below); nothing aborts, throws or traps on the device.  Results are
 * exact integers: there is no tolerance anywhere in this library.
 *
 * Thread safety: distinct plans may be used from distinct host threads; one
 * plan must not be used from two threads at once.
 */
#ifndef LIBMERTENS_H
#define LIBMERTENS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MERTENS_OK 0
#define MERTENS_EINVAL 1    /* an argument is out of range (see each call)  */
#define MERTENS_ENOMEM 2    /* a device or host allocation failed           */
#define MERTENS_ECUDA 3     /* a CUDA runtime call failed                   */
#define MERTENS_ETIMEOUT 4  /* a bounded device wait expired                */
#define MERTENS_ENOTREADY 5 /* result asked for before mertens_run          */
#define MERTENS_ENOTSUP 6   /* input outside what this build supports       */
#define MERTENS_EOVERFLOW 7 /* a value left its integer type (see notes)    */

/* Unsigned 128-bit integer as two 64-bit words: value = hi * 2^64 + lo. */
typedef struct {
    uint64_t lo, hi;
} mertens_u128;

/* Opaque plan: the targets, their arrays and every device buffer. */
typedef struct mertens_plan_s *mertens_plan_t;

/* Human-readable text for a status code (static storage, never NULL). */
const char *mertens_strerror(int code);

/* Text of the last error raised on this host thread (static per thread). */
const char *mertens_last_error(void);

/*
 * Device-memory hook.  By default the library allocates stream-ordered
 * (cudaMallocAsync / cudaFreeAsync on a non-blocking library stream, then
 * waits for that stream alone), so plans can be created and destroyed while
 * other work runs on the device.  A caller (for example a PyTorch process that wants
 * the caching allocator) may install its own pair; `ctx` is passed back
 * unchanged.  alloc must return 256-byte aligned device memory or NULL.
 * Passing alloc = NULL restores the default.  Applies to plans created after
 * the call; each plan frees with the pair it allocated with.
 */
typedef void *(*mertens_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*mertens_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
int mertens_set_allocator(mertens_alloc_fn alloc, mertens_free_fn release, void *ctx);

/*
 * mertens_plan -- prepare the computation of M(n_i), i < count, with one
 * shared sieve pass (Sec. 2 notes that close targets can share one sieve).
 *
 *   out        receives the plan (owned by the caller; free with
 *              mertens_destroy).
 *   n          `count` targets, each 1 <= n_i < 2^127 (else MERTENS_EINVAL).
 *              Array entries with k = floor(n_i/x) >= 2^63 (x <= n_i/2^63,
 *              so only for n_i >= 2^63) are computed with two-word (128-bit)
 *              quotients (the paper, Sec. 5, uses 128-bit integers there);
 *              all others with one-word quotients.  Copied; the caller
 *              keeps ownership.
 *   u          sieve limit shared by all targets.  {0,0} = chosen by the
 *              library: a batch limit ub = f g (sum n)^(2/3) (f from
 *              mertens_tuning, g = clamp((max n/1e18)^(-1/4), 1, 1.78)),
 *              and per target
 *              u_i = min(n_i, ub), raised above floor(sqrt(n_i)) where
 *              needed; the sieve runs to the largest targets' need.  Otherwise it must
 *              satisfy floor(sqrt(n_i)) < u <= n_i for every i (u = 1 is
 *              allowed for n_i = 1), else MERTENS_EINVAL.  u < 2^64 (else
 *              MERTENS_ENOTSUP).  Each target's array has X_i = floor(n_i/u_i)
 *              entries (Sec. 2); X_i >= 2^32 is MERTENS_ENOTSUP.
 *   block_len  length of a sieve block in y (Sec. 3 processes the y-axis
 *              block by block); 0 = chosen by the library.  Any value >= 1
 *              is honoured exactly.
 *
 * Allocates all device memory of the plan on the current device (through the
 * hook above).  Host-side work only otherwise; no kernel is launched.
 * Errors: MERTENS_EINVAL (count = 0, bad n or u), MERTENS_ENOTSUP,
 * MERTENS_ENOMEM, MERTENS_ECUDA.  On error *out is set to NULL.
 */
int mertens_plan(mertens_plan_t *out, const mertens_u128 *n, size_t count,
                 mertens_u128 u, uint64_t block_len);

/*
 * Resident M(y) table.  The sieve's output (steps a1 + a2: M(y) for
 * 1 <= y <= y_max) is computed once and kept in device memory (about
 * 2 bytes per y), together with what the update needs independently of the
 * target for all n <= n_max (the divisor magics and the squarefree list of
 * the dense form).  Plans made on it read M(y) from the table for every sieve
 * block that ends at or below y_max and sieve only the blocks above it; their
 * sieve limit u is at least min(n, y_max + 1) (the table's part of the sieve
 * costs nothing and the update's terms fall as 1/sqrt(u)) and at least the
 * automatic limit of a sieving plan for the same targets; a target
 * n <= y_max is read from the table directly.  The paper sieves per target
 * (Sec. 3); sharing one sieve between queries is what Sec. 2 allows for close
 * targets, taken to every target the table covers.
 *
 *   mertens_table_create: 1 <= y_max < 2^40, 1 <= n_max < 2^127; sieves on
 *     `stream` and returns when done.  The table lives on the current device
 *     and owns its memory (allocated through the allocator hook).
 *     Errors: MERTENS_EINVAL, MERTENS_ENOMEM, MERTENS_ECUDA.
 *   mertens_table_info: y_max, n_max and the device bytes held (each output
 *     may be NULL).  Errors: MERTENS_EINVAL (NULL table).
 *   mertens_plan_on_table: as mertens_plan, on the table's device; u = {0,0}
 *     picks the larger of min(n, y_max + 1) and the automatic limit per
 *     target.  MERTENS_ENOTSUP when a target exceeds n_max or needs dense
 *     cut-offs or divisors beyond the table; block_len must be a multiple of
 *     2048 (0: 2^30).  The table must outlive its plans.
 *   mertens_table_destroy: waits for the device, then frees the table.
 */
typedef struct mertens_table_s *mertens_table_t;
int mertens_table_create(mertens_table_t *out, uint64_t y_max, mertens_u128 n_max, void *stream);
int mertens_table_info(mertens_table_t table, uint64_t *y_max, mertens_u128 *n_max, size_t *bytes);
int mertens_plan_on_table(mertens_plan_t *out, mertens_table_t table, const mertens_u128 *n,
                          size_t count, mertens_u128 u, uint64_t block_len);
void mertens_table_destroy(mertens_table_t table);

/*
 * mertens_plan_window -- like mertens_plan, but the run covers only the sieve
 * blocks of y in [y_first, y_last] (clipped to the targets' largest y) and
 * stops before resolve.  Every contribution of the window to entry x's sum
 * S[x] is affine in the window's unknown carry C = M(y_first - 1): direct and
 * gathered terms are sums of M(y) = M_loc(y) + C, with M_loc the prefix sum
 * of mu from y_first (Sec. 2-3; the paper has no window form, this is the
 * decomposition that lets windows run in any order or on several devices).
 * The run computes S_loc (C taken as 0); the plan also knows coef[x], the
 * coefficient of C, so the window adds S_loc[x] + C coef[x] (mod 2^64).
 * Windows that partition [1, y_max], each with its carry, sum to the S of a
 * whole run; resolve is then M[x] = 1 - S[x] - sum_{j>=2} M[xj].
 * Errors: those of mertens_plan; MERTENS_EINVAL when y_first = 0 or
 * y_last < y_first.  mertens_result on a window plan is MERTENS_EINVAL.
 */
int mertens_plan_window(mertens_plan_t *out, const mertens_u128 *n, size_t count,
                        mertens_u128 u, uint64_t block_len, uint64_t y_first, uint64_t y_last);

/*
 * mertens_resolve -- the last step on its own (Sec. 2): given every entry's
 * update sum S[x-1], x = 1..X = floor(n/u) (host array, uint64, mod 2^64 --
 * for instance the windows of a partition of [1, y_max] added up as
 * S_loc + C coef), computes M_out[x-1] = M(floor(n/x)) by
 * M[x] = 1 - S[x] - sum_{j>=2} M[xj] on the device.  Host buffers; runs on
 * `stream` and returns when done.  Errors: MERTENS_EINVAL, MERTENS_ENOMEM,
 * MERTENS_ECUDA.
 */
int mertens_resolve(mertens_u128 n, uint64_t u, const uint64_t *S, int64_t *M_out, void *stream);

/*
 * The exchange step on the device, for windows run on several devices (or
 * in any order on one).  An exchange buffer holds 2 X int64 words: word
 * 2(x-1) the low and word 2(x-1)+1 the high 32-bit half of entry x's 64-bit
 * sum, so buffers can be added element-wise (an all-reduce SUM of int64 over
 * up to 2^31 windows, in any backend) without signed overflow.
 *
 * mertens_window_accumulate -- adds target i's window sums of window plan
 * `plan` (after its mertens_run), S_loc[x] + C coef[x] (mod 2^64), into the
 * exchange buffer X2_dev, where the carry C = M(y_first - 1) is the sum of
 * the mu sums of the windows below this one, mu_before[0..count) (host
 * array; each window's mu sum is the *mu_sum of mertens_window_result).
 * Sec. 2-3: every contribution of a window is affine in its carry.  Waits
 * for the plan's last run (to read its sieve status), then enqueues the
 * addition on `stream` and returns.
 * X2_dev: device, 8-byte aligned, 2 X_i int64 words, owned by the caller and
 * zeroed by the caller before the first window is added.
 * Errors: MERTENS_EINVAL (NULL or unaligned buffer, bad index, not a window
 * plan, mu_before NULL with count > 0), MERTENS_ENOTREADY (not run),
 * a sieve status of the run (MERTENS_EOVERFLOW, MERTENS_ETIMEOUT),
 * MERTENS_ECUDA.
 *
 * mertens_resolve_exchange -- mertens_resolve from an exchange buffer on the
 * device: M_dev[x-1] = M(floor(n/x)), x = 1..X = floor(n/u), from the sums
 * S[x] = X2_dev[2(x-1)] + 2^32 X2_dev[2(x-1)+1] (mod 2^64).  Both buffers are
 * device memory owned by the caller (X2_dev 2 X int64 words, M_dev X int64
 * words, 8-byte aligned).  Runs on `stream` and returns when done (its
 * scratch is allocated through the allocator hook).  Errors: MERTENS_EINVAL,
 * MERTENS_ENOMEM, MERTENS_ECUDA.
 */
int mertens_window_accumulate(mertens_plan_t plan, size_t i, const int64_t *mu_before,
                              size_t count, int64_t *X2_dev, void *stream);
int mertens_resolve_exchange(mertens_u128 n, uint64_t u, const int64_t *X2_dev, int64_t *M_dev,
                             void *stream);

/*
 * mertens_window_result -- wait for the last run of window plan `plan` and
 * return target i's partial sums: S_loc[x-1] and coef[x-1] for
 * x = 1..min(cap, X_i) (either may be NULL; uint64, mod 2^64), *len = X_i,
 * and *mu_sum = M(y_last) - M(y_first - 1), the carry the next window adds.
 * Errors: MERTENS_EINVAL (not a window plan, bad i), MERTENS_ENOTREADY,
 * MERTENS_ECUDA.
 */
int mertens_window_result(mertens_plan_t plan, size_t i, uint64_t *S_loc, uint64_t *coef,
                          size_t cap, size_t *len, int64_t *mu_sum);

/*
 * mertens_run -- enqueue the whole computation on `stream`: for every sieve
 * block, mu_sieve (segmented Moebius sieve, Sec. 3), m_scan (M(y) by prefix
 * sum with the carry of the previous block), mertens_update (every array
 * entry's contributions from the block, Sec. 2-3); then resolve (Sec. 2: the
 * final values of M follow from the update sums by the recursion).  Returns
 * once everything
 * is enqueued; the work runs asynchronously.  May be called again on the same
 * plan (the arrays are reset first).  Errors: MERTENS_EINVAL (NULL plan),
 * MERTENS_ECUDA (a launch failed).
 */
int mertens_run(mertens_plan_t plan, void *stream);

/*
 * mertens_result -- wait for the last mertens_run of `plan`, then return
 * target i's results.
 *   M_n      receives M(n_i) (may be NULL).
 *   entries  NULL, or a host buffer of `cap` int64 that receives
 *            M(floor(n_i/x)) for x = 1..min(cap, X_i) -- the paper's array
 *            of M at every floor(n/x) (Sec. 1-2).
 *   len      receives X_i (may be NULL).
 * Values are exact; they are computed mod 2^64 and read as int64, which is
 * exact while |M| < 2^63.  Errors: MERTENS_EINVAL (bad i), MERTENS_ENOTREADY
 * (no run yet), MERTENS_ETIMEOUT (a bounded device wait gave up),
 * MERTENS_EOVERFLOW (some |M(y)| of the sieve did not fit the M(y) block
 * type), MERTENS_ECUDA.
 */
int mertens_result(mertens_plan_t plan, size_t i, int64_t *M_n, int64_t *entries,
                   size_t cap, size_t *len);

/* Frees every buffer of the plan (after waiting for its last run). NULL ok. */
void mertens_destroy(mertens_plan_t plan);

/* ---- host-only planning queries (no GPU needed) ------------------------- */

/* Per-target shape of a plan or of a would-be plan. */
typedef struct {
    mertens_u128 n;          /* target                                      */
    mertens_u128 u;          /* sieve limit used                            */
    uint64_t X;              /* array length floor(n/u) (Sec. 2)            */
    uint64_t y_max;          /* largest y whose M(y) the update reads       */
    uint64_t direct_terms;   /* sum over x of floor(sqrt(floor(n/x)))       */
    uint64_t gathered_terms; /* sum over x of the j-range of gathered terms */
} mertens_query_info;

/*
 * mertens_describe -- fill `info` for target n with sieve limit u ({0,0} =
 * the library's choice), without touching the GPU.  The term counts are the
 * closed forms of the update's work (Sec. 2): entry x with k = floor(n/x) and
 * s = floor(sqrt(k)) has s direct terms M(y)(floor(k/y) - floor(k/(y+1))),
 * y = 1..s, and floor(k/(s+1)) - floor(k/u) gathered terms M(floor(k/j)),
 * j = floor(k/u)+1 .. floor(k/(s+1)).  Errors: MERTENS_EINVAL, MERTENS_ENOTSUP.
 */
int mertens_describe(mertens_u128 n, mertens_u128 u, mertens_query_info *info);

/* mertens_plan_info -- the same record for target i of an existing plan. */
int mertens_plan_info(mertens_plan_t plan, size_t i, mertens_query_info *info);

/* Run statistics.  Phase times are CUDA-event device times averaged over the
 * runs made since profiling was last enabled (0 when profiling is off). */
typedef struct {
    double total_ms;      /* whole run, first kernel to last               */
    double sieve_ms;      /* a1 mu_sieve, all blocks                        */
    double scan_ms;       /* a2 m_scan (tile carries + M(y)), all blocks    */
    double update_ms;     /* a3 mertens_update = dense + gathered           */
    double dense_ms;      /*    dense part (squarefree list + mu-form sums) */
    double gather_ms;     /*    gathered part, all blocks                   */
    double resolve_ms;    /* a4 resolve                                     */
    uint64_t runs;        /* runs averaged                                  */
    uint64_t blocks;      /* sieve blocks                                   */
    uint64_t y_sieved;    /* y values sieved                                */
    uint64_t terms;       /* direct + gathered update terms, all targets    */
    uint64_t kernels;     /* kernel launches of the last run                */
    uint64_t dense_y;     /* y values covered by the dense (mu-form) part,
                             summed over entries                            */
    uint64_t gather_j;    /* gathered terms (one per j), all entries        */
    double sieve_updates; /* sieve updates: sum over blocks of the block
                             length times sum_{p <= sqrt(block end)}
                             (1/p + 1/p^2)                                  */
    uint64_t h2d_bytes;   /* host-to-device bytes of the plan's inputs      */
    uint64_t d2h_bytes;   /* device-to-host bytes read by mertens_result
                             since the last mertens_run                     */
    uint64_t gather_j_exec; /* gathered terms evaluated: entry 2x takes the
                             terms at j' <= floor(jtop_x/2) from entry x's
                             even j (floor(floor(n/x)/2j') =
                             floor(floor(n/2x)/j')), so these are fewer
                             than gather_j                                  */
    uint64_t dense_odd_skip; /* odd y left out of the dense sums, summed over
                             entries: entry 2x takes its odd-y terms up to
                             half of entry x's cut-off from entry x's
                             even-y terms (mu(y) floor(floor(n/2x)/y) =
                             -mu(2y) floor(floor(n/x)/2y)); the squarefree
                             ones among them, about 8/pi^2 of these, are
                             not evaluated                                  */
} mertens_run_stats;

/* Enables (1) or disables (0) per-phase events for later runs of `plan`
 * and clears the runs recorded so far (off by default; the events add
 * records to the stream but serialise nothing). */
int mertens_plan_set_profiling(mertens_plan_t plan, int enable);

/* Waits for the last run and fills `stats`. */
int mertens_run_stats_get(mertens_plan_t plan, mertens_run_stats *stats);

/* ---- step-level entry points (one step of the path on device buffers) --- */

/*
 * mertens_sieve_mu -- step a1 alone: mu(y) for y = y1 .. y1+len-1 into
 * mu_dev[0..len) (int8), by the segmented log sieve (Sec. 3) with an exact
 * decision rule.  1 <= y1, y1+len-1 < 2^63, len <= 2^31.  Scratch is taken
 * from the allocator hook and freed before return (the call synchronises
 * `stream`).  Errors: MERTENS_EINVAL, MERTENS_ENOMEM, MERTENS_ECUDA.
 */
int mertens_sieve_mu(uint64_t y1, uint64_t len, int8_t *mu_dev, void *stream);

/*
 * mertens_sieve_M -- steps a1+a2: M(y) for y = y1 .. y1+len-1 into
 * M_dev[0..len) (int32), given carry = M(y1-1) (Sec. 3, step 5: the running
 * sum of mu(y)).  Same limits and scratch rule as mertens_sieve_mu.
 * MERTENS_EOVERFLOW if some |M(y)| >= 2^31.
 */
int mertens_sieve_M(uint64_t y1, uint64_t len, int64_t carry, int32_t *M_dev,
                    void *stream);

/* ---- tuning ------------------------------------------------------------ */

/*
 * Performance parameters used for plans created afterwards (process-wide).
 * None of them changes any result -- only speed (Sec. 3 likewise tunes its
 * constants and thresholds for speed alone).
 *   u_factor      automatic sieve limit
 *                 u = u_factor * g * (count * n)^(2/3), g as in
 *                 mertens_plan, clamped to (floor(sqrt(n)), n] (Sec. 2:
 *                 u = O(n^(2/3)), batched u = O((nN)^(2/3))); default 0.45
 *   dense_c       dense cut-off y_c ~ dense_c * sqrt(floor(n/x)) per entry
 *                 (the paper's regions 1/1' bound c1);     default 1.4
 *   gather_scale  multiplies the automatic end of the shared-memory gather
 *                 range;                                   default 1.0
 *   block_cap     largest automatic sieve block (0 = 2^28, or 2^30 above
 *                 2^36 sieved y); otherwise in [2^16, 2^31]
 */
typedef struct {
    double u_factor;
    double dense_c;
    double gather_scale;
    uint64_t block_cap;
} mertens_tuning;

int mertens_set_tuning(const mertens_tuning *t);  /* MERTENS_EINVAL if out of range */
int mertens_get_tuning(mertens_tuning *t);

/*
 * mertens_autotune -- times candidate tunings on the current device for the
 * targets n[0..count) (one plan per candidate, a warm-up run, then `runs`
 * timed runs with CUDA events) by coordinate search over u_factor, dense_c
 * and gather_scale, starting from the tuning in force.  Writes the fastest
 * to *best and its time per run to *best_ms; does not apply it (call
 * mertens_set_tuning).  The work is that of ~10 candidates x (runs + 1)
 * whole computations.  Errors: those of mertens_plan / mertens_run.
 */
int mertens_autotune(const mertens_u128 *n, size_t count, int runs, mertens_tuning *best,
                     double *best_ms);

/*
 * mertens_scan_extremes -- M(y) for every y in [y_first, y_last] from a known
 * carry = M(y_first - 1), by the sieve and prefix scan (Sec. 3), reduced to
 * the extremes of M(y) and of M(y)/sqrt(y) over the interval (the scan of
 * Sec. 6 around a candidate for a new extreme value).  Ratios are compared
 * exactly (M1^2 y2 against M2^2 y1 in 128 bits); ties go to the smallest y.
 * 1 <= y_first <= y_last < 2^62.  Runs on `stream`, returns when done; all
 * scratch (about 2 GB for intervals of 2^30 y or more) is allocated through
 * the allocator hook and freed before returning.
 * Errors: MERTENS_EINVAL, MERTENS_ENOTSUP (intervals of 2^46 y or more),
 * MERTENS_ENOMEM, MERTENS_ECUDA.
 */
typedef struct {
    int64_t M_last;               /* M(y_last)                                  */
    int64_t M_max, M_min;         /* largest and smallest M(y) ...              */
    uint64_t y_M_max, y_M_min;    /* ... and where                              */
    int64_t R_max_M, R_min_M;     /* M(y) at the largest and smallest M/sqrt(y) */
    uint64_t y_R_max, y_R_min;    /* ... and where                              */
    double R_max, R_min;          /* those two ratios, rounded to double        */
} mertens_extremes;
int mertens_scan_extremes(uint64_t y_first, uint64_t y_last, int64_t carry,
                          mertens_extremes *out, void *stream);

/*
 * mertens_probe_int_peaks -- measured integer rates of the current device,
 * for roofline denominators (no counterpart in the paper): the update's
 * inner step acc += mulhi64(m, 2k) >> l (terms/s), 32-bit IMAD (per s),
 * LOP3+IADD3 pairs (per s) and the shared-memory gather's quotient step
 * (float estimate of (k - t1 j)/j, truncation, one exact remainder test;
 * terms/s), each from the best of two timed runs of independent chains over
 * the whole device after one warm-up run.  Runs on `stream`, returns when
 * done.  Errors: MERTENS_EINVAL, MERTENS_ENOMEM, MERTENS_ECUDA.
 */
typedef struct {
    double mulhi_terms_per_s;
    double imad32_per_s;
    double alu_pairs_per_s;
    int sms;
    double fquot_terms_per_s;
} mertens_int_peaks;
int mertens_probe_int_peaks(mertens_int_peaks *out, void *stream);

/*
 * mertens_division_constants -- host only, no device needed: the
 * invariant-divisor constants the kernels use for divisor d (Granlund and
 * Montgomery, "Division by invariant integers using multiplication", PLDI
 * 1994, Sec. 4), so that tests can hold them to integer division.
 *   *m64, *l64: for 1 <= d < 2^63, floor(k/d) = mulhi64(m64, 2k) >> l64 for
 *     every k < 2^63 (l64 = ceil(log2 d)).
 *   *m32, *s32: for 2 <= d < 2^31, floor(v/d) = mulhi32(m32, v) >> s32 for
 *     every v < 2^31 (both 0 for other d).
 * Any output may be NULL.  Errors: MERTENS_EINVAL for d = 0 or d >= 2^63.
 * The paper names precomputed multiply-and-shift constants for small
 * divisors (Sec. 3); these are the library's own.
 */
int mertens_division_constants(uint64_t d, uint64_t *m64, uint32_t *l64, uint32_t *m32,
                               uint32_t *s32);

/* ---- serving: continuous batching of M(n) queries ---------------------- */

/*
 * A server owns one worker thread on `device`.  Queries are submitted from
 * any host thread and answered asynchronously.  The worker groups waiting
 * queries of the same magnitude class (floor(bitlength(n)/20)) into batches
 * of at most `max_batch` targets -- one plan, one shared sieve pass per
 * batch (Sec. 2: close values share the sieve; every target of a batch takes
 * u = min(n, the batch's sieve limit)) -- and keeps up to `max_inflight` batches
 * running at once, each on its own stream, admitting a new batch whenever a
 * slot is free and its estimated device memory fits what is left of
 * `mem_budget_bytes`.  Queries that arrive while others run on the GPU are
 * admitted as slots and memory free up; their work overlaps on the device.
 * Results are exact and do not depend on how queries were batched.
 *
 *   mertens_server_create: device >= 0; mem_budget_bytes = 0 means 80% of the
 *     free device memory; max_inflight 1..16 (0 = 4); max_batch 1..4096
 *     (0 = 128).  Errors: MERTENS_EINVAL, MERTENS_ECUDA, MERTENS_ENOMEM.
 *   mertens_server_submit: 1 <= n < 2^63 (else MERTENS_ENOTSUP / EINVAL);
 *     *ticket receives the query's id.
 *   mertens_server_poll: MERTENS_OK with *M_n set once the answer is there,
 *     MERTENS_ENOTREADY before, MERTENS_EINVAL for an unknown ticket, or the
 *     status the query's batch failed with.
 *   mertens_server_wait: blocks up to timeout_s (< 0: forever); MERTENS_ETIMEOUT
 *     when it runs out.
 *   mertens_server_times: host steady-clock nanoseconds of submission and of
 *     the answer (0 if not answered yet).
 *   mertens_server_destroy: finishes the admitted batches, drops queries
 *     still waiting, joins the worker and frees everything.
 */
typedef struct mertens_server_s *mertens_server_t;

typedef struct {
    uint64_t submitted;      /* queries submitted                          */
    uint64_t answered;       /* queries answered                           */
    uint64_t batches;        /* batches (plans) run                        */
    uint64_t max_inflight;   /* most batches in flight at once             */
    uint64_t max_batch_seen; /* largest batch                              */
    uint64_t failed;         /* queries whose batch failed                 */
} mertens_server_stats;

int mertens_server_create(mertens_server_t *out, int device, size_t mem_budget_bytes,
                          uint32_t max_inflight, uint32_t max_batch);
int mertens_server_submit(mertens_server_t srv, mertens_u128 n, uint64_t *ticket);
/*
 * mertens_server_use_table: batches admitted from now on whose targets are all
 * <= the table's n_max are planned on `table` (mertens_plan_on_table: no
 * sieve; u = min(n, y_max + 1)); others, and any batch the table cannot
 * serve, get ordinary plans.  NULL detaches.  The table must be on the
 * server's device and outlive the server's use of it.
 * Errors: MERTENS_EINVAL.
 */
int mertens_server_use_table(mertens_server_t srv, mertens_table_t table);
int mertens_server_poll(mertens_server_t srv, uint64_t ticket, int64_t *M_n);
int mertens_server_wait(mertens_server_t srv, uint64_t ticket, int64_t *M_n, double timeout_s);
int mertens_server_times(mertens_server_t srv, uint64_t ticket, uint64_t *t_submit_ns,
                         uint64_t *t_done_ns);
int mertens_server_stats_get(mertens_server_t srv, mertens_server_stats *stats);
void mertens_server_destroy(mertens_server_t srv);

/*
 * mertens_sieve_M_noalloc -- the same result as mertens_sieve_M (M(y) for
 * y = y1 .. y1+len-1 into M_dev as int32, given carry = M(y1-1)), for callers
 * that cannot allocate device memory: for example code that runs inside a
 * framework which has reserved the device memory for its own pool, or a
 * latency-critical loop that cannot afford the device-wide synchronisation
 * and the possible failure of cudaMalloc/cudaFree.  The paper has no
 * counterpart; this is a property of the library, not of the method.
 *
 * All scratch (prime table, pre-sieve pattern, int16 partial sums, segment
 * offsets, carry and status words; about 6.2 MB) lives in one fixed device
 * array inside the library, held on every GPU that loads the library until
 * the process exits.  Limits: 1 <= len <= 2^21 and y1 + len - 1 < 2^40,
 * otherwise MERTENS_EINVAL with an explanatory mertens_last_error().
 * The call allocates no device memory and no host heap memory.  It sieves
 * with the 16-bit log-sieve kernel (the allocating call takes the byte
 * kernel where that one is exact); the results are the same.
 *
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture on the
 * device.  Every call uses the same array and leaves its contents behind, so
 * calls that overlap on the GPU race: serialise them (one stream, or wait for
 * one call before starting another).  The call synchronises `stream`.
 * M_dev: device, 4-byte aligned, len int32, owned by the caller.
 * Errors: MERTENS_EINVAL, MERTENS_EOVERFLOW (some |M(y)| >= 2^31),
 * MERTENS_ECUDA.
 */
int mertens_sieve_M_noalloc(uint64_t y1, uint64_t len, int64_t carry, int32_t *M_dev,
                            void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LIBMERTENS_H */
