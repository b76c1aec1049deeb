// libmertens C ABI: planning, the block loop of mertens_run, results.
// The method is that of arXiv:1108.0135, Sec. 2-3; the kernels live in
// sieve.cu (a1, a2) and update.cu (a3, a4).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/libmertens.h"
#include "common.cuh"
#include "internal.h"
#include "update.h"

namespace mert {

// Runs f(lo, hi) over [0, n) in contiguous pieces of at least min_piece on up
// to 16 host threads (host planning only; f must not throw).  Falls back to
// the calling thread alone when a thread cannot be started.
template <typename F>
static void parallel_for(size_t n, size_t min_piece, const F &f)
{
    const unsigned hw = std::thread::hardware_concurrency();
    size_t nt = std::min<size_t>(hw ? hw : 1, 16);
    nt = std::min(nt, std::max<size_t>(1, n / std::max<size_t>(min_piece, 1)));
    if (nt <= 1) {
        f((size_t)0, n);
        return;
    }
    const size_t step = (n + nt - 1) / nt;
    std::vector<std::thread> th;
    size_t done_from = step;  // pieces from here on not started on a thread
    try {
        for (size_t lo = step; lo < n; lo += step) {
            th.emplace_back([&f, lo, n, step]() { f(lo, std::min(n, lo + step)); });
            done_from = lo + step;
        }
    } catch (...) {
    }
    f((size_t)0, std::min(n, step));
    if (done_from < n)
        f(done_from, n);
    for (auto &t : th)
        t.join();
}

// ---------------------------------------------------------------------------
// Errors and allocation.
// ---------------------------------------------------------------------------
static thread_local char g_last_error[512] = "";

void set_last_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

static std::mutex g_alloc_mu;
static mertens_alloc_fn g_alloc = nullptr;
static mertens_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;

Allocator current_allocator()
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    Allocator a;
    a.alloc = g_alloc;
    a.release = g_free;
    a.ctx = g_alloc_ctx;
    return a;
}

// Default device memory: stream-ordered allocation on one non-blocking
// library stream per device, so that creating or destroying a plan never
// waits for other work on the device (the allocation is made usable on every
// stream by waiting for that stream alone).  Freed memory stays in the
// process's default pool for reuse.
constexpr int kMaxDevices = 64;
static cudaStream_t g_alloc_stream[kMaxDevices];

static cudaStream_t alloc_stream()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return nullptr;
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (!g_alloc_stream[dev]) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            return nullptr;
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        g_alloc_stream[dev] = s;
    }
    return g_alloc_stream[dev];
}

void *dev_alloc(const Allocator &a, size_t bytes)
{
    if (bytes == 0)
        bytes = 16;
    if (a.alloc)
        return a.alloc(bytes, nullptr, a.ctx);
    void *p = nullptr;
    cudaStream_t s = alloc_stream();
    if (!s || cudaMallocAsync(&p, bytes, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

// Callers free only memory no queued work still uses.
void dev_free(const Allocator &a, void *p, size_t bytes)
{
    if (!p)
        return;
    if (a.alloc) {
        a.release(p, bytes, nullptr, a.ctx);
        return;
    }
    cudaStream_t s = alloc_stream();
    if (s)
        cudaFreeAsync(p, s);
}

static uint64_t isqrt64(uint64_t v)
{
    uint64_t r = (uint64_t)std::sqrt((double)v);
    while (r > 0 && r > v / r)
        --r;
    while ((r + 1) <= v / (r + 1))
        ++r;
    return r;
}

typedef unsigned __int128 u128;
constexpr u128 kTwo63 = (u128)1 << 63;

static u128 to_u128(mertens_u128 v) { return ((u128)v.hi << 64) | v.lo; }

// floor(sqrt(v)) for v < 2^128: a double estimate, one Newton step, then
// exact +-1 corrections on 128-bit squares.
static uint64_t isqrt128(u128 v)
{
    if (v < kTwo63)
        return isqrt64((uint64_t)v);
    u128 r = (u128)std::sqrt((double)v);
    r = (r + v / r) / 2;
    while (r * r > v)
        --r;
    while ((r + 1) * (r + 1) <= v)
        ++r;
    return (uint64_t)r;
}

// Entries with k at or above this take the two-word kernel: 2^63, or a
// lower MERTENS_WIDE_FROM (so that tests can run that kernel on targets the
// oracle reaches).  k = 1 never does (the split form needs k >= 2).
static u128 wide_threshold()
{
    const char *e = getenv("MERTENS_WIDE_FROM");
    if (e) {
        const unsigned long long v = strtoull(e, nullptr, 10);
        if (v >= 2 && v < (1ull << 63))
            return v;
    }
    return kTwo63;
}

}  // namespace mert

using namespace mert;

// ---------------------------------------------------------------------------
// The plan.
// ---------------------------------------------------------------------------
// Phases of a run timed with CUDA events when profiling is on.
enum { kPhSieve = 0, kPhScan = 1, kPhDense = 2, kPhGather = 3, kPhResolve = 4, kPhTotal = 5,
       kPhases = 6 };

struct PhaseEvents {
    int phase;
    cudaEvent_t a, b;
};

struct mertens_plan_s {
    Allocator al;
    std::vector<std::pair<void *, size_t>> allocs;
    // targets
    size_t nq = 0;
    std::vector<uint64_t> n, n_hi, u, X, off;
    std::vector<uint64_t> direct, gathered, ymax_q;
    uint64_t nent = 0;
    uint64_t y_max = 0, block_len = 0, nblocks = 0, ydense = 0, jmax = 0, mg_n = 0;
    uint32_t gquot = 1;  // GatherArgs::quot of this plan
    // sieved range: [1, y_max] for a whole run; a window plan runs only the
    // blocks of [y_first, y_last], with M(y_first - 1) taken as 0, and returns
    // per entry S_loc and the coefficient of that carry (coef)
    uint64_t y_first = 1, y_last = 0;
    bool window = false;
    std::vector<uint64_t> coef;
    uint64_t *dcoef = nullptr;  // the same on the device (window plans)
    // plans on a resident table: M(y), the divisor magics and the dense list
    // are the table's; targets n <= table y_max are read from it directly
    // (entry, y) pairs
    mertens_table_s *table = nullptr;
    bool sieves = true;  // some block is sieved (always without a table)
    std::vector<uint64_t> lookups;
    uint64_t *dlook = nullptr;
    mertens_tuning tuning{};
    uint64_t terms = 0, dense_y = 0, gather_j = 0;
    double sieve_updates = 0;
    // device buffers
    PrimeTable pt;
    uint64_t *dK = nullptr, *dJLO = nullptr, *dJC0 = nullptr, *dJCUR = nullptr, *dYCE = nullptr;
    uint32_t *dEMIT = nullptr;
    uint64_t gather_j_exec = 0;  // gathered terms evaluated (after sharing)
    uint64_t dense_odd_skip = 0; // odd y left out of dense sums (taken from entries x/2)
    uint64_t *dS = nullptr, *dR = nullptr;
    // chunks of the global gather's heavy entries, per block (qcap records)
    uint4 *dqueue = nullptr;
    uint32_t *dqlen = nullptr;
    uint32_t qcap = 0;
    int8_t *dmu_aux = nullptr;
    int16_t *dMloc[2] = {nullptr, nullptr};      // sieve output, two blocks in flight
    int32_t *dsegsum[2] = {nullptr, nullptr};
    int64_t *dsegoff[2] = {nullptr, nullptr};
    int64_t *dcarry = nullptr;
    // streams and events of a run (sieve chain, gathered updates, dense part)
    bool serial = false;
    cudaStream_t st_sieve = nullptr, st_upd = nullptr, st_dense = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_reset = nullptr, ev_dense_done = nullptr;
    cudaEvent_t ev_sieve_done = nullptr, ev_join = nullptr;
    std::vector<cudaEvent_t> ev_sieved, ev_upd;
    uint32_t *dcounter_dense = nullptr, *dcounter_gather = nullptr;
    // shared-memory gather path: tiles and items of every block, item range
    // [gblk[b], gblk[b+1]) and last y covered, per block
    GatherTile *dgtiles = nullptr;
    GatherItem *dgitems = nullptr;
    std::vector<uint32_t> gblk;
    std::vector<uint64_t> gend;
    std::vector<uint64_t> ktile;  // per block: entries with k >= this take its tiles
    uint64_t gather_smem_end = 0;
    uint32_t *derr = nullptr, *dcounter = nullptr;
    uint64_t *dMG = nullptr, *ddl_m = nullptr;
    uint16_t *ddl_yo = nullptr;
    uint2 *ddl_cnt = nullptr;
    Group *dgroups = nullptr;
    DenseItem *ditems = nullptr;
    uint32_t nitems = 0;
    QueryDev *dqs = nullptr;
    // entries with k >= 2^63 (targets n >= 2^63) and the wide kernel's
    // grid width per block (0: no terms in the block)
    std::vector<WideEntry> wide;
    WideEntry *dwide = nullptr;
    std::vector<uint32_t> wide_grid;
    bool mg_built = false;
    // run state
    cudaEvent_t done = nullptr;
    bool ran = false;
    bool prof = false;
    std::vector<PhaseEvents> evs;  // every timed phase since profiling was enabled
    uint64_t prof_runs = 0;
    uint64_t kernels = 0;
    uint64_t h2d_bytes = 0, d2h_bytes = 0;
    // captured whole run (replayed by later runs)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    uint64_t graph_kernels = 0;

    template <typename T>
    T *alloc(size_t count)
    {
        size_t bytes = count * sizeof(T);
        void *p = dev_alloc(al, bytes);
        if (p)
            allocs.push_back({p, bytes});
        return (T *)p;
    }
};

// y range of block b of a plan.
static void block_range(const mertens_plan_s *p, uint64_t b, uint64_t *y1, uint64_t *y2)
{
    *y1 = p->y_first + b * p->block_len;
    *y2 = std::min(*y1 + p->block_len - 1, p->y_last);
}

// Tuning in force for new plans (mertens_set_tuning); MERTENS_* environment
// variables override single fields for experiments.
static std::mutex g_tune_mu;
static mertens_tuning g_tuning = {0.45, 1.4, 1.0, 0};

static mertens_tuning tuning_now()
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tuning;
}

static double dense_factor(const mertens_tuning &t)
{
    const char *e = getenv("MERTENS_DENSE_C");
    double c = e ? atof(e) : t.dense_c;
    return c > 0 ? c : 1.4;
}

// Shape of one target (host only): X, y_max and the closed-form term counts.
static int describe_target(u128 n, uint64_t u, uint64_t *X, uint64_t *direct,
                           uint64_t *gathered)
{
    *X = (uint64_t)(n / u);
    uint64_t d = 0, g = 0;
    for (uint64_t x = 1; x <= *X; ++x) {
        const u128 k = n / x;
        const uint64_t s = isqrt128(k);
        const uint64_t jlo = *X / x + 1, jhi = (uint64_t)(k / ((u128)s + 1));
        d += s;
        if (jhi >= jlo)
            g += jhi - jlo + 1;
    }
    *direct = d;
    *gathered = g;
    return 0;
}

// Sieve limit of one target given the batch's shared limit ub: as large as
// ub but above floor(sqrt(n)) and at most n.
static uint64_t target_u(u128 n, double ub)
{
    if (n <= 3)
        return (uint64_t)n;
    uint64_t u = ub >= 1.8e19 ? UINT64_MAX : (uint64_t)ub;
    const uint64_t r = isqrt128(n);
    if (u <= r)
        u = r + 1;
    if ((u128)u > n)
        u = (uint64_t)n;
    return u;
}

// Shared sieve limit of a batch: ub = f g (sum n)^(2/3).  The sieve costs
// ~ub and the update ~sum_i n_i/sqrt(u_i) (Sec. 2), balanced at
// ub ~ (sum n)^(2/3); every target then takes u_i = min(n_i, ub) (a small
// target costs no extra sieve and fewer terms the larger its u).  f = 0.45 by
// default; g = clamp((max n / 1e18)^(-1/4), 1, 1.78) raises the limit for
// batches whose largest target is below 1e18.  Both are timings on GB300:
// M(1e18) alone runs fastest at 0.45 (its upper blocks take the bucketed
// sieve kernel, dearer per y), 1e17 alone and a batch of 64 targets near
// 1e17 at about 0.8 (0.770 s against 0.834 s; 15.8 s against 18.6 s).
static double batch_ub(const std::vector<u128> &ns, const mertens_tuning &t)
{
    const char *e = getenv("MERTENS_U_FACTOR");
    const double f = e ? atof(e) : (t.u_factor > 0 ? t.u_factor : 0.45);
    double sum = 0, mx = 0;
    for (u128 n : ns) {
        sum += (double)n;
        mx = std::max(mx, (double)n);
    }
    if (mx <= 0)
        return 1;
    const double g = std::min(1.78, std::max(1.0, std::pow(mx / 1e18, -0.25)));
    return f * g * std::pow(sum, 2.0 / 3.0);
}

static uint64_t auto_u(u128 n, size_t count, const mertens_tuning &t)
{
    std::vector<u128> ns(count ? count : 1, n);
    return target_u(n, batch_ub(ns, t));
}

namespace mert {
// Dense cut-off factor of new plans (c in y_c ~ c sqrt(k)).
double plan_dense_factor() { return dense_factor(tuning_now()); }
// The sieve limits the library picks for the targets of a batch.
std::vector<uint64_t> plan_auto_u(const std::vector<uint64_t> &ns)
{
    std::vector<u128> v(ns.begin(), ns.end());
    const double ub = batch_ub(v, tuning_now());
    std::vector<uint64_t> out;
    for (uint64_t n : ns)
        out.push_back(target_u(n, ub));
    return out;
}
// Device bytes a plan holds (its buffers and its prime table).
size_t plan_device_bytes(mertens_plan_t p)
{
    if (!p)
        return 0;
    size_t b = 0;
    for (auto &a : p->allocs)
        b += a.second;
    b += (size_t)p->pt.np * 25 + 2 * kPatternWords * 4;
    return b;
}
}  // namespace mert

// Sieve limit of a target on a resident table of M(y), y <= y_max: at least
// as large as the table reaches (its part of the sieve costs nothing, and the
// update's terms fall as 1/sqrt(u)), and at least the automatic limit of a
// sieving plan; blocks above y_max are sieved as usual.
static uint64_t on_table_u(u128 n, double ub, uint64_t y_max)
{
    const u128 t = (u128)y_max + 1;
    const uint64_t ut = (uint64_t)(n < t ? n : t);
    const uint64_t ua = target_u(n, ub);
    return ut > ua ? ut : ua;
}

static int check_u(u128 n, uint64_t u)
{
    if (n == 1)
        return u == 1 ? MERTENS_OK : MERTENS_EINVAL;
    const uint64_t r = isqrt128(n);
    if (u <= r || (u128)u > n)
        return MERTENS_EINVAL;
    return MERTENS_OK;
}

// Limits of this build: n < 2^127 (u < 2^64 then follows from u <= n for
// n < 2^64, and is required above it), X = floor(n/u) < 2^32 entries.
static int check_n(mertens_u128 n, const char *who, size_t i)
{
    if (n.lo == 0 && n.hi == 0) {
        set_last_error("%s: n[%zu] = 0", who, i);
        return MERTENS_EINVAL;
    }
    if (n.hi >= (1ull << 63)) {
        set_last_error("%s: n[%zu] >= 2^127", who, i);
        return MERTENS_EINVAL;
    }
    return MERTENS_OK;
}

extern "C" {

const char *mertens_strerror(int code)
{
    switch (code) {
    case MERTENS_OK: return "ok";
    case MERTENS_EINVAL: return "invalid argument";
    case MERTENS_ENOMEM: return "out of memory";
    case MERTENS_ECUDA: return "CUDA runtime error";
    case MERTENS_ETIMEOUT: return "bounded device wait expired";
    case MERTENS_ENOTREADY: return "no run to read";
    case MERTENS_ENOTSUP: return "not supported by this build";
    case MERTENS_EOVERFLOW: return "integer overflow in M(y) block";
    default: return "unknown status";
    }
}

const char *mertens_last_error(void) { return g_last_error; }

int mertens_set_allocator(mertens_alloc_fn alloc, mertens_free_fn release, void *ctx)
{
    if (alloc && !release) {
        set_last_error("mertens_set_allocator: alloc without release");
        return MERTENS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = alloc ? release : nullptr;
    g_alloc_ctx = alloc ? ctx : nullptr;
    return MERTENS_OK;
}

int mertens_describe(mertens_u128 n, mertens_u128 u, mertens_query_info *info)
{
    if (!info) {
        set_last_error("mertens_describe: NULL info");
        return MERTENS_EINVAL;
    }
    if (check_n(n, "mertens_describe", 0) != MERTENS_OK)
        return MERTENS_EINVAL;
    if (u.hi != 0) {
        set_last_error("mertens_describe: u >= 2^64 is not supported by this build");
        return MERTENS_ENOTSUP;
    }
    const u128 nn = to_u128(n);
    uint64_t uu = u.lo ? u.lo : auto_u(nn, 1, tuning_now());
    if (check_u(nn, uu) != MERTENS_OK) {
        set_last_error("mertens_describe: u must satisfy floor(sqrt(n)) < u <= n");
        return MERTENS_EINVAL;
    }
    if (nn / uu >= ((u128)1 << 32)) {
        set_last_error("mertens_describe: n/u >= 2^32 array entries");
        return MERTENS_ENOTSUP;
    }
    memset(info, 0, sizeof(*info));
    info->n = n;
    info->u.lo = uu;
    uint64_t X, d, g;
    describe_target(nn, uu, &X, &d, &g);
    info->X = X;
    info->direct_terms = d;
    info->gathered_terms = g;
    // largest y read: the direct range ends at s <= sqrt(n); the gathered
    // range of x = 1 ends at floor(n/(X+1)).
    const uint64_t r = isqrt128(nn);
    const uint64_t yg = (uint64_t)(nn / ((u128)X + 1));
    info->y_max = std::max(r, yg);
    return MERTENS_OK;
}

static int plan_create(mertens_plan_t *out, const mertens_u128 *n, size_t count, mertens_u128 u,
                       uint64_t block_len, const mertens_tuning &tn, bool window = false,
                       uint64_t w_first = 1, uint64_t w_last = UINT64_MAX,
                       mertens_table_s *table = nullptr)
{
    if (!out)
        return MERTENS_EINVAL;
    *out = nullptr;
    if (!n || count == 0 || count > (1u << 20)) {
        set_last_error("mertens_plan: need 1 <= count <= 2^20 targets");
        return MERTENS_EINVAL;
    }
    if (u.hi != 0) {
        set_last_error("mertens_plan: u >= 2^64 is not supported by this build");
        return MERTENS_ENOTSUP;
    }
    for (size_t i = 0; i < count; ++i)
        if (check_n(n[i], "mertens_plan", i) != MERTENS_OK)
            return MERTENS_EINVAL;
    std::vector<u128> n128(count);
    for (size_t i = 0; i < count; ++i)
        n128[i] = to_u128(n[i]);
    const double ub = batch_ub(n128, tn);
    for (size_t i = 0; i < count; ++i) {
        const u128 nn = to_u128(n[i]);
        if (u.lo != 0 && check_u(nn, u.lo) != MERTENS_OK) {
            set_last_error("mertens_plan: u = %llu invalid for n[%zu] "
                           "(need floor(sqrt(n)) < u <= n)",
                           (unsigned long long)u.lo, i);
            return MERTENS_EINVAL;
        }
        if (table) {
            const u128 nmax = ((u128)table->n_max_hi << 64) | table->n_max_lo;
            if (nn > nmax) {
                set_last_error("mertens_plan_on_table: n[%zu] is beyond the table's n_max", i);
                return MERTENS_ENOTSUP;
            }
        }
        const uint64_t uu = u.lo ? u.lo : (table ? on_table_u(nn, ub, table->y_max)
                                                 : target_u(nn, ub));
        if (nn / uu >= ((u128)1 << 32)) {
            set_last_error("mertens_plan: n[%zu]/u >= 2^32 array entries", i);
            return MERTENS_ENOTSUP;
        }
    }
    mertens_plan_s *p = new (std::nothrow) mertens_plan_s();
    if (!p)
        return MERTENS_ENOMEM;
    p->al = current_allocator();
    p->nq = count;
    p->tuning = tn;
    const double dc = dense_factor(tn);

    // ---- per-entry host planning ----
    std::vector<uint64_t> K, JLO, JC0, YCE;
    std::vector<Group> groups;
    const char *share_env = getenv("MERTENS_SHARE");
    const bool share_dense = !window && !(share_env && share_env[0] == '0');
    for (size_t i = 0; i < count; ++i) {
        const u128 nn = to_u128(n[i]);
        const uint64_t uu = u.lo ? u.lo : (table ? on_table_u(nn, ub, table->y_max)
                                                 : target_u(nn, ub));
        const uint64_t X = (uint64_t)(nn / uu);
        p->n.push_back((uint64_t)nn);
        p->n_hi.push_back((uint64_t)(nn >> 64));
        p->u.push_back(uu);
        p->X.push_back(X);
        p->off.push_back(K.size());
        uint64_t d = 0, g = 0, ymq = 0;
        if (table && nn <= table->y_max && X == 1) {
            // M(n) is in the table: one entry, no terms, read after resolve
            p->lookups.push_back(K.size());
            p->lookups.push_back((uint64_t)nn);
            K.push_back(0);
            JLO.push_back(1);
            YCE.push_back(0);
            JC0.push_back(0);
            Group G;
            G.first = (uint32_t)(K.size() - 1);
            G.count = 1;
            G.pred = 1;
            G.emit = 0;
            G.yc = 0;
            G.olo = 0;
            G.x0 = 1;
            G.stride = 1;
            groups.push_back(G);
            p->direct.push_back(0);
            p->gathered.push_back(0);
            p->ymax_q.push_back(0);
            continue;
        }
        // blocks of 64 consecutive x share a dense cut-off; each is two groups
        // of 32 (odd x, even x), so the entries x/2 of an even group lie in
        // one earlier block and share its cut-off (the dense form's sharing)
        const size_t gstart = groups.size();  // this target's groups: two per block
        std::vector<uint64_t> S_(64), VH(64);
        std::vector<uint8_t> WD(64);
        const u128 wide_from = wide_threshold();
        // per entry, on host threads: k = floor(n/x) (0 for a two-word entry),
        // s = floor(sqrt(k)) and the top of its valid dense cut-offs
        std::vector<uint64_t> Kx(X), Sx(X), VHx(X), JLx(X);
        parallel_for(X, 4096, [&](size_t lo, size_t hi) {
            for (size_t i = lo; i < hi; ++i) {
                const uint64_t x = i + 1;
                const u128 k128 = nn / x;
                JLx[i] = X / x + 1;  // = floor(k/u) + 1
                if (k128 >= wide_from) {
                    Kx[i] = Sx[i] = VHx[i] = 0;
                    continue;
                }
                const uint64_t k = (uint64_t)k128, sq = isqrt64(k), jlo = JLx[i];
                Kx[i] = k;
                Sx[i] = sq;
                // valid dense cut-offs: [s, floor(k/jlo) - 1] when the entry
                // has gathered terms, else exactly s
                VHx[i] = (jlo <= k / (sq + 1)) ? (k / jlo - 1) : sq;
            }
        });
        for (uint64_t x0 = 1; x0 <= X; x0 += 64) {
            const uint32_t cnt = (uint32_t)std::min<uint64_t>(64, X - x0 + 1);
            uint64_t lo = 0, hi = UINT64_MAX, kf = 0;
            bool any_wide = false;
            for (uint32_t t = 0; t < cnt; ++t) {
                const uint64_t x = x0 + t;
                const uint64_t jlo = JLx[x - 1];
                if (Kx[x - 1] == 0) {
                    const u128 k128 = nn / x;
                    // two-word entry: its own kernel; k = 0 (no terms) here
                    WideEntry W;
                    W.k_lo = (uint64_t)k128;
                    W.k_hi = (uint64_t)(k128 >> 64);
                    W.s = isqrt128(k128);
                    W.jlo = jlo;
                    W.jhi = (uint64_t)(k128 / ((u128)W.s + 1));
                    W.e = K.size();
                    p->wide.push_back(W);
                    d += W.s;
                    uint64_t need = W.s;
                    if (W.jhi >= W.jlo) {
                        g += W.jhi - W.jlo + 1;
                        need = std::max(need, (uint64_t)(k128 / W.jlo));
                    }
                    ymq = std::max(ymq, need);
                    S_[t] = 0;
                    VH[t] = 0;
                    WD[t] = 1;
                    any_wide = true;
                    K.push_back(0);
                    JLO.push_back(1);
                    continue;
                }
                const uint64_t k = Kx[x - 1], s = Sx[x - 1], vh = VHx[x - 1];
                S_[t] = s;
                VH[t] = vh;
                WD[t] = 0;
                if (kf == 0)
                    kf = k;
                lo = std::max(lo, s);
                hi = std::min(hi, vh);
                d += s;
                K.push_back(k);
                JLO.push_back(jlo);
            }
            uint64_t target = (uint64_t)(dc * std::sqrt((double)kf));
            target = ((target + 1 + kChunk - 1) / kChunk) * kChunk - 1;  // chunk aligned
            Group G;
            G.first = (uint32_t)(K.size() - cnt);
            G.count = cnt;
            G.emit = 0;
            G.olo = 0;
            G.x0 = (uint32_t)x0;
            G.stride = 1;
            if (any_wide) {
                // per-entry cut-offs; the two-word entries take none
                G.pred = 1;
                G.yc = 0;
                for (uint32_t t = 0; t < cnt; ++t) {
                    const uint64_t yc =
                        WD[t] ? 0 : std::min(std::max(target, S_[t]), VH[t]);
                    YCE.push_back(yc);
                    G.yc = std::max(G.yc, yc);
                }
            } else if (lo <= hi) {
                const uint64_t yc = std::min(std::max(target, lo), hi);
                G.pred = 0;
                G.yc = yc;
                for (uint32_t t = 0; t < cnt; ++t)
                    YCE.push_back(yc);
            } else {
                G.pred = 1;
                G.yc = 0;
                for (uint32_t t = 0; t < cnt; ++t) {
                    const uint64_t yc = std::min(std::max(target, S_[t]), VH[t]);
                    YCE.push_back(yc);
                    G.yc = std::max(G.yc, yc);
                }
            }
            {
                // the block as two stride-2 groups (odd x, then even x)
                Group H = G;
                H.stride = 2;
                H.count = (cnt + 1) / 2;
                groups.push_back(H);
                if (cnt > 1) {
                    H.first = G.first + 1;
                    H.x0 = G.x0 + 1;
                    H.count = cnt / 2;
                    groups.push_back(H);
                }
            }
        }
        {
            // per entry, on host threads: the top of the gathered range
            // JC0 = floor(k/(yc+1)), the largest y it needs, and the totals
            const size_t o = p->off.back();
            JC0.resize(o + X, 0);
            struct Part {
                uint64_t ymq = 0, ydense = 0, jmax = 0, dense_y = 0, gather_j = 0, g = 0;
            };
            const size_t npart = 64;
            std::vector<Part> parts(npart);
            const size_t per = (X + npart - 1) / npart;
            parallel_for(npart, 1, [&](size_t lo, size_t hi) {
                for (size_t q = lo; q < hi; ++q) {
                    Part &P = parts[q];
                    for (size_t i = q * per; i < std::min<size_t>(X, (q + 1) * per); ++i) {
                        const size_t e = o + i;
                        const uint64_t k = K[e];
                        if (k == 0)
                            continue;  // two-word entry (counted with the others above)
                        const uint64_t yc = YCE[e], jc0 = k / (yc + 1);
                        JC0[e] = jc0;
                        uint64_t need = yc;
                        if (JLO[e] <= jc0)
                            need = std::max(need, k / JLO[e]);
                        P.ymq = std::max(P.ymq, need);
                        P.ydense = std::max(P.ydense, yc);
                        P.jmax = std::max(P.jmax, jc0);
                        P.dense_y += yc;
                        if (jc0 >= JLO[e])
                            P.gather_j += jc0 - JLO[e] + 1;
                        const uint64_t jhi = k / (Sx[i] + 1);  // the split form's t = s + 1
                        if (jhi >= JLO[e])
                            P.g += jhi - JLO[e] + 1;
                    }
                }
            });
            for (const Part &P : parts) {
                ymq = std::max(ymq, P.ymq);
                p->ydense = std::max(p->ydense, P.ydense);
                p->jmax = std::max(p->jmax, P.jmax);
                p->dense_y += P.dense_y;
                p->gather_j += P.gather_j;
                g += P.g;
            }
        }
        // ---- the dense form's terms shared between entries x and 2x ----
        // mu(y) floor(floor(n/2x)/y) = -mu(2y) floor(floor(n/x)/2y) for odd y,
        // and the even squarefree y' <= yc_x are exactly 2y for the odd
        // squarefree y <= floor(yc_x/2).  So the even group of block M
        // (x = 64M + 2, ..., whose x/2 = 32M + 1, ... lie in block M/2) leaves
        // out its odd y <= b = floor(yc/2) of that block's common cut-off when
        // b is within every one of its entries' cut-offs, and those x/2 add
        // minus their even-y sums to it.  Not in window plans (their dense
        // part is cut to the window's y, which 2y can leave).
        if (share_dense) {
            const size_t nblk = (X + 63) / 64;
            for (size_t M = 0; M < nblk; ++M) {
                const size_t gr = gstart + 2 * M + 1;  // even group of block M
                if (64 * M + 2 > X || gr >= groups.size())
                    continue;
                Group &R = groups[gr];
                const Group &Sg = groups[gstart + 2 * (M / 2)];
                if (Sg.pred || Sg.yc < 2)
                    continue;
                const uint64_t b = Sg.yc / 2;
                bool ok = true;
                for (uint32_t t = 0; t < R.count && ok; ++t) {
                    const size_t e = (size_t)R.first + 2 * t;
                    ok = K[e] != 0 && b <= YCE[e];
                }
                if (!ok)
                    continue;
                R.olo = b;
                p->dense_odd_skip += (b + 1) / 2 * (uint64_t)R.count;
                for (uint32_t t = 0; t < R.count; ++t) {
                    const uint64_t xs = 32 * M + 1 + t;       // source x
                    const uint64_t o = xs - (64 * (M / 2) + 1);  // offset in its block
                    groups[gstart + 2 * (M / 2) + (o & 1)].emit |= 1u << (o >> 1);
                }
            }
        }
        p->direct.push_back(d);
        p->gathered.push_back(g);
        p->ymax_q.push_back(ymq);
        p->terms += d + g;
        p->y_max = std::max(p->y_max, ymq);
    }
    p->nent = K.size();
    if (p->nent >= (1ull << 32)) {
        set_last_error("mertens_plan: more than 2^32 array entries");
        delete p;
        return MERTENS_ENOTSUP;
    }
    // ---- gathered terms shared along chains x, 2x, 4x, 8x, 16x ----
    // floor(floor(n/x)/j) = floor(n/(x j)), so entry 2x's term at j' is entry
    // x's term at j = 2j'.  The link x -> 2x (one-word entries of one target)
    // is valid when h = floor(JC0_x/2) lies in [JLO_2x, JC0_2x]: entry x's
    // whole range then holds, at its even j, exactly entry 2x's terms
    // j' in [JLO_2x, h] (JLO = floor(X/x) + 1 on both sides), so entry 2x
    // evaluates only j' > h itself.  The j' <= h are the terms of x's whole
    // range, which x and the entries before it in the chain evaluate: each
    // entry adds the sum of its own terms at j = 0 mod 2^s to entry 2^s x
    // along valid links.  Chains restart at every x whose power of two is
    // 0 mod 5 (at most four links, the four levels of the kernels' sums).
    // JOWN replaces JLO on the device; the host keeps JLO for the rest.
    std::vector<uint64_t> JOWN(JLO);
    std::vector<uint32_t> EMIT(K.size(), 0u);
    {
        const char *e = getenv("MERTENS_SHARE");
        const bool share = !(e && e[0] == '0');
        std::vector<uint8_t> link;
        for (size_t i = 0; share && i < count; ++i) {
            const uint64_t o = p->off[i], X = p->X[i];
            if (X < 2)
                continue;
            link.assign(X / 2 + 1, 0);
            // x < 2^29: EMIT holds x in 29 bits (larger x take no part)
            for (uint64_t x = 1; 2 * x <= X && x < (1ull << 29); ++x) {
                if (__builtin_ctzll(2 * x) % (kShareLevels + 1) == 0)
                    continue;  // 2x starts a chain
                const size_t e1 = o + x - 1, e2 = o + 2 * x - 1;
                if (!K[e1] || !K[e2])
                    continue;
                const uint64_t h = JC0[e1] / 2;
                if (h < JLO[e2] || h > JC0[e2])
                    continue;
                link[x] = 1;
                JOWN[e2] = h + 1;
            }
            for (uint64_t x = 1; 2 * x <= X && x < (1ull << 29); ++x) {
                uint32_t L = 0;
                for (uint64_t y = x; L < kShareLevels && 2 * y <= X && link[y]; y *= 2)
                    ++L;
                if (L)
                    EMIT[o + x - 1] = (uint32_t)x | (L << 29);
            }
        }
        for (size_t e2 = 0; e2 < K.size(); ++e2)
            if (K[e2] && JC0[e2] >= JOWN[e2])
                p->gather_j_exec += JC0[e2] - JOWN[e2] + 1;
    }
    p->table = table;
    if (table) {
        if (block_len == 0)
            block_len = 1ull << 30;
        if (block_len % kSegY) {
            set_last_error("mertens_plan_on_table: block_len must be a multiple of %d", kSegY);
            delete p;
            return MERTENS_EINVAL;
        }
    }
    p->window = window;
    p->y_first = window ? w_first : 1;
    p->y_last = window ? std::min(w_last, p->y_max) : p->y_max;
    const uint64_t span = p->y_last >= p->y_first ? p->y_last - p->y_first + 1 : 0;
    if (block_len == 0) {
        // one block when it fits 2^28 y, else 2^28 (up to 2^36 y) or 2^30 y blocks
        uint64_t cap = p->y_last > (1ull << 36) ? (1ull << 30) : (1ull << 28);
        if (tn.block_cap >= kSieveTile && tn.block_cap <= (1ull << 31))
            cap = tn.block_cap;
        block_len = std::max<uint64_t>(
            1, std::min<uint64_t>(((span + kSieveTile - 1) / kSieveTile) * kSieveTile, cap));
    }
    if (block_len > (1ull << 31)) {
        set_last_error("mertens_plan: block_len must be <= 2^31");
        delete p;
        return MERTENS_EINVAL;
    }
    p->block_len = block_len;
    p->nblocks = (span + block_len - 1) / block_len;
    if (window) {
        // only the window's part of the dense list, and divisor magics for
        // the j whose quotient can reach the window
        p->ydense = p->y_first <= p->ydense ? std::min(p->ydense, p->y_last) : 0;
        p->jmax = 0;
        for (size_t e = 0; e < K.size(); ++e)
            if (K[e])
                p->jmax = std::max(p->jmax, std::min(JC0[e], K[e] / p->y_first));
    }
    p->mg_n = std::max(p->jmax, p->ydense) + 1;
    // quotients of the shared-memory gather: the float estimate, with a
    // 32-bit remainder while every gathered j is below 2^31 (MERTENS_GATHER_QUOT
    // = 0 forces the multiply-high magics, = 2 the 64-bit remainder)
    p->gquot = p->jmax < (1ull << 31) ? 1u : 2u;
    if (const char *e = getenv("MERTENS_GATHER_QUOT")) {
        if (e[0] == '0')
            p->gquot = 0;
        else if (e[0] == '2')
            p->gquot = 2;
    }
    if (table && (p->ydense > table->ydense || p->mg_n > table->mg_n)) {
        set_last_error("mertens_plan_on_table: the targets need dense cut-offs or divisors "
                       "beyond the table");
        delete p;
        return MERTENS_ENOTSUP;
    }

    // ---- dense work items: groups sorted by cut-off, chunk ranges ----
    std::vector<uint32_t> order(groups.size());
    for (size_t i = 0; i < order.size(); ++i)
        order[i] = (uint32_t)i;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return groups[a].yc > groups[b].yc; });
    std::vector<Group> sg(groups.size());
    for (size_t i = 0; i < order.size(); ++i)
        sg[i] = groups[order[i]];
    const uint64_t nchunks = p->ydense / kChunk + 1;
    std::vector<DenseItem> items;
    const uint32_t gpi = (kDenseThreads / 32) * 4;
    size_t pref = sg.size();
    for (uint64_t c0 = 0; c0 < nchunks; c0 += kDenseChunks) {
        const uint64_t ys = c0 * kChunk;
        while (pref > 0 && sg[pref - 1].yc < ys)
            --pref;
        if (pref == 0)
            break;
        for (size_t g0 = 0; g0 < pref; g0 += gpi) {
            DenseItem it;
            it.c0 = (uint32_t)c0;
            it.c1 = (uint32_t)std::min<uint64_t>(c0 + kDenseChunks, nchunks);
            it.g0 = (uint32_t)g0;
            it.g1 = (uint32_t)std::min<size_t>(g0 + gpi, pref);
            items.push_back(it);
        }
    }
    p->nitems = (uint32_t)items.size();

    // ---- shared-memory gather tiles: y in [block start, min(block end, Y_s)]
    // of each block, items of up to 1024 entries of one target whose dense
    // cut-off is below the tile end (a suffix of the target's entries, found
    // on the running minimum of the cut-offs) ----
    std::vector<uint64_t> ycmin(YCE.size());
    std::vector<double> kpre(YCE.size() + 1, 0.0);  // prefix sums of k over all entries
    for (size_t e = 0; e < K.size(); ++e)
        kpre[e + 1] = kpre[e] + (double)K[e];
    for (size_t i = 0; i < count; ++i) {
        uint64_t run = UINT64_MAX;
        for (uint64_t x = 0; x < p->X[i]; ++x) {
            const size_t e = p->off[i] + x;
            if (K[e] != 0)  // two-word entries have no terms here
                run = std::min(run, YCE[e]);
            ycmin[e] = run;
        }
    }
    const double kItemWork = 2.0e5;
    {
        // Gathered terms per y near y are about (n / y^2) ln X summed over
        // the targets; shared-memory tiles pay while that is at least ~2,
        // i.e. up to y ~ sqrt(sum n ln X / 2) (2.5e8 for n = 1e16, X = 2.5e5).
        // A tile pays while its terms (32768 (sum n ln X) / y^2) are at least
        // a quarter of the entries it must check (all of them, E).
        double acc = 0;
        for (size_t i = 0; i < count; ++i)
            acc += ((double)p->n[i] + 18446744073709551616.0 * (double)p->n_hi[i]) *
                   std::log((double)std::max<uint64_t>(p->X[i], 2));
        const double E = (double)std::max<uint64_t>(p->nent, 1);
        const double gs = tn.gather_scale > 0 ? tn.gather_scale : 1.0;
        uint64_t ys = (uint64_t)(gs * std::min(std::sqrt(acc / 2.0),
                                               std::sqrt(4.0 * kGatherTile * acc / E)));
        const char *e = getenv("MERTENS_GATHER_END");
        if (e)
            ys = strtoull(e, nullptr, 10);
        p->gather_smem_end = std::min(ys, p->y_max);
    }
    std::vector<GatherTile> gtiles;
    std::vector<GatherItem> gitems;
    // Blocks above the tile range: tiles over the whole block for the
    // entries with k >= kt_fac y1^2 / kGatherTile (about kt_fac terms or more
    // per tile; a prefix of each target's entries), when they have at least
    // kt_min terms per tile together; the global path takes the others.
    double kt_fac = 1.0, kt_min = 700.0;
    if (const char *e = getenv("MERTENS_TILE_KT"))
        kt_fac = atof(e);
    if (const char *e = getenv("MERTENS_TILE_MIN"))
        kt_min = atof(e);
    for (uint64_t b = 0; b < p->nblocks; ++b) {
        uint64_t y1, y2;
        block_range(p, b, &y1, &y2);
        p->gblk.push_back((uint32_t)gitems.size());
        uint64_t end = std::min(y2, p->gather_smem_end);
        p->gend.push_back(y1 <= end ? end : y1 - 1);
        uint64_t kt = UINT64_MAX;  // entries with k >= kt take this block's tiles
        if (y1 > p->gather_smem_end && kt_fac > 0) {
            const double k0 = kt_fac * (double)y1 * (double)y1 / kGatherTile;
            double ksum = 0;
            for (size_t i = 0; i < count; ++i) {
                const uint64_t o = p->off[i], X = p->X[i];
                const double xt = std::min((double)X,
                                           std::floor(((double)p->n[i] +
                                                       18446744073709551616.0 *
                                                           (double)p->n_hi[i]) / k0));
                ksum += kpre[o + (uint64_t)xt] - kpre[o];
            }
            if (ksum * kGatherTile / ((double)y1 * (double)y1) >= kt_min) {
                kt = (uint64_t)std::ceil(k0);
                end = y2;
            }
        }
        p->ktile.push_back(kt);
        // the block's tiles on host threads, then appended in order (a tile
        // is kept when some entry range can have terms in it)
        const uint64_t ntile = y1 <= end ? (end - y1) / kGatherTile + 1 : 0;
        std::vector<GatherTile> btiles(ntile);
        std::vector<std::vector<GatherItem>> bitems(ntile);
        parallel_for(ntile, 64, [&](size_t qlo, size_t qhi) {
            std::vector<std::pair<uint64_t, uint64_t>> ranges;
            for (size_t q = qlo; q < qhi; ++q) {
                const uint64_t t1 = y1 + q * kGatherTile;
                const uint64_t t2 = std::min(t1 + kGatherTile - 1, end);
                GatherTile &T = btiles[q];
                T.t1 = t1;
                T.len = (uint32_t)(t2 - t1 + 1);
                T.m1 = magic_of(t1);
                T.l1 = magic_shift(t1);
                T.m2 = magic_of(t2 + 1);
                T.l2 = magic_shift(t2 + 1);
                T.pad = 0;
                // entries that can have terms here: per target the suffix
                // whose cut-off lies below t2 (found on the running minimum);
                // suffixes of consecutive targets separated by short gaps are
                // merged (an entry outside its suffix simply has no terms in
                // the tile)
                ranges.clear();
                for (size_t i = 0; i < count; ++i) {
                    const uint64_t o = p->off[i], X = p->X[i];
                    uint64_t lo = 0, hi = X;  // first x index with ycmin < t2
                    while (lo < hi) {
                        const uint64_t mid = (lo + hi) / 2;
                        if (ycmin[o + mid] < t2)
                            hi = mid;
                        else
                            lo = mid + 1;
                    }
                    // above the tile range only the prefix with k >= kt
                    uint64_t top = X;
                    if (kt != UINT64_MAX) {
                        uint64_t a = 0, z = X;  // first x index with k < kt
                        while (a < z) {
                            const uint64_t mid = (a + z) / 2;
                            if (K[o + mid] >= kt || K[o + mid] == 0)
                                a = mid + 1;
                            else
                                z = mid;
                        }
                        top = a;
                    }
                    if (lo >= top)
                        continue;
                    if (!ranges.empty() && o + lo <= ranges.back().second + 4096 &&
                        kt == UINT64_MAX)
                        ranges.back().second = o + top;
                    else
                        ranges.push_back({o + lo, o + top});
                }
                // work of entries [f, g): about one range check each plus
                // sum k * len / t1^2 gathered terms; items of ~kItemWork
                const double per_k = (double)T.len / ((double)t1 * (double)t1);
                for (const auto &rg : ranges) {
                    for (uint64_t f = rg.first; f < rg.second;) {
                        uint64_t g = std::min<uint64_t>(f + 1024, rg.second);
                        while (g < rg.second) {
                            const double work =
                                (double)(g - f) + per_k * (kpre[g] - kpre[f]);
                            if (work >= kItemWork)
                                break;
                            g = std::min<uint64_t>(g + 1024, rg.second);
                        }
                        GatherItem it;
                        it.tile = 0;  // set when the tile is appended
                        it.e0 = (uint32_t)f;
                        it.e1 = (uint32_t)g;
                        it.pad = 0;
                        bitems[q].push_back(it);
                        f = g;
                    }
                }
            }
        });
        for (size_t q = 0; q < ntile; ++q) {
            if (bitems[q].empty())
                continue;
            const uint32_t ti = (uint32_t)gtiles.size();
            gtiles.push_back(btiles[q]);
            for (GatherItem it : bitems[q]) {
                it.tile = ti;
                gitems.push_back(it);
            }
        }
    }
    p->gblk.push_back((uint32_t)gitems.size());
    // ---- two-word entries: grid width per block ----
    if (!p->wide.empty()) {
        p->wide_grid.assign(p->nblocks, 0);
        for (uint64_t b = 0; b < p->nblocks; ++b) {
            uint64_t y1, y2;
            block_range(p, b, &y1, &y2);
            uint64_t most = 0;
            for (const WideEntry &W : p->wide) {
                uint64_t nd, ja, ng;
                wide_ranges(W, y1, y2, &nd, &ja, &ng);
                most = std::max(most, nd + ng);
            }
            p->wide_grid[b] = (uint32_t)((most + kWideUnitsPerCta - 1) / kWideUnitsPerCta);
        }
    }

    // ---- window plans: coefficient of the carry M(y_first - 1) per entry ----
    // gathered terms: one per j with floor(k/j) in the window; the dense
    // form's boundary term -M(yc) floor(k/(yc+1)) when yc is in it; direct
    // terms of two-word entries: sum of floor(k/y) - floor(k/(y+1)) over the
    // window's y <= s, which telescopes.
    if (window) {
        const uint64_t a = p->y_first, z = p->y_last;
        p->coef.assign(K.size(), 0);
        if (z >= a) {
            for (size_t e = 0; e < K.size(); ++e) {
                const uint64_t k = K[e];
                if (k == 0)
                    continue;
                const uint64_t jb = std::max(JLO[e], k / (z + 1) + 1);
                const uint64_t jt = std::min(JC0[e], k / a);
                uint64_t c = jt >= jb ? jt - jb + 1 : 0;
                if (YCE[e] >= a && YCE[e] <= z)
                    c -= JC0[e];
                p->coef[e] = c;
            }
            for (const WideEntry &W : p->wide) {
                const u128 k = ((u128)W.k_hi << 64) | W.k_lo;
                uint64_t c = 0;
                const uint64_t dl = std::min(z, W.s);
                if (a <= dl)
                    c += (uint64_t)(k / a) - (uint64_t)(k / ((u128)dl + 1));
                uint64_t nd, ja, ng;
                wide_ranges(W, a, z, &nd, &ja, &ng);
                c += ng;
                p->coef[W.e] = c;
            }
        }
    }

    // ---- device buffers ----
    int rc = MERTENS_OK;
    const size_t E = p->nent;
    p->dK = p->alloc<uint64_t>(E);
    p->dJLO = p->alloc<uint64_t>(E);
    p->dEMIT = p->alloc<uint32_t>(E);
    p->dJC0 = p->alloc<uint64_t>(E);
    p->dJCUR = p->alloc<uint64_t>(E);
    p->dYCE = p->alloc<uint64_t>(E);
    p->dS = p->alloc<uint64_t>(E);
    p->dR = p->alloc<uint64_t>(E);
    {
        // chunk records of a block's global gather: an entry with cnt terms
        // there posts ceil(cnt / kSparseItem) of them when cnt > 48; cnt is
        // at most k (1/y_lo - 1/(y2+1)) + 1, so a block posts at most
        // C/kSparseItem + min(E, C/48) with C = (sum k)(1/y_lo - 1/(y2+1)) + E
        double most = 0;
        for (uint64_t b = 0; b < p->nblocks; ++b) {
            uint64_t y1, y2;
            block_range(p, b, &y1, &y2);
            const uint64_t ylo = std::max(p->gend[b] + 1, y1);
            if (ylo > y2)
                continue;
            const double C = kpre[K.size()] * (1.0 / (double)ylo - 1.0 / ((double)y2 + 1.0)) +
                             (double)E;
            most = std::max(most, C / kSparseItem + std::min((double)E, C / 48.0));
        }
        p->qcap = (uint32_t)std::min(most * 1.01 + 256.0, 4.0e9);
        p->dqueue = p->alloc<uint4>(p->qcap);
        p->dqlen = p->alloc<uint32_t>(1);
    }
    const uint64_t L = block_len;
    const uint64_t nseg = sieve_segments(L);
    // One stream by default: on GB300 the three-stream schedule measured
    // slower (the sieve and the updates contend for the same SM resources);
    // MERTENS_OVERLAP=1 selects it.  Plans on a table have no sieve.
    p->serial = getenv("MERTENS_OVERLAP") == nullptr || p->nblocks == 1 || table;
    // a plan on a table sieves only the blocks that end above the table
    p->sieves = !table || p->y_last > table->y_max;
    if (table) {
        // the table's M(y) blocks are addressed per block at run time
        p->dmu_aux = nullptr;
        p->dMG = table->MG;
        p->ddl_m = table->dl_m;
        p->ddl_yo = table->dl_yo;
        p->ddl_cnt = table->dl_cnt;
        p->mg_built = true;
        if (!p->lookups.empty())
            p->dlook = p->alloc<uint64_t>(p->lookups.size());
    }
    if (p->sieves) {
        if (!table)
            p->dmu_aux = p->alloc<int8_t>(p->ydense + 16);
        const int nbuf = p->serial ? 1 : 2;
        for (int i = 0; i < 2; ++i) {
            if (i < nbuf) {
                p->dMloc[i] = p->alloc<int16_t>(L + 16);  // tiles copy whole 16-byte units
                p->dsegsum[i] = p->alloc<int32_t>(nseg);
                p->dsegoff[i] = p->alloc<int64_t>(nseg);
            } else {
                p->dMloc[i] = p->dMloc[0];
                p->dsegsum[i] = p->dsegsum[0];
                p->dsegoff[i] = p->dsegoff[0];
            }
        }
        if (!table) {
            p->dMG = p->alloc<uint64_t>(p->mg_n + 1);
            p->ddl_m = p->alloc<uint64_t>(nchunks * kChunkCapPad);
            p->ddl_yo = p->alloc<uint16_t>(nchunks * kChunkCapPad);
            p->ddl_cnt = p->alloc<uint2>(nchunks);
        }
    }
    p->dcarry = p->alloc<int64_t>(p->nblocks + 1);
    p->dgtiles = p->alloc<GatherTile>(gtiles.size() + 1);
    p->dgitems = p->alloc<GatherItem>(gitems.size() + 1);

    p->derr = p->alloc<uint32_t>(1);
    p->dcounter = p->alloc<uint32_t>(1);
    p->dcounter_dense = p->alloc<uint32_t>(1);
    p->dcounter_gather = p->alloc<uint32_t>(1);
    p->dgroups = p->alloc<Group>(sg.size());
    p->ditems = p->alloc<DenseItem>(items.size());
    p->dqs = p->alloc<QueryDev>(count);
    if (!p->wide.empty())
        p->dwide = p->alloc<WideEntry>(p->wide.size());
    if (window)
        p->dcoef = p->alloc<uint64_t>(E);
    for (auto &a : p->allocs)
        if (!a.first)
            rc = MERTENS_ENOMEM;
    bool any_null = !p->dK || !p->dJLO || !p->dEMIT || !p->dJC0 || !p->dJCUR || !p->dYCE || !p->dqueue ||
                    !p->dqlen || !p->dS || !p->dR ||
                    (!table && !p->dmu_aux) ||
                    (p->sieves && (!p->dMloc[0] || !p->dsegsum[0] || !p->dsegoff[0] ||
                                   !p->dMloc[1] || !p->dsegsum[1] || !p->dsegoff[1])) ||
                    (!p->lookups.empty() && !p->dlook) || !p->dgtiles ||
                    !p->dcounter_dense || !p->dcounter_gather ||
                    !p->dgitems || !p->dcarry || !p->derr || !p->dcounter || !p->dMG ||
                    !p->ddl_m || !p->ddl_yo || !p->ddl_cnt || !p->dgroups || !p->ditems ||
                    !p->dqs || (!p->wide.empty() && !p->dwide) || (window && !p->dcoef);
    if (any_null)
        rc = MERTENS_ENOMEM;
    if (rc == MERTENS_OK && p->sieves) {
        int prc = prime_table_create(&p->pt, p->al, std::max<uint64_t>(p->y_last, 1), nullptr);
        if (prc == 0)
            prc = sieve_scratch_create(&p->pt, block_len);
        if (prc != 0)
            rc = prc == 6 ? MERTENS_ENOTSUP : (prc == 2 ? MERTENS_ENOMEM : MERTENS_ECUDA);
    }
    if (rc == MERTENS_OK && p->sieves) {
        // algorithmic sieve updates: each block of length len sieved with the
        // primes p <= max(7, sqrt(block end)) costs len * sum (1/p + 1/p^2)
        std::vector<double> pre(p->pt.np + 1, 0.0);
        for (uint32_t i = 0; i < p->pt.np; ++i) {
            const double q = (double)p->pt.host_p[i];
            pre[i + 1] = pre[i] + 1.0 / q + 1.0 / (q * q);
        }
        for (uint64_t b = 0; b < p->nblocks; ++b) {
            uint64_t y1, y2;
            block_range(p, b, &y1, &y2);
            if (table && y2 <= table->y_max)
                continue;  // read from the table
            const uint64_t P = std::max<uint64_t>(7, isqrt64(y2));
            p->sieve_updates += (double)(y2 - y1 + 1) * pre[prime_count_upto(&p->pt, P)];
        }
    }
    if (rc == MERTENS_OK) {
        std::vector<QueryDev> qs(count);
        for (size_t i = 0; i < count; ++i) {
            qs[i].X = p->X[i];
            qs[i].off = p->off[i];
        }
        cudaMemcpy(p->dK, K.data(), E * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(p->dJLO, JOWN.data(), E * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(p->dEMIT, EMIT.data(), E * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(p->dJC0, JC0.data(), E * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(p->dYCE, YCE.data(), E * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(p->dgroups, sg.data(), sg.size() * sizeof(Group), cudaMemcpyHostToDevice);
        if (!items.empty())
            cudaMemcpy(p->ditems, items.data(), items.size() * sizeof(DenseItem),
                       cudaMemcpyHostToDevice);
        cudaMemcpy(p->dqs, qs.data(), count * sizeof(QueryDev), cudaMemcpyHostToDevice);
        if (!p->wide.empty())
            cudaMemcpy(p->dwide, p->wide.data(), p->wide.size() * sizeof(WideEntry),
                       cudaMemcpyHostToDevice);
        if (!p->lookups.empty())
            cudaMemcpy(p->dlook, p->lookups.data(), p->lookups.size() * 8,
                       cudaMemcpyHostToDevice);
        if (window)
            cudaMemcpy(p->dcoef, p->coef.data(), E * 8, cudaMemcpyHostToDevice);
        if (!gtiles.empty())
            cudaMemcpy(p->dgtiles, gtiles.data(), gtiles.size() * sizeof(GatherTile),
                       cudaMemcpyHostToDevice);
        if (!gitems.empty())
            cudaMemcpy(p->dgitems, gitems.data(), gitems.size() * sizeof(GatherItem),
                       cudaMemcpyHostToDevice);
        p->h2d_bytes = 4 * E * 8 + E * 4 + sg.size() * sizeof(Group) + items.size() * sizeof(DenseItem) +
                       count * sizeof(QueryDev) + gtiles.size() * sizeof(GatherTile) +
                       gitems.size() * sizeof(GatherItem) + p->wide.size() * sizeof(WideEntry);
        if (cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess)
            rc = MERTENS_ECUDA;
        if (rc == MERTENS_OK && !p->serial) {
            const unsigned fl = cudaEventDisableTiming;
            bool ok = cudaStreamCreateWithFlags(&p->st_sieve, cudaStreamNonBlocking) == cudaSuccess &&
                      cudaStreamCreateWithFlags(&p->st_upd, cudaStreamNonBlocking) == cudaSuccess &&
                      cudaStreamCreateWithFlags(&p->st_dense, cudaStreamNonBlocking) == cudaSuccess &&
                      cudaEventCreateWithFlags(&p->ev_fork, fl) == cudaSuccess &&
                      cudaEventCreateWithFlags(&p->ev_reset, fl) == cudaSuccess &&
                      cudaEventCreateWithFlags(&p->ev_dense_done, fl) == cudaSuccess &&
                      cudaEventCreateWithFlags(&p->ev_sieve_done, fl) == cudaSuccess &&
                      cudaEventCreateWithFlags(&p->ev_join, fl) == cudaSuccess;
            p->ev_sieved.assign(p->nblocks, nullptr);
            p->ev_upd.assign(p->nblocks, nullptr);
            for (uint64_t b = 0; ok && b < p->nblocks; ++b)
                ok = cudaEventCreateWithFlags(&p->ev_sieved[b], fl) == cudaSuccess &&
                     cudaEventCreateWithFlags(&p->ev_upd[b], fl) == cudaSuccess;
            if (!ok)
                rc = MERTENS_ECUDA;
        }
    }
    if (rc != MERTENS_OK) {
        if (rc == MERTENS_ENOMEM)
            set_last_error("mertens_plan: device allocation failed");
        else if (rc == MERTENS_ECUDA)
            set_last_error("mertens_plan: CUDA error %s", cudaGetErrorString(cudaGetLastError()));
        mertens_destroy(p);
        return rc;
    }
    *out = p;
    return MERTENS_OK;
}

int mertens_plan(mertens_plan_t *out, const mertens_u128 *n, size_t count, mertens_u128 u,
                 uint64_t block_len)
{
    return plan_create(out, n, count, u, block_len, tuning_now());
}

}  // extern "C"

namespace mert {
// A plan with an explicit tuning (the autotuner's candidates).
int plan_create_tuned(mertens_plan_t *out, const mertens_u128 *n, size_t count,
                      const mertens_tuning &t)
{
    mertens_u128 u0 = {0, 0};
    return plan_create(out, n, count, u0, 0, t);
}
}  // namespace mert

extern "C" {

int mertens_set_tuning(const mertens_tuning *t)
{
    if (!t || !(t->u_factor > 0.0 && t->u_factor < 100.0) ||
        !(t->dense_c > 0.0 && t->dense_c < 1000.0) ||
        !(t->gather_scale > 0.0 && t->gather_scale < 1000.0) ||
        (t->block_cap != 0 && (t->block_cap < (uint64_t)kSieveTile || t->block_cap > (1ull << 31)))) {
        set_last_error("mertens_set_tuning: factors must be positive and finite, block_cap 0 or "
                       "in [2^16, 2^31]");
        return MERTENS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuning = *t;
    return MERTENS_OK;
}

int mertens_get_tuning(mertens_tuning *t)
{
    if (!t)
        return MERTENS_EINVAL;
    *t = tuning_now();
    return MERTENS_OK;
}

static void ev_begin(mertens_plan_s *p, int phase, cudaStream_t s, PhaseEvents *pe)
{
    if (!p->prof)
        return;
    pe->phase = phase;
    cudaEventCreate(&pe->a);
    cudaEventCreate(&pe->b);
    cudaEventRecord(pe->a, s);
}

static void ev_end(mertens_plan_s *p, cudaStream_t s, PhaseEvents *pe)
{
    if (!p->prof)
        return;
    cudaEventRecord(pe->b, s);
    p->evs.push_back(*pe);
}

static void clear_events(mertens_plan_s *p)
{
    for (auto &e : p->evs) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    p->evs.clear();
    p->prof_runs = 0;
}

// Enqueues one whole run (all blocks, then resolve) forked from stream
// `origin` onto three streams and joined back: the sieve chain (block by
// block, two output buffers), the per-block gathered updates (each after its
// block's sieve; the sieve of block b+2 waits for them, as it reuses the
// buffer), and the dense update (after the block that completes the
// squarefree list).  S only receives commutative atomic additions, so the
// dense and gathered updates may interleave.  *out = kernels launched.
static int run_enqueue(mertens_plan_s *p, cudaStream_t origin, uint64_t *out)
{
    uint64_t launches = 0;
    int r;
    const size_t E = p->nent;
    const bool serial = p->serial;
    cudaStream_t ss = serial ? origin : p->st_sieve;
    cudaStream_t su = serial ? origin : p->st_upd;
    cudaStream_t sd = serial ? origin : p->st_dense;
    if (!serial) {
        cudaEventRecord(p->ev_fork, origin);
        cudaStreamWaitEvent(ss, p->ev_fork, 0);
        cudaStreamWaitEvent(su, p->ev_fork, 0);
        cudaStreamWaitEvent(sd, p->ev_fork, 0);
    }
    cudaMemsetAsync(p->dS, 0, E * 8, su);
    cudaMemcpyAsync(p->dJCUR, p->dJC0, E * 8, cudaMemcpyDeviceToDevice, su);
    const mertens_table_s *tab = p->table;
    cudaMemsetAsync(p->dcarry, 0, 8 * (p->nblocks + 1), ss);
    cudaMemsetAsync(p->derr, 0, 4, su);
    if (p->window && p->y_first <= p->ydense && !tab)
        cudaMemsetAsync(p->dmu_aux, 0, p->ydense + 1, ss);  // mu outside the window: none
    if (!p->mg_built) {
        r = magic_table_enqueue(p->dMG, p->mg_n, su);
        if (r < 0)
            goto fail;
        launches += r;
        p->mg_built = true;
    }
    if (!serial) {
        // the dense update needs S cleared and the divisor magics
        cudaEventRecord(p->ev_reset, su);
        cudaStreamWaitEvent(sd, p->ev_reset, 0);
    }
    {
        // the dense part runs once mu is known up to Y_dense (or up to the
        // window's end); a window above Y_dense has none
        bool dense_done = p->y_first > p->ydense;
        const uint64_t dense_at = std::min(p->ydense, p->y_last);
        if (tab && !dense_done) {
            // the squarefree list is the table's: the dense part needs no block
            PhaseEvents pe;
            ev_begin(p, kPhDense, su, &pe);
            DenseArgs da;
            da.items = p->ditems;
            da.nitems = p->nitems;
            da.counter = p->dcounter_dense;
            da.groups = p->dgroups;
            da.K = p->dK;
            da.YCE = p->dYCE;
            da.dl_m = p->ddl_m;
            da.dl_yo = p->ddl_yo;
            da.dl_cnt = p->ddl_cnt;
            da.S = p->dS;
            da.ctas_per_sm = 0;
            r = dense_update_enqueue(da, su);
            ev_end(p, su, &pe);
            if (r < 0)
                goto fail;
            launches += r;
            dense_done = true;
        }
        for (uint64_t b = 0; b < p->nblocks; ++b) {
            uint64_t y1, y2;
            block_range(p, b, &y1, &y2);
            const int buf = (int)(b & 1);
            // M(y) of the block: the table's where it covers the whole block,
            // else the plan's buffer (sieved below)
            const bool from_table = tab && y2 <= tab->y_max;
            const int16_t *Mb = from_table ? tab->Mloc + (y1 - 1) : p->dMloc[buf];
            const int64_t *Sb =
                from_table ? tab->segoff + ((y1 - 1) >> kSegShift) : p->dsegoff[buf];
            if (!serial && b >= 2)
                cudaStreamWaitEvent(ss, p->ev_upd[b - 2], 0);
            cudaStream_t s = ss;
            if (tab && !from_table && y1 > 1 && y1 - 1 <= tab->y_max) {
                // the first sieved block above the table: its carry M(y1 - 1)
                // is the table's
                r = carry_from_table_enqueue(tab->Mloc, tab->segoff, y1 - 1, p->dcarry + b, ss);
                if (r < 0)
                    goto fail;
                launches += r;
            }
            if (!from_table) {
                SieveLaunch L;
                L.y1 = y1;
                L.len = y2 - y1 + 1;
                L.Mloc = p->dMloc[buf];
                L.segsum = p->dsegsum[buf];
                L.segoff = p->dsegoff[buf];
                L.carry_in = p->dcarry + b;
                L.carry_out = p->dcarry + b + 1;
                L.mu_out = (y1 <= p->ydense) ? p->dmu_aux : nullptr;
                L.mu_base = 1;
                L.mu_end = p->ydense;
                PhaseEvents pe, pe2;
                ev_begin(p, kPhSieve, s, &pe);
                if (p->prof) {
                    pe2.phase = kPhScan;
                    cudaEventCreate(&pe2.a);
                    cudaEventCreate(&pe2.b);
                    L.mid = pe.b;
                    L.mid2 = pe2.a;
                }
                r = sieve_block_enqueue(&p->pt, L, s);
                if (p->prof) {
                    p->evs.push_back(pe);
                    cudaEventRecord(pe2.b, s);
                    p->evs.push_back(pe2);
                }
                if (r < 0)
                    goto fail;
                launches += r;
                if (!serial)
                    cudaEventRecord(p->ev_sieved[b], ss);
                if (!dense_done && y2 >= dense_at) {
                    s = sd;
                    if (!serial)
                        cudaStreamWaitEvent(sd, p->ev_sieved[b], 0);
                    ev_begin(p, kPhDense, s, &pe);
                    r = dense_list_enqueue(p->dmu_aux, p->ydense, p->dMG, p->ddl_m, p->ddl_yo,
                                           p->ddl_cnt, s);
                    if (r < 0)
                        goto fail;
                    launches += r;
                    DenseArgs da;
                    da.items = p->ditems;
                    da.nitems = p->nitems;
                    da.counter = p->dcounter_dense;
                    da.groups = p->dgroups;
                    da.K = p->dK;
                    da.YCE = p->dYCE;
                    da.dl_m = p->ddl_m;
                    da.dl_yo = p->ddl_yo;
                    da.dl_cnt = p->ddl_cnt;
                    da.S = p->dS;
                    da.ctas_per_sm = serial ? 0 : 1;
                    r = dense_update_enqueue(da, s);
                    ev_end(p, s, &pe);
                    if (r < 0)
                        goto fail;
                    launches += r;
                    dense_done = true;
                }
            }  // sieve of the block
            PhaseEvents pe;
            s = su;
            if (!serial)
                cudaStreamWaitEvent(su, p->ev_sieved[b], 0);
            SparseBlockArgs sb;
            sb.y1 = y1;
            sb.y2 = y2;
            sb.m_y1 = magic_of(y1);
            sb.l_y1 = magic_shift(y1);
            sb.m_y2p1 = magic_of(y2 + 1);
            sb.l_y2p1 = magic_shift(y2 + 1);
            SparseArgs sa;
            sa.nent = E;
            sa.K = p->dK;
            sa.JLO = p->dJLO;
            sa.EMIT = p->dEMIT;
            sa.JC0 = p->dJC0;
            sa.YCE = p->dYCE;
            sa.MG = p->dMG;
            sa.S = p->dS;
            sa.queue = p->dqueue;
            sa.qlen = p->dqlen;
            sa.qcap = p->qcap;
            sa.err = p->derr;
            sa.Mloc = Mb;
            sa.segoff = Sb;
            sa.y_lo = p->gend[b] + 1 > y1 ? p->gend[b] + 1 : y1;
            sa.kmax = p->ktile[b];
            sa.m_ylo = magic_of(sa.y_lo);
            sa.l_ylo = magic_shift(sa.y_lo);
            if (p->gblk[b + 1] > p->gblk[b]) {
                GatherArgs ga;
                ga.y1 = y1;
                ga.tiles = p->dgtiles;
                ga.items = p->dgitems + p->gblk[b];
                ga.nitems = p->gblk[b + 1] - p->gblk[b];
                ga.counter = p->dcounter_gather;
                ga.Mloc = Mb;
                ga.segoff = Sb;
                ga.err = p->derr;
                ga.threads = serial ? 512 : 256;
                ga.ctas_per_sm = serial ? 0 : 2;
                ga.quot = p->gquot;
                ga.K = p->dK;
                ga.JLO = p->dJLO;
                ga.EMIT = p->dEMIT;
                ga.JCUR = p->dJCUR;
                ga.MG = p->dMG;
                ga.S = p->dS;
                ev_begin(p, kPhGather, s, &pe);
                r = gather_tiles_enqueue(ga, s);
                ev_end(p, s, &pe);
                if (r < 0)
                    goto fail;
                launches += r;
            }
            ev_begin(p, kPhGather, s, &pe);
            r = sparse_block_enqueue(sb, sa, s);
            ev_end(p, s, &pe);
            if (r < 0)
                goto fail;
            launches += r;
            if (!p->wide.empty() && p->wide_grid[b]) {
                WideArgs wa;
                wa.W = p->dwide;
                wa.y1 = y1;
                wa.y2 = y2;
                wa.Mloc = Mb;
                wa.segoff = Sb;
                wa.S = p->dS;
                ev_begin(p, kPhGather, s, &pe);
                r = wide_update_enqueue(wa, (uint32_t)p->wide.size(), p->wide_grid[b], s);
                ev_end(p, s, &pe);
                if (r < 0)
                    goto fail;
                launches += r;
            }
            if (!serial)
                cudaEventRecord(p->ev_upd[b], su);
        }
        if (!serial) {
            // resolve after every update; join all streams back to origin
            cudaEventRecord(p->ev_dense_done, sd);
            cudaStreamWaitEvent(su, p->ev_dense_done, 0);
            cudaEventRecord(p->ev_sieve_done, ss);
            cudaStreamWaitEvent(su, p->ev_sieve_done, 0);
        }
        if (!p->window) {
            PhaseEvents pe;
            ev_begin(p, kPhResolve, su, &pe);
            r = resolve_enqueue(p->dqs, (uint32_t)p->nq, p->dS, p->dK, p->dR, su);
            if (r >= 0 && !p->lookups.empty()) {
                const int r2 = table_lookup_enqueue(p->dlook, (uint32_t)(p->lookups.size() / 2),
                                                    tab->Mloc, tab->segoff, p->dR, su);
                r = r2 < 0 ? r2 : r + r2;
            }
            ev_end(p, su, &pe);
            if (r < 0)
                goto fail;
            launches += r;
        }
        if (!serial) {
            cudaEventRecord(p->ev_join, su);
            cudaStreamWaitEvent(origin, p->ev_join, 0);
        }
    }
    *out = launches;
    return MERTENS_OK;
fail:
    set_last_error("mertens_run: launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return MERTENS_ECUDA;
}

// Whole runs after the first are replayed from a CUDA graph captured on the
// plan's own stream (kernel arguments of a plan never change between runs),
// unless profiling is on or MERTENS_NO_GRAPH is set.
int mertens_run(mertens_plan_t p, void *stream)
{
    if (!p) {
        set_last_error("mertens_run: NULL plan");
        return MERTENS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t launches = 0;
    const bool graph_ok = !p->prof && p->ran && !getenv("MERTENS_NO_GRAPH");
    if (!graph_ok) {
        PhaseEvents total;
        ev_begin(p, kPhTotal, s, &total);
        const int rc = run_enqueue(p, s, &launches);
        if (rc != MERTENS_OK)
            return rc;
        ev_end(p, s, &total);
        if (p->prof)
            ++p->prof_runs;
    } else {
        if (!p->gexec) {
            if (!p->cap_stream &&
                cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
                set_last_error("mertens_run: cannot create the capture stream");
                return MERTENS_ECUDA;
            }
            if (cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal) !=
                cudaSuccess) {
                set_last_error("mertens_run: cannot begin capture: %s",
                               cudaGetErrorString(cudaGetLastError()));
                return MERTENS_ECUDA;
            }
            const int rc = run_enqueue(p, p->cap_stream, &launches);
            cudaGraph_t g = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &g);
            if (rc != MERTENS_OK || ce != cudaSuccess || !g) {
                if (g)
                    cudaGraphDestroy(g);
                set_last_error("mertens_run: capture failed: %s", cudaGetErrorString(ce));
                return MERTENS_ECUDA;
            }
            const cudaError_t ie = cudaGraphInstantiate(&p->gexec, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) {
                p->gexec = nullptr;
                set_last_error("mertens_run: graph instantiation failed: %s",
                               cudaGetErrorString(ie));
                return MERTENS_ECUDA;
            }
            p->graph_kernels = launches;
        }
        if (cudaGraphLaunch(p->gexec, s) != cudaSuccess) {
            set_last_error("mertens_run: graph launch failed: %s",
                           cudaGetErrorString(cudaGetLastError()));
            return MERTENS_ECUDA;
        }
        launches = p->graph_kernels;
    }
    if (cudaEventRecord(p->done, s) != cudaSuccess) {
        set_last_error("mertens_run: %s", cudaGetErrorString(cudaGetLastError()));
        return MERTENS_ECUDA;
    }
    p->kernels = launches;
    p->d2h_bytes = 0;
    p->ran = true;
    return MERTENS_OK;
}

int mertens_result(mertens_plan_t p, size_t i, int64_t *M_n, int64_t *entries, size_t cap,
                   size_t *len)
{
    if (!p || i >= p->nq) {
        set_last_error("mertens_result: bad plan or index");
        return MERTENS_EINVAL;
    }
    if (!p->ran) {
        set_last_error("mertens_result: mertens_run was not called");
        return MERTENS_ENOTREADY;
    }
    if (cudaEventSynchronize(p->done) != cudaSuccess) {
        set_last_error("mertens_result: %s", cudaGetErrorString(cudaGetLastError()));
        return MERTENS_ECUDA;
    }
    if (p->window) {
        set_last_error("mertens_result: a window plan has partial sums only "
                       "(mertens_window_result)");
        return MERTENS_EINVAL;
    }
    uint32_t err = 0;
    if (cudaMemcpy(&err, p->derr, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return MERTENS_ECUDA;
    if (p->sieves) {
        const uint32_t st = sieve_scratch_status(&p->pt);
        if (st) {
            set_last_error("mertens_result: %s", sieve_status_text(st));
            return sieve_status_code(st);
        }
    }
    if (err & kErrTimeout) {
        set_last_error("mertens_result: a bounded wait for a bulk copy in the update gave up");
        return MERTENS_ETIMEOUT;
    }
    if (err & kErrMOverflow) {
        set_last_error("mertens_result: |M(y)| exceeded the int32 block type");
        return MERTENS_EOVERFLOW;
    }
    if (err & kErrQueue) {
        set_last_error("mertens_result: the global gather's chunk queue overflowed");
        return MERTENS_EOVERFLOW;
    }
    if (len)
        *len = p->X[i];
    const uint64_t o = p->off[i];
    if (M_n) {
        if (cudaMemcpy(M_n, p->dR + o, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return MERTENS_ECUDA;
        p->d2h_bytes += 8;
    }
    if (entries && cap) {
        const size_t m = std::min<size_t>(cap, p->X[i]);
        if (cudaMemcpy(entries, p->dR + o, m * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return MERTENS_ECUDA;
        p->d2h_bytes += m * 8;
    }
    return MERTENS_OK;
}

int mertens_resolve(mertens_u128 n, uint64_t u, const uint64_t *S, int64_t *M_out, void *stream)
{
    if (check_n(n, "mertens_resolve", 0) != MERTENS_OK || !S || !M_out)
        return MERTENS_EINVAL;
    const u128 nn = to_u128(n);
    if (check_u(nn, u) != MERTENS_OK || nn / u >= ((u128)1 << 32)) {
        set_last_error("mertens_resolve: need floor(sqrt(n)) < u <= n and n/u < 2^32");
        return MERTENS_EINVAL;
    }
    const uint64_t X = (uint64_t)(nn / u);
    cudaStream_t s = (cudaStream_t)stream;
    const Allocator al = current_allocator();
    std::vector<uint64_t> K(X);
    for (uint64_t x = 1; x <= X; ++x) {
        const u128 k = nn / x;
        K[x - 1] = k >= kTwo63 ? 0 : (uint64_t)k;  // only k == 1 is looked at
    }
    uint64_t *dS = (uint64_t *)dev_alloc(al, X * 8);
    uint64_t *dK = (uint64_t *)dev_alloc(al, X * 8);
    uint64_t *dR = (uint64_t *)dev_alloc(al, X * 8);
    QueryDev *dq = (QueryDev *)dev_alloc(al, sizeof(QueryDev));
    int rc = MERTENS_OK;
    if (!dS || !dK || !dR || !dq)
        rc = MERTENS_ENOMEM;
    if (rc == MERTENS_OK) {
        QueryDev q;
        q.X = X;
        q.off = 0;
        if (cudaMemcpyAsync(dS, S, X * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(dK, K.data(), X * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(dq, &q, sizeof q, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            resolve_enqueue(dq, 1, dS, dK, dR, s) < 0 ||
            cudaMemcpyAsync(M_out, dR, X * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = MERTENS_ECUDA;
    }
    if (rc == MERTENS_ECUDA)
        set_last_error("mertens_resolve: %s", cudaGetErrorString(cudaGetLastError()));
    dev_free(al, dS, X * 8);
    dev_free(al, dK, X * 8);
    dev_free(al, dR, X * 8);
    dev_free(al, dq, sizeof(QueryDev));
    return rc;
}

int mertens_division_constants(uint64_t d, uint64_t *m64, uint32_t *l64, uint32_t *m32,
                               uint32_t *s32)
{
    if (d == 0 || d >= (1ull << 63)) {
        set_last_error("mertens_division_constants: need 1 <= d < 2^63");
        return MERTENS_EINVAL;
    }
    if (m64)
        *m64 = magic_of(d);
    if (l64)
        *l64 = magic_shift(d);
    uint32_t m = 0;
    unsigned sh = 0;
    if (d >= 2 && d < (1ull << 31))
        m = magic32_of((uint32_t)d, &sh);
    if (m32)
        *m32 = m;
    if (s32)
        *s32 = m ? sh : 0;
    return MERTENS_OK;
}

int mertens_window_accumulate(mertens_plan_t p, size_t i, const int64_t *mu_before,
                              size_t count, int64_t *X2_dev, void *stream)
{
    if (!p || i >= p->nq || !p->window || !X2_dev || ((uintptr_t)X2_dev & 7u) ||
        (count && !mu_before)) {
        set_last_error("mertens_window_accumulate: bad plan, index, buffer or mu sums, or not "
                       "a window plan");
        return MERTENS_EINVAL;
    }
    if (!p->ran) {
        set_last_error("mertens_window_accumulate: mertens_run was not called");
        return MERTENS_ENOTREADY;
    }
    if (p->sieves) {
        // the sieve's status words are read after the run has finished
        if (cudaEventSynchronize(p->done) != cudaSuccess) {
            set_last_error("mertens_window_accumulate: %s", cudaGetErrorString(cudaGetLastError()));
            return MERTENS_ECUDA;
        }
        const uint32_t st = sieve_scratch_status(&p->pt);
        if (st) {
            set_last_error("mertens_window_accumulate: %s", sieve_status_text(st));
            return sieve_status_code(st);
        }
    }
    // C = M(y_first - 1): the windows below this one, summed mod 2^64
    uint64_t C = 0;
    for (size_t g = 0; g < count; ++g)
        C += (uint64_t)mu_before[g];
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t o = p->off[i];
    if (cudaStreamWaitEvent(s, p->done, 0) != cudaSuccess ||
        window_accumulate_enqueue(p->dS + o, p->dcoef + o, C, p->X[i], X2_dev, s) < 0) {
        set_last_error("mertens_window_accumulate: %s", cudaGetErrorString(cudaGetLastError()));
        return MERTENS_ECUDA;
    }
    return MERTENS_OK;
}

int mertens_resolve_exchange(mertens_u128 n, uint64_t u, const int64_t *X2_dev, int64_t *M_dev,
                             void *stream)
{
    if (check_n(n, "mertens_resolve_exchange", 0) != MERTENS_OK || !X2_dev || !M_dev ||
        ((uintptr_t)X2_dev & 7u) || ((uintptr_t)M_dev & 7u))
        return MERTENS_EINVAL;
    const u128 nn = to_u128(n);
    if (check_u(nn, u) != MERTENS_OK || nn / u >= ((u128)1 << 32)) {
        set_last_error("mertens_resolve_exchange: need floor(sqrt(n)) < u <= n and n/u < 2^32");
        return MERTENS_EINVAL;
    }
    const uint64_t X = (uint64_t)(nn / u);
    cudaStream_t s = (cudaStream_t)stream;
    const Allocator al = current_allocator();
    std::vector<uint64_t> K(X);
    for (uint64_t x = 1; x <= X; ++x) {
        const u128 k = nn / x;
        K[x - 1] = k >= kTwo63 ? 0 : (uint64_t)k;  // only k == 1 is looked at
    }
    uint64_t *dS = (uint64_t *)dev_alloc(al, X * 8);
    uint64_t *dK = (uint64_t *)dev_alloc(al, X * 8);
    QueryDev *dq = (QueryDev *)dev_alloc(al, sizeof(QueryDev));
    int rc = MERTENS_OK;
    if (!dS || !dK || !dq)
        rc = MERTENS_ENOMEM;
    if (rc == MERTENS_OK) {
        QueryDev q;
        q.X = X;
        q.off = 0;
        if (cudaMemcpyAsync(dK, K.data(), X * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(dq, &q, sizeof q, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            halves_to_sums_enqueue(X2_dev, X, dS, s) < 0 ||
            resolve_enqueue(dq, 1, dS, dK, (uint64_t *)M_dev, s) < 0 ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = MERTENS_ECUDA;
    }
    if (rc == MERTENS_ECUDA)
        set_last_error("mertens_resolve_exchange: %s", cudaGetErrorString(cudaGetLastError()));
    dev_free(al, dS, X * 8);
    dev_free(al, dK, X * 8);
    dev_free(al, dq, sizeof(QueryDev));
    return rc;
}

int mertens_plan_on_table(mertens_plan_t *out, mertens_table_t table, const mertens_u128 *n,
                          size_t count, mertens_u128 u, uint64_t block_len)
{
    if (out)
        *out = nullptr;
    if (!table) {
        set_last_error("mertens_plan_on_table: NULL table");
        return MERTENS_EINVAL;
    }
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != table->device) {
        set_last_error("mertens_plan_on_table: the table lives on device %d, current is %d",
                       table->device, dev);
        return MERTENS_EINVAL;
    }
    return plan_create(out, n, count, u, block_len, tuning_now(), false, 1, UINT64_MAX, table);
}

int mertens_plan_window(mertens_plan_t *out, const mertens_u128 *n, size_t count,
                        mertens_u128 u, uint64_t block_len, uint64_t y_first, uint64_t y_last)
{
    if (out)
        *out = nullptr;
    if (y_first == 0 || y_last < y_first) {
        set_last_error("mertens_plan_window: need 1 <= y_first <= y_last");
        return MERTENS_EINVAL;
    }
    return plan_create(out, n, count, u, block_len, tuning_now(), true, y_first, y_last);
}

int mertens_window_result(mertens_plan_t p, size_t i, uint64_t *S_loc, uint64_t *coef,
                          size_t cap, size_t *len, int64_t *mu_sum)
{
    if (!p || i >= p->nq || !p->window) {
        set_last_error("mertens_window_result: bad plan, index, or not a window plan");
        return MERTENS_EINVAL;
    }
    if (!p->ran) {
        set_last_error("mertens_window_result: mertens_run was not called");
        return MERTENS_ENOTREADY;
    }
    if (cudaEventSynchronize(p->done) != cudaSuccess) {
        set_last_error("mertens_window_result: %s", cudaGetErrorString(cudaGetLastError()));
        return MERTENS_ECUDA;
    }
    if (p->sieves) {
        const uint32_t st = sieve_scratch_status(&p->pt);
        if (st) {
            set_last_error("mertens_window_result: %s", sieve_status_text(st));
            return sieve_status_code(st);
        }
    }
    uint32_t err = 0;
    if (cudaMemcpy(&err, p->derr, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return MERTENS_ECUDA;
    if (err & kErrTimeout) {
        set_last_error("mertens_window_result: a bounded wait for a bulk copy in the update "
                       "gave up");
        return MERTENS_ETIMEOUT;
    }
    if (err & kErrQueue) {
        set_last_error("mertens_window_result: the global gather's chunk queue overflowed");
        return MERTENS_EOVERFLOW;
    }
    if (len)
        *len = p->X[i];
    const uint64_t o = p->off[i];
    const size_t m = std::min<size_t>(cap, p->X[i]);
    if (S_loc && m) {
        if (cudaMemcpy(S_loc, p->dS + o, m * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return MERTENS_ECUDA;
        p->d2h_bytes += m * 8;
    }
    if (coef && m)
        memcpy(coef, p->coef.data() + o, m * 8);
    if (mu_sum) {
        *mu_sum = 0;
        if (p->nblocks &&
            cudaMemcpy(mu_sum, p->dcarry + p->nblocks, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return MERTENS_ECUDA;
    }
    return MERTENS_OK;
}

void mertens_destroy(mertens_plan_t p)
{
    if (!p)
        return;
    if (p->done) {
        cudaEventSynchronize(p->done);
        cudaEventDestroy(p->done);
    }
    clear_events(p);
    if (p->gexec)
        cudaGraphExecDestroy(p->gexec);
    if (p->cap_stream)
        cudaStreamDestroy(p->cap_stream);
    for (cudaStream_t s : {p->st_sieve, p->st_upd, p->st_dense})
        if (s)
            cudaStreamDestroy(s);
    for (cudaEvent_t e : {p->ev_fork, p->ev_reset, p->ev_dense_done, p->ev_sieve_done, p->ev_join})
        if (e)
            cudaEventDestroy(e);
    for (cudaEvent_t e : p->ev_sieved)
        if (e)
            cudaEventDestroy(e);
    for (cudaEvent_t e : p->ev_upd)
        if (e)
            cudaEventDestroy(e);
    if (p->pt.np)
        prime_table_destroy(&p->pt);
    for (auto &a : p->allocs)
        dev_free(p->al, a.first, a.second);
    delete p;
}

int mertens_plan_info(mertens_plan_t p, size_t i, mertens_query_info *info)
{
    if (!p || i >= p->nq || !info)
        return MERTENS_EINVAL;
    memset(info, 0, sizeof(*info));
    info->n.lo = p->n[i];
    info->n.hi = p->n_hi[i];
    info->u.lo = p->u[i];
    info->X = p->X[i];
    info->y_max = p->ymax_q[i];
    info->direct_terms = p->direct[i];
    info->gathered_terms = p->gathered[i];
    return MERTENS_OK;
}

int mertens_plan_set_profiling(mertens_plan_t p, int enable)
{
    if (!p)
        return MERTENS_EINVAL;
    if (p->done)
        cudaEventSynchronize(p->done);
    clear_events(p);
    p->prof = enable != 0;
    return MERTENS_OK;
}

int mertens_run_stats_get(mertens_plan_t p, mertens_run_stats *st)
{
    if (!p || !st)
        return MERTENS_EINVAL;
    memset(st, 0, sizeof(*st));
    if (!p->ran)
        return MERTENS_ENOTREADY;
    if (cudaEventSynchronize(p->done) != cudaSuccess)
        return MERTENS_ECUDA;
    st->blocks = p->nblocks;
    st->y_sieved = p->y_last >= p->y_first ? p->y_last - p->y_first + 1 : 0;
    if (p->table) {
        // blocks read from the table are not sieved
        st->y_sieved = 0;
        for (uint64_t b = 0; b < p->nblocks; ++b) {
            uint64_t y1, y2;
            block_range(p, b, &y1, &y2);
            if (y2 > p->table->y_max)
                st->y_sieved += y2 - y1 + 1;
        }
    }
    st->terms = p->terms;
    st->kernels = p->kernels;
    st->dense_y = p->dense_y;
    st->gather_j = p->gather_j;
    st->gather_j_exec = p->gather_j_exec;
    st->dense_odd_skip = p->dense_odd_skip;
    st->sieve_updates = p->sieve_updates;
    st->h2d_bytes = p->h2d_bytes;
    st->d2h_bytes = p->d2h_bytes;
    st->runs = p->prof_runs;
    if (p->prof_runs) {
        double acc[kPhases] = {0, 0, 0, 0, 0, 0};
        for (auto &e : p->evs) {
            float t = 0;
            cudaEventElapsedTime(&t, e.a, e.b);
            acc[e.phase] += t;
        }
        const double r = (double)p->prof_runs;
        st->sieve_ms = acc[kPhSieve] / r;
        st->scan_ms = acc[kPhScan] / r;
        st->dense_ms = acc[kPhDense] / r;
        st->gather_ms = acc[kPhGather] / r;
        st->update_ms = (acc[kPhDense] + acc[kPhGather]) / r;
        st->resolve_ms = acc[kPhResolve] / r;
        st->total_ms = acc[kPhTotal] / r;
    }
    return MERTENS_OK;
}

// ---- step-level entry points ----
static int sieve_window(uint64_t y1, uint64_t len, int8_t *mu_dev, int64_t carry, int32_t *M_dev,
                        void *stream)
{
    if (y1 == 0 || len == 0 || len > (1ull << 31) || y1 + len - 1 < y1 ||
        y1 + len - 1 >= (1ull << 62)) {
        set_last_error("sieve: need y1 >= 1, 1 <= len <= 2^31, y1+len-1 < 2^62");
        return MERTENS_EINVAL;
    }
    if (mu_dev && ((uintptr_t)mu_dev & 15u)) {
        set_last_error("sieve: mu_dev must be 16-byte aligned");
        return MERTENS_EINVAL;
    }
    if (M_dev && ((uintptr_t)M_dev & 3u)) {
        set_last_error("sieve: M_dev must be 4-byte aligned");
        return MERTENS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Allocator al = current_allocator();
    PrimeTable pt;
    int prc = prime_table_create(&pt, al, y1 + len - 1, s);
    if (prc == 0 && len <= (1ull << 30))
        prc = sieve_scratch_create(&pt, len);
    if (prc != 0) {
        if (pt.np)
            prime_table_destroy(&pt);
        return prc == 6 ? MERTENS_ENOTSUP : (prc == 2 ? MERTENS_ENOMEM : MERTENS_ECUDA);
    }
    const uint64_t nseg = sieve_segments(len);
    int16_t *ml = (int16_t *)dev_alloc(al, (len + 2) * 2);
    int32_t *ss = (int32_t *)dev_alloc(al, nseg * 4);
    int64_t *so = (int64_t *)dev_alloc(al, nseg * 8);
    int64_t *cy = (int64_t *)dev_alloc(al, 16);
    uint32_t *er = (uint32_t *)dev_alloc(al, 4);
    int rc = MERTENS_OK;
    if (!ml || !ss || !so || !cy || !er)
        rc = MERTENS_ENOMEM;
    if (rc == MERTENS_OK) {
        cudaMemcpyAsync(cy, &carry, 8, cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(er, 0, 4, s);
        SieveLaunch L;
        L.y1 = y1;
        L.len = len;
        L.Mloc = ml;
        L.segsum = ss;
        L.segoff = so;
        L.carry_in = cy;
        L.carry_out = cy + 1;
        L.mu_out = mu_dev;
        L.mu_base = y1;
        L.mu_end = y1 + len - 1;
        if (sieve_block_enqueue(&pt, L, s) < 0)
            rc = MERTENS_ECUDA;
        if (rc == MERTENS_OK && M_dev && expand_M_enqueue(ml, so, len, M_dev, er, s) < 0)
            rc = MERTENS_ECUDA;
        uint32_t e = 0;
        if (cudaMemcpyAsync(&e, er, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = MERTENS_ECUDA;
        // the sieve's own status first: a tile it gave up on leaves garbage
        // that the int32 check below would report instead
        if (rc == MERTENS_OK) {
            const uint32_t st = sieve_scratch_status(&pt);
            if (st) {
                set_last_error("sieve: %s", sieve_status_text(st));
                rc = sieve_status_code(st);
            }
        }
        if (rc == MERTENS_OK && (e & kErrMOverflow))
            rc = MERTENS_EOVERFLOW;
    }
    if (rc == MERTENS_ECUDA)
        set_last_error("sieve: %s", cudaGetErrorString(cudaGetLastError()));
    dev_free(al, ml, (len + 2) * 2);
    dev_free(al, ss, nseg * 4);
    dev_free(al, so, nseg * 8);
    dev_free(al, cy, 16);
    dev_free(al, er, 4);
    prime_table_destroy(&pt);
    return rc;
}

int mertens_sieve_mu(uint64_t y1, uint64_t len, int8_t *mu_dev, void *stream)
{
    if (!mu_dev)
        return MERTENS_EINVAL;
    return sieve_window(y1, len, mu_dev, 0, nullptr, stream);
}

int mertens_sieve_M(uint64_t y1, uint64_t len, int64_t carry, int32_t *M_dev, void *stream)
{
    if (!M_dev)
        return MERTENS_EINVAL;
    return sieve_window(y1, len, nullptr, carry, M_dev, stream);
}

}  // extern "C"
