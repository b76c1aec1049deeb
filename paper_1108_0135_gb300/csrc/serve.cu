// Serving: continuous batching of M(n) queries on one device.
//
// A worker thread groups waiting queries of one magnitude class into a
// batch, which becomes one plan with one shared sieve pass (Sec. 2 of
// arXiv:1108.0135: close values need the sieve only once), and keeps several
// batches in flight on separate streams.  A batch is admitted whenever a slot
// is free and its estimated device memory fits the budget, so queries that
// arrive while others run are taken up as soon as slots and memory free up.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/libmertens.h"
#include "common.cuh"
#include "internal.h"

namespace mert {
std::vector<uint64_t> plan_auto_u(const std::vector<uint64_t> &ns);
size_t plan_device_bytes(mertens_plan_t p);
double plan_dense_factor();
}  // namespace mert

using namespace mert;

namespace {

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Query {
    uint64_t n, ticket;
};

struct Result {
    bool done = false;
    int status = MERTENS_OK;
    int64_t M = 0;
    uint64_t t_submit = 0, t_done = 0;
};

struct Inflight {
    mertens_plan_t plan = nullptr;
    int slot = 0;
    cudaEvent_t ev = nullptr;
    std::vector<uint64_t> tickets;
    size_t bytes = 0;
};

// Device memory of a batch planned on a resident table: entry arrays, and a
// sieving plan's buffers when the batch's sieve limit reaches above the table
// (those blocks are sieved).
size_t estimate_batch_bytes(const std::vector<uint64_t> &ns);
size_t estimate_table_batch_bytes(const std::vector<uint64_t> &ns, uint64_t y_max)
{
    const std::vector<uint64_t> us = plan_auto_u(ns);
    double entries = 0;
    bool above = false;
    for (size_t i = 0; i < ns.size(); ++i) {
        const uint64_t u = std::max<uint64_t>(us[i], std::min<uint64_t>(ns[i], y_max + 1));
        entries += (double)(ns[i] / u);
        above = above || u > y_max + 1;
    }
    return above ? estimate_batch_bytes(ns) : (size_t)(110.0 * entries + 64.0e6);
}

// Device memory a batch's plan will take, estimated from the plan's shapes
// (entry arrays, one sieve block of int16 M, the divisor-magic table and the
// squarefree list up to the dense cut-off, dense_c sqrt(n), dense_c at least
// 1.6), with slack.
size_t estimate_batch_bytes(const std::vector<uint64_t> &ns)
{
    double entries = 0, ymax = 0, nmax = 0;
    const std::vector<uint64_t> us = plan_auto_u(ns);
    for (size_t i = 0; i < ns.size(); ++i) {
        const uint64_t n = ns[i], u = us[i];
        entries += (double)(n / u);
        ymax = std::max(ymax, (double)u);
        nmax = std::max(nmax, (double)n);
    }
    const double L = std::min(ymax, ymax > 6.9e10 ? 1073741824.0 : 268435456.0);
    const double ydense = std::max(plan_dense_factor(), 1.6) * std::sqrt(nmax) + 8192.0;
    return (size_t)(110.0 * entries + 2.0 * L + 17.0 * ydense + 64.0e6);
}

}  // namespace

struct mertens_server_s {
    int device = 0;
    size_t budget = 0;
    uint32_t max_inflight = 4, max_batch = 128;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Query> queue;
    std::unordered_map<uint64_t, Result> results;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    std::vector<cudaStream_t> streams;
    mertens_server_stats st{};
    mertens_table_t table = nullptr;  // when set, batches that fit are planned on it
    int init_status = MERTENS_OK;
    bool ready = false;

    void finish(Inflight &f, int status)
    {
        std::vector<int64_t> vals(f.tickets.size(), 0);
        int rc = status;
        if (rc == MERTENS_OK) {
            for (size_t i = 0; i < f.tickets.size() && rc == MERTENS_OK; ++i)
                rc = mertens_result(f.plan, i, &vals[i], nullptr, 0, nullptr);
        }
        const uint64_t t = now_ns();
        {
            std::lock_guard<std::mutex> lk(mu);
            for (size_t i = 0; i < f.tickets.size(); ++i) {
                Result &r = results[f.tickets[i]];
                r.done = true;
                r.status = rc;
                r.M = vals[i];
                r.t_done = t;
            }
            st.answered += f.tickets.size();
            if (rc != MERTENS_OK)
                st.failed += f.tickets.size();
        }
        cv.notify_all();
        if (f.ev)
            cudaEventDestroy(f.ev);
        mertens_destroy(f.plan);
        f.plan = nullptr;
    }

    void run()
    {
        if (cudaSetDevice(device) != cudaSuccess) {
            init_status = MERTENS_ECUDA;
        } else {
            for (uint32_t i = 0; i < max_inflight && init_status == MERTENS_OK; ++i) {
                cudaStream_t s = nullptr;
                if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
                    init_status = MERTENS_ECUDA;
                streams.push_back(s);
            }
            if (init_status == MERTENS_OK && budget == 0) {
                size_t fr = 0, tot = 0;
                cudaMemGetInfo(&fr, &tot);
                budget = (size_t)(0.8 * (double)fr);
            }
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            ready = true;
        }
        cv.notify_all();
        if (init_status != MERTENS_OK)
            return;

        std::vector<Inflight> inflight;
        std::vector<int> free_slots;
        for (uint32_t i = 0; i < max_inflight; ++i)
            free_slots.push_back((int)i);
        size_t in_use = 0;
        for (;;) {
            bool progressed = false;
            // retire finished batches
            for (size_t i = 0; i < inflight.size();) {
                const cudaError_t q = cudaEventQuery(inflight[i].ev);
                if (q == cudaErrorNotReady) {
                    ++i;
                    continue;
                }
                finish(inflight[i], q == cudaSuccess ? MERTENS_OK : MERTENS_ECUDA);
                in_use -= inflight[i].bytes;
                free_slots.push_back(inflight[i].slot);
                inflight.erase(inflight.begin() + (long)i);
                progressed = true;
            }
            // admit new batches: the oldest waiting query's magnitude class,
            // FIFO within the class
            while (!free_slots.empty()) {
                std::vector<Query> batch;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    if (queue.empty())
                        break;
                    // classes of a factor 2^20 in n: a batch shares one sieve
                    // limit set by its largest targets (smaller ones take
                    // u = min(n, that limit)), and small queries do not wait
                    // behind the largest ones
                    const unsigned cls = bitlen64(queue.front().n) / 20;
                    for (auto it = queue.begin(); it != queue.end() && batch.size() < max_batch;) {
                        if (bitlen64(it->n) / 20 == cls) {
                            batch.push_back(*it);
                            it = queue.erase(it);
                        } else {
                            ++it;
                        }
                    }
                }
                std::vector<uint64_t> ns;
                for (const Query &q : batch)
                    ns.push_back(q.n);
                mertens_table_t tab = nullptr;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    tab = table;
                }
                uint64_t nmax = 0;
                for (uint64_t v : ns)
                    nmax = std::max(nmax, v);
                if (tab && (tab->n_max_hi == 0 && nmax > tab->n_max_lo))
                    tab = nullptr;
                const size_t est = tab ? estimate_table_batch_bytes(ns, tab->y_max)
                                       : estimate_batch_bytes(ns);
                auto put_back = [&]() {
                    std::lock_guard<std::mutex> lk(mu);
                    for (auto it = batch.rbegin(); it != batch.rend(); ++it)
                        queue.push_front(*it);
                };
                if (!inflight.empty() && in_use + est > budget) {
                    put_back();
                    break;
                }
                std::vector<mertens_u128> nv(ns.size());
                for (size_t i = 0; i < ns.size(); ++i) {
                    nv[i].lo = ns[i];
                    nv[i].hi = 0;
                }
                mertens_u128 u0 = {0, 0};
                Inflight f;
                int rc = MERTENS_ENOTSUP;
                if (tab)
                    rc = mertens_plan_on_table(&f.plan, tab, nv.data(), nv.size(), u0, 0);
                if (rc == MERTENS_ENOTSUP)
                    rc = mertens_plan(&f.plan, nv.data(), nv.size(), u0, 0);
                if (rc == MERTENS_ENOMEM && !inflight.empty()) {
                    put_back();
                    break;
                }
                for (const Query &q : batch)
                    f.tickets.push_back(q.ticket);
                f.slot = free_slots.back();
                if (rc == MERTENS_OK)
                    rc = mertens_run(f.plan, streams[f.slot]);
                if (rc == MERTENS_OK &&
                    (cudaEventCreateWithFlags(&f.ev, cudaEventDisableTiming) != cudaSuccess ||
                     cudaEventRecord(f.ev, streams[f.slot]) != cudaSuccess))
                    rc = MERTENS_ECUDA;
                if (rc != MERTENS_OK) {
                    finish(f, rc);
                    progressed = true;
                    continue;
                }
                free_slots.pop_back();
                f.bytes = std::max(est, plan_device_bytes(f.plan));
                in_use += f.bytes;
                inflight.push_back(std::move(f));
                {
                    std::lock_guard<std::mutex> lk(mu);
                    st.batches += 1;
                    st.max_inflight = std::max<uint64_t>(st.max_inflight, inflight.size());
                    st.max_batch_seen = std::max<uint64_t>(st.max_batch_seen, batch.size());
                }
                progressed = true;
            }
            {
                std::unique_lock<std::mutex> lk(mu);
                if (stop && inflight.empty())
                    break;
                if (!progressed)
                    cv.wait_for(lk, std::chrono::microseconds(inflight.empty() ? 2000 : 100));
            }
        }
        for (cudaStream_t s : streams)
            cudaStreamDestroy(s);
    }
};

extern "C" {

int mertens_server_create(mertens_server_t *out, int device, size_t mem_budget_bytes,
                          uint32_t max_inflight, uint32_t max_batch)
{
    if (!out)
        return MERTENS_EINVAL;
    *out = nullptr;
    if (max_inflight == 0)
        max_inflight = 4;
    if (max_batch == 0)
        max_batch = 128;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        set_last_error("mertens_server_create: no CUDA device");
        return MERTENS_ECUDA;
    }
    if (device < 0 || device >= ndev || max_inflight > 16 || max_batch > 4096) {
        set_last_error("mertens_server_create: need a valid device, max_inflight <= 16, "
                       "max_batch <= 4096");
        return MERTENS_EINVAL;
    }
    mertens_server_s *s = new (std::nothrow) mertens_server_s();
    if (!s)
        return MERTENS_ENOMEM;
    s->device = device;
    s->budget = mem_budget_bytes;
    s->max_inflight = max_inflight;
    s->max_batch = max_batch;
    s->worker = std::thread([s]() { s->run(); });
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv.wait(lk, [s]() { return s->ready; });
    }
    if (s->init_status != MERTENS_OK) {
        const int rc = s->init_status;
        s->worker.join();
        delete s;
        set_last_error("mertens_server_create: worker set-up failed");
        return rc;
    }
    *out = s;
    return MERTENS_OK;
}

int mertens_server_use_table(mertens_server_t s, mertens_table_t table)
{
    if (!s) {
        set_last_error("mertens_server_use_table: NULL server");
        return MERTENS_EINVAL;
    }
    if (table && table->device != s->device) {
        set_last_error("mertens_server_use_table: the table lives on another device");
        return MERTENS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->table = table;
    return MERTENS_OK;
}

int mertens_server_submit(mertens_server_t s, mertens_u128 n, uint64_t *ticket)
{
    if (!s || !ticket || (n.lo == 0 && n.hi == 0)) {
        set_last_error("mertens_server_submit: need a server, a ticket pointer and n >= 1");
        return MERTENS_EINVAL;
    }
    if (n.hi != 0 || n.lo >= (1ull << 63)) {
        set_last_error("mertens_server_submit: n >= 2^63 is not supported by this build");
        return MERTENS_ENOTSUP;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop)
            return MERTENS_EINVAL;
        const uint64_t t = s->next_ticket++;
        Result &r = s->results[t];
        r.t_submit = now_ns();
        s->queue.push_back({n.lo, t});
        s->st.submitted += 1;
        *ticket = t;
    }
    s->cv.notify_all();
    return MERTENS_OK;
}

int mertens_server_poll(mertens_server_t s, uint64_t ticket, int64_t *M_n)
{
    if (!s)
        return MERTENS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end())
        return MERTENS_EINVAL;
    if (!it->second.done)
        return MERTENS_ENOTREADY;
    if (M_n)
        *M_n = it->second.M;
    return it->second.status;
}

int mertens_server_wait(mertens_server_t s, uint64_t ticket, int64_t *M_n, double timeout_s)
{
    if (!s)
        return MERTENS_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end())
        return MERTENS_EINVAL;
    auto pred = [&]() { return it->second.done; };
    if (timeout_s < 0) {
        s->cv.wait(lk, pred);
    } else if (!s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
        return MERTENS_ETIMEOUT;
    }
    if (M_n)
        *M_n = it->second.M;
    return it->second.status;
}

int mertens_server_times(mertens_server_t s, uint64_t ticket, uint64_t *t_submit_ns,
                         uint64_t *t_done_ns)
{
    if (!s)
        return MERTENS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end())
        return MERTENS_EINVAL;
    if (t_submit_ns)
        *t_submit_ns = it->second.t_submit;
    if (t_done_ns)
        *t_done_ns = it->second.done ? it->second.t_done : 0;
    return MERTENS_OK;
}

int mertens_server_stats_get(mertens_server_t s, mertens_server_stats *out)
{
    if (!s || !out)
        return MERTENS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    return MERTENS_OK;
}

void mertens_server_destroy(mertens_server_t s)
{
    if (!s)
        return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->queue.clear();
    }
    s->cv.notify_all();
    if (s->worker.joinable())
        s->worker.join();
    delete s;
}

}  // extern "C"
