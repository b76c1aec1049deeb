// mertens_autotune: picks the performance parameters of a workload by timing
// candidate plans on the device (coordinate search).  Results never depend on
// the parameters; only the time does.
#include <cstdio>
#include <vector>

#include "../../include/libmertens.h"
#include "internal.h"

namespace mert {
int plan_create_tuned(mertens_plan_t *out, const mertens_u128 *n, size_t count,
                      const mertens_tuning &t);
}  // namespace mert

using namespace mert;

namespace {

// Milliseconds per whole run of the workload under tuning t (a warm-up run
// first, which also builds the plan's tables), or a negative status.
double time_candidate(const mertens_u128 *n, size_t count, const mertens_tuning &t, int runs,
                      cudaStream_t s, int *status)
{
    mertens_plan_t p = nullptr;
    int rc = plan_create_tuned(&p, n, count, t);
    if (rc != MERTENS_OK) {
        *status = rc;
        return -1.0;
    }
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    rc = mertens_run(p, s);
    if (rc == MERTENS_OK && cudaStreamSynchronize(s) != cudaSuccess)
        rc = MERTENS_ECUDA;
    float ms = -1.0f;
    if (rc == MERTENS_OK) {
        cudaEventRecord(a, s);
        for (int i = 0; i < runs && rc == MERTENS_OK; ++i)
            rc = mertens_run(p, s);
        cudaEventRecord(b, s);
        if (rc == MERTENS_OK && cudaEventSynchronize(b) == cudaSuccess)
            cudaEventElapsedTime(&ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    mertens_destroy(p);
    *status = rc;
    return rc == MERTENS_OK ? (double)ms / runs : -1.0;
}

}  // namespace

extern "C" int mertens_autotune(const mertens_u128 *n, size_t count, int runs,
                                mertens_tuning *best, double *best_ms)
{
    if (!n || count == 0 || !best || runs < 1 || runs > 100) {
        set_last_error("mertens_autotune: need targets, 1 <= runs <= 100 and an output");
        return MERTENS_EINVAL;
    }
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        set_last_error("mertens_autotune: cannot create a stream");
        return MERTENS_ECUDA;
    }
    mertens_tuning cur;
    mertens_get_tuning(&cur);
    int status = MERTENS_OK;
    double cur_ms = time_candidate(n, count, cur, runs, s, &status);
    if (cur_ms < 0) {
        cudaStreamDestroy(s);
        return status;
    }
    const double uf[] = {0.3, 0.45, 0.6, 0.8, 1.1};
    const double dc[] = {1.2, 1.4, 1.6, 2.1};
    const double gs[] = {0.5, 1.0, 2.0};
    for (int axis = 0; axis < 3; ++axis) {
        const double *vals = axis == 0 ? uf : (axis == 1 ? dc : gs);
        const int nv = axis == 0 ? 5 : (axis == 1 ? 4 : 3);
        mertens_tuning best_here = cur;
        double best_here_ms = cur_ms;
        for (int i = 0; i < nv; ++i) {
            mertens_tuning t = cur;
            double *field = axis == 0 ? &t.u_factor : (axis == 1 ? &t.dense_c : &t.gather_scale);
            if (*field == vals[i])
                continue;
            *field = vals[i];
            const double ms = time_candidate(n, count, t, runs, s, &status);
            if (ms >= 0 && ms < best_here_ms) {
                best_here_ms = ms;
                best_here = t;
            }
        }
        cur = best_here;
        cur_ms = best_here_ms;
    }
    cudaStreamDestroy(s);
    *best = cur;
    if (best_ms)
        *best_ms = cur_ms;
    return MERTENS_OK;
}
