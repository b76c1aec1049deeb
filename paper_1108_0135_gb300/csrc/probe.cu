// Integer-pipe probes: the rates of the update's inner step and of plain
// 32-bit integer arithmetic on the current device, measured with CUDA events,
// so that roofline denominators are taken on the machine that runs the
// computation (the paper has no counterpart).
//
// The update's quotient q = floor(k/d) = mulhi64(m_d, 2k) >> l_d is one
// 64x64 -> 128-bit multiply-high, a shift and an add per term; the probe runs
// exactly that step in eight independent accumulators per thread, with the
// multiplier changing every step so nothing can be hoisted; a fourth probe
// runs the shared-memory gather's float-estimate quotient the same way.
#include <cstdint>

#include "../../include/libmertens.h"
#include "common.cuh"
#include "internal.h"

using namespace mert;

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) probe_mulhi_kernel(uint64_t *out, uint64_t m0,
                                                                   int iters)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t k2 = (tid * 0x9E3779B97F4A7C15ull) | 1ull;
    const unsigned l = 20u + (unsigned)(tid & 7u);
    uint64_t acc[kProbeChains] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint64_t m = m0;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j)
            acc[j] += __umul64hi(k2, m + (uint64_t)j) >> l;
        m += 0x1234567ull;
    }
    uint64_t s = 0;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j)
        s ^= acc[j];
    out[tid] = s;
}

// The gathered terms' float-estimate quotient (the shared-memory gather's
// step): R and j stepped by fused multiply-adds, f = R (1/j) rounded to an
// integer through the 1.5 2^23 bias, one exact 32-bit remainder test.
__global__ void __launch_bounds__(kProbeThreads) probe_fquot_kernel(uint64_t *out, uint32_t t1,
                                                                   int iters)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t R[kProbeChains], j[kProbeChains], acc[kProbeChains];
    float Rf0[kProbeChains], jf0[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) {
        R[c] = (uint32_t)(tid * 977ull) + (uint32_t)c * 131u;
        j[c] = 100000000u + (uint32_t)(tid & 1023u) * 32u + (uint32_t)c;
        Rf0[c] = (float)R[c];
        jf0[c] = (float)j[c];
        acc[c] = 0;
    }
    const uint32_t dR = t1 << 5;
    const float dRf = (float)dR;
    float fi = 0.0f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
            const float Rf = __fmaf_rn(fi, dRf, Rf0[c]), jf = __fmaf_rn(fi, -32.0f, jf0[c]);
            float rj;
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rj) : "f"(jf));
            const float t = __fadd_rn(__fmaf_rn(Rf, rj, -0.53125f), 12582912.0f);
            uint32_t q = (uint32_t)(__float_as_int(t) - 0x4B400000);
            const uint32_t rem = R[c] - q * j[c];
            q += rem >= j[c] ? 1u : 0u;
            acc[c] += q;
            R[c] += dR;
            j[c] -= 32u;
        }
        fi += 1.0f;
    }
    uint64_t s = 0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c)
        s ^= acc[c];
    out[tid] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_imad_kernel(uint64_t *out, uint32_t m,
                                                                  int iters)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[kProbeChains];
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j)
        a[j] = (uint32_t)tid * 2654435761u + (uint32_t)j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j)
            a[j] = a[j] * m + (uint32_t)j;
    }
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j)
        s ^= a[j];
    out[tid] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_alu_kernel(uint64_t *out, uint32_t m,
                                                                 int iters)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[kProbeChains];
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j)
        a[j] = (uint32_t)tid * 2654435761u + (uint32_t)j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j)
            a[j] = (a[j] ^ m) + (uint32_t)(j + i);  // one LOP3 + one IADD3
    }
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j)
        s ^= a[j];
    out[tid] = s;
}

}  // namespace

extern "C" int mertens_probe_int_peaks(mertens_int_peaks *out, void *stream)
{
    if (!out)
        return MERTENS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_last_error("mertens_probe_int_peaks: no usable device");
        return MERTENS_ECUDA;
    }
    const int blocks = sms * 8, iters = 8192;
    const size_t nthr = (size_t)blocks * kProbeThreads;
    const Allocator al = current_allocator();
    uint64_t *buf = (uint64_t *)dev_alloc(al, nthr * 8);
    cudaEvent_t a = nullptr, b = nullptr;
    if (!buf || cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        dev_free(al, buf, nthr * 8);
        set_last_error("mertens_probe_int_peaks: set-up failed");
        return MERTENS_ENOMEM;
    }
    const double ops = (double)nthr * iters * kProbeChains;
    double rate[4] = {0, 0, 0, 0};
    int rc = MERTENS_OK;
    for (int which = 0; which < 4 && rc == MERTENS_OK; ++which) {
        float best = 0;
        for (int rep = 0; rep < 3; ++rep) {  // the first run warms up
            cudaEventRecord(a, s);
            if (which == 0)
                probe_mulhi_kernel<<<blocks, kProbeThreads, 0, s>>>(buf, 0xF00DBABEDEADBEEFull, iters);
            else if (which == 1)
                probe_imad_kernel<<<blocks, kProbeThreads, 0, s>>>(buf, 2654435761u, iters);
            else if (which == 2)
                probe_alu_kernel<<<blocks, kProbeThreads, 0, s>>>(buf, 2654435761u, iters);
            else
                probe_fquot_kernel<<<blocks, kProbeThreads, 0, s>>>(buf, 1000007u, iters);
            cudaEventRecord(b, s);
            float ms = 0;
            if (cudaEventSynchronize(b) != cudaSuccess ||
                cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
                rc = MERTENS_ECUDA;
                break;
            }
            if (rep > 0 && (best == 0 || ms < best))
                best = ms;
        }
        if (best > 0)
            rate[which] = ops / (best * 1e-3);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    dev_free(al, buf, nthr * 8);
    if (rc != MERTENS_OK) {
        set_last_error("mertens_probe_int_peaks: %s", cudaGetErrorString(cudaGetLastError()));
        return rc;
    }
    out->mulhi_terms_per_s = rate[0];
    out->imad32_per_s = rate[1];
    out->alu_pairs_per_s = rate[2];
    out->sms = sms;
    out->fquot_terms_per_s = rate[3];
    return MERTENS_OK;
}
