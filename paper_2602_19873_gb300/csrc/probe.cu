// FP32 issue-rate probe: the measured denominator of the ALU rooflines.
//
// The pair search and the pair passes are bound by FP32 instruction issue,
// not by memory, so their roofline needs the GPU's own FP32 rate.  This
// kernel runs long independent chains of fused multiply-adds on every lane of
// every SM (scalar fma.rn.f32, or the packed two-lane fma.rn.f32x2 of sm_100
// and later) and the entry point times it with CUDA events on the caller's
// stream.  One lane operation = one FP32 add, multiply, fused multiply-add
// or compare of one element, the unit in which the rooflines count the
// method's work; a packed instruction counts two.
#include "nl_internal.cuh"

namespace nlg {
nl_status report_error(nl_status st, const char *msg);
}

using namespace nlg;

namespace {

constexpr int kChains = 8;     // independent accumulators per thread
constexpr int kUnroll = 16;    // fused multiply-adds per chain per loop trip
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fp32_rate_scalar(float *sink, int iters, float a,
                                                               float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                asm("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(a), "f"(b));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) sink[0] = s;   // keeps the chains live; never true for a, b below
}

__global__ void __launch_bounds__(kThreads) k_fp32_rate_packed(float *sink, int iters, float a,
                                                               float b)
{
    unsigned long long x[kChains / 2];
    unsigned long long a2, b2;
    asm("mov.b64 %0, {%1, %1};" : "=l"(a2) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(b2) : "f"(b));
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) {
        float lo = (float)(threadIdx.x + 2 * c) * 1e-3f, hi = (float)(threadIdx.x + 2 * c + 1) * 1e-3f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(lo), "f"(hi));
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains / 2; ++c)
                asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(a2), "l"(b2));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == 12345.678f) sink[0] = s;
}

}  // namespace

extern "C" nl_status nl_probe_fp32_rate(int32_t packed, int32_t reps, double *ops_per_s,
                                        double *ms_out, void *stream)
{
    if (!ops_per_s) return report_error(NL_ERR_ARG, "nl_probe_fp32_rate: NULL output");
    if (reps < 1 || reps > 1000) return report_error(NL_ERR_ARG, "nl_probe_fp32_rate: reps in 1..1000");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void *fn = packed ? (const void *)k_fp32_rate_packed : (const void *)k_fp32_rate_scalar;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0);
    if (e != cudaSuccess || sms < 1 || per_sm < 1) {
        (void)cudaGetLastError();
        return report_error(NL_ERR_CUDA, "nl_probe_fp32_rate: device query failed");
    }
    const int grid = sms * per_sm;
    const int iters = 4096;   // about 10 ms per launch at 150 SMs, 2 GHz
    // the sink is never written (the guarded store cannot fire), so a null
    // pointer would do; a valid device word keeps the kernel well-defined
    float *sink = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaMallocAsync(&sink, sizeof(float), s);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    float best = 0.f;
    for (int r = -1; e == cudaSuccess && r < reps; ++r) {   // r = -1: warm-up launch
        e = cudaEventRecord(t0, s);
        if (e != cudaSuccess) break;
        if (packed)
            k_fp32_rate_packed<<<grid, kThreads, 0, s>>>(sink, iters, 0.999f, 1e-4f);
        else
            k_fp32_rate_scalar<<<grid, kThreads, 0, s>>>(sink, iters, 0.999f, 1e-4f);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(t1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && r >= 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (sink) cudaFreeAsync(sink, s);
    if (e != cudaSuccess || !(best > 0.f)) {
        (void)cudaGetLastError();
        return report_error(NL_ERR_CUDA, "nl_probe_fp32_rate: timing failed");
    }
    const double lane_ops = (double)grid * kThreads * (double)iters * kUnroll * kChains;
    *ops_per_s = lane_ops / (best * 1e-3);
    if (ms_out) *ms_out = best;
    return NL_OK;
}
