// Pipe-rate probes: measured peaks for the rooflines of the force kernels
// (FP32 FMA lanes as scalar and as packed f32x2 instructions, FP64 FMA, the
// MUFU reciprocal square root).  Each thread runs kChains independent
// dependency chains of one operation; 8 CTAs of 256 threads per SM keep every
// scheduler supplied; the launch is timed with CUDA events after a warm-up
// launch.  Loop counts are fixed, every launch ends by itself.
#include <cmath>

#include "sp2_internal.h"

namespace sp2 {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 8;

__device__ __forceinline__ float2 probe_fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm volatile("{.reg .b64 pa, pb, pc, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
                 "mov.b64 pc, {%6, %7};\n\tfma.rn.ftz.f32x2 pd, pa, pb, pc;\n\tmov.b64 {%0, %1}, pd;}"
                 : "=f"(d.x), "=f"(d.y)
                 : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// KIND 0: FFMA, 1: packed f32x2 FMA, 2: DFMA, 3: MUFU rsqrt.  The result is
// stored only when keep != 0 (never, at run time), which the compiler cannot
// know, so no chain is removed.
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) probe_kernel(int iters, float a, float b, int keep, float *sink) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    float total = 0.f;
    if constexpr (KIND == 0) {
        float acc[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = 1.f + 1e-3f * static_cast<float>(k + tid % 7);
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = fmaf(acc[k], a, b);
#pragma unroll
        for (int k = 0; k < kChains; ++k) total += acc[k];
    } else if constexpr (KIND == 1) {
        float2 acc[kChains];
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = make_float2(1.f + 1e-3f * k, 1.f - 1e-3f * static_cast<float>(tid % 7));
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = probe_fma2(acc[k], a2, b2);
#pragma unroll
        for (int k = 0; k < kChains; ++k) total += acc[k].x + acc[k].y;
    } else if constexpr (KIND == 2) {
        double acc[kChains];
        const double ad = a, bd = b;
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = 1.0 + 1e-3 * static_cast<double>(k + tid % 7);
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], ad, bd);
#pragma unroll
        for (int k = 0; k < kChains; ++k) total += static_cast<float>(acc[k]);
    } else {
        float acc[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = 1.5f + 1e-3f * static_cast<float>(k + tid % 7);
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = rsqrtf(acc[k]);  // converges to 1, stays finite
#pragma unroll
        for (int k = 0; k < kChains; ++k) total += acc[k];
    }
    if (keep) sink[tid] = total;
}

// Operations per second of one probe: one warm-up launch, then one timed one.
template <int KIND>
cudaError_t time_probe(int grid, int iters, double ops_per_iter_thread, cudaStream_t s, double *rate) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        probe_kernel<KIND><<<grid, kProbeThreads, 0, s>>>(iters / 8, 0.999999f, 1e-6f, 0, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        probe_kernel<KIND><<<grid, kProbeThreads, 0, s>>>(iters, 0.999999f, 1e-6f, 0, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e == cudaSuccess)
        *rate = static_cast<double>(grid) * kProbeThreads * static_cast<double>(iters) * ops_per_iter_thread /
                (static_cast<double>(ms) * 1e-3);
    return e;
}

}  // namespace
}  // namespace sp2

extern "C" sp2_status sp2_measure_pipe_peaks(sp2_pipe_peaks *out) {
    using namespace sp2;
    if (!out) return SP2_ERR_ARG;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    const int grid = sms * kProbeCtasPerSm;
    // loop counts for launches of roughly 10-50 ms at the nominal rates
    if (e == cudaSuccess) e = time_probe<0>(grid, 1 << 17, kChains, s, &out->fp32_fma_lane_ops);
    if (e == cudaSuccess) e = time_probe<1>(grid, 1 << 16, 2.0 * kChains, s, &out->fp32x2_fma_lane_ops);
    if (e == cudaSuccess) e = time_probe<2>(grid, 1 << 11, kChains, s, &out->fp64_fma_ops);
    if (e == cudaSuccess) e = time_probe<3>(grid, 1 << 14, kChains, s, &out->rsqrt_ops);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SP2_ERR_CUDA;
    }
    return SP2_OK;
}
