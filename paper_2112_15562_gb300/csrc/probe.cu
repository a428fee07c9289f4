// Arithmetic-rate probes: the FMA throughput of the SMs in FP32 (scalar and paired
// f32x2 instructions) and FP64, measured with CUDA events on the caller's stream.
// They give the compute rooflines against which the FFT kernels' instruction
// counts are judged; nothing here is on the solver's path.
#include <cuda_runtime.h>

#include "gj_internal.h"

namespace gj {
namespace {

constexpr int kChains = 8;  // independent FMA chains per thread (hides the FMA latency)

template <typename R>
__global__ void __launch_bounds__(256) k_fma_scalar(int iters, R a, R b, R *out) {
    R x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (R)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    R s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (R)-12345.678) out[0] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(256) k_fma_pair(int iters, float a, float b, float *out) {
    float2 x[kChains];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2((float)threadIdx.x + c, (float)c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == -12345.678f) out[0] = s;
}

}  // namespace
}  // namespace gj

extern "C" gj_status gj_probe_fma_rate(int kind, int iters, double *gflops, double *ms, gj_stream_t stream) {
    if (!gflops || !ms || iters < 1 || kind < 0 || kind > 2) {
        gj::set_error("gj_probe_fma_rate: kind must be 0, 1 or 2, iters >= 1, outputs non-NULL");
        return GJ_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    GJ_CUDA(cudaGetDevice(&dev));
    GJ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256;  // 64 warps per SM
    void *sink = nullptr;
    GJ_CUDA(cudaMalloc(&sink, sizeof(double)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&](int it) {
        if (kind == 0) gj::k_fma_scalar<float><<<blocks, threads, 0, st>>>(it, 0.999f, 1e-3f, (float *)sink);
        else if (kind == 1) gj::k_fma_pair<<<blocks, threads, 0, st>>>(it, 0.999f, 1e-3f, (float *)sink);
        else gj::k_fma_scalar<double><<<blocks, threads, 0, st>>>(it, 0.999, 1e-3, (double *)sink);
    };
    launch(iters);  // warm-up
    cudaEventRecord(e0, st);
    launch(iters);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return gj::cuda_fail(e, "gj_probe_fma_rate");
    const double lanes = (kind == 1) ? 2.0 : 1.0;  // FMAs per thread per instruction
    const double fmas = (double)blocks * threads * iters * 16.0 * gj::kChains * lanes;
    *ms = t;
    *gflops = 2.0 * fmas / (t * 1e-3) / 1e9;
    return GJ_OK;
}
