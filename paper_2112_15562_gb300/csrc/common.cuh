// Shared device helpers: complex arithmetic, block reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <set>
#include <utility>

namespace gj {

template <typename R> struct CplxOf;
template <> struct CplxOf<float> { using T = float2; };
template <> struct CplxOf<double> { using T = double2; };
template <typename R> using cpx = typename CplxOf<R>::T;

template <typename C> __host__ __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
    C c; c.x = a; c.y = b; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
// Blackwell paired FP32 arithmetic: one instruction per complex add or subtract
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);  // a - b, exact product by -1
}
#endif
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
    return mk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <typename C, bool INV> __device__ __forceinline__ C mul_mi(C a) {
    return INV ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}
template <typename C> __device__ __forceinline__ C czero() { return mk<C>(0, 0); }

// Sum of `v` over the block; every thread gets the result.  `scratch` holds
// at least 32 doubles.  All threads of the block must call it.
__device__ __forceinline__ double block_sum(double v, double *scratch) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double t = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
    if (warp == 0) {
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) scratch[0] = t;
    }
    __syncthreads();
    double r = scratch[0];
    __syncthreads();
    return r;
}

// Adds per-thread partials acc[0..K) into out[0..K) (one double atomic per
// block per entry).  All K sums share one pass: warp shuffles, one barrier, and
// the first warp finishes.  `scratch` holds at least K * warps doubles (the fast
// kernels reserve 128: K <= 4 with up to 32 warps).
// All threads must call it.
template <int K, typename A>
__device__ __forceinline__ void block_accumulate(const A *acc, double *out, double *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    double v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        v[k] = (double)acc[k];
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    __syncthreads();  // scratch may still be in use by an earlier call
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) scratch[k * nw + warp] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = lane < nw ? scratch[k * nw + lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0 && out) atomicAdd(out + k, t);
        }
    }
}

// Allows launches of `f` with any dynamic shared memory up to the device's opt-in
// maximum less the kernel's static shared memory.  The attribute belongs to the
// function, not to a launch, so setting it to the maximum keeps callers with
// different sizes from overriding each other.
// Done once per kernel and device: later calls return at once, so that a product's
// launches cost no attribute queries on the host.
template <typename F>
inline cudaError_t allow_max_smem(F *f) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const std::pair<int, const void *> key{dev, reinterpret_cast<const void *>(f)};
    {
        std::lock_guard<std::mutex> lk(mu);
        if (done.count(key)) return cudaSuccess;
    }
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) optin = 48 * 1024;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    const int dyn = optin - (int)fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn > 0 ? dyn : 0);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(mu);
        done.insert(key);
    }
    return e;
}

}  // namespace gj
