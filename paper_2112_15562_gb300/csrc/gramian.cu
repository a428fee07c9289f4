// The Gramian coupling term (Eq. Gramian) and its ascent directions (RRCG:2-3).
#include <mutex>
#include <string>

#include "view.cuh"

namespace gj {

// Pass 1: per-block partial sums of (m1,m1), (m2,m2), (m1,m2).  Products and the
// per-thread sums use the vector precision; block and grid sums use FP64.
template <typename R>
__global__ void __launch_bounds__(256) k_gram_dots(int64_t n, const R *m1, const R *m2, double *part) {
    __shared__ double red[32];
    R a11 = 0, a22 = 0, a12 = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R x = m1[i], y = m2[i];
        a11 += x * x; a22 += y * y; a12 += x * y;
    }
    const double s11 = block_sum((double)a11, red);
    const double s22 = block_sum((double)a22, red);
    const double s12 = block_sum((double)a12, red);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = s11;
        part[3 * blockIdx.x + 1] = s22;
        part[3 * blockIdx.x + 2] = s12;
    }
}

// Pass 2 (one block): fixed-order sum of the partials into sums[0..3).
__global__ void k_gram_finish(int nb, const double *part, double *sums) {
    __shared__ double red[32];
    for (int c = 0; c < 3; ++c) {
        double t = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) t += part[3 * b + c];
        t = block_sum(t, red);
        if (threadIdx.x == 0) sums[c] = t;
    }
}

// Pass 3: ascent directions and ||m2 - (a12/a11) m1||^2 partials, which give
// S = a11 ||m2 - (a12/a11) m1||^2 without the cancellation of a11 a22 - a12^2.
template <typename R>
__global__ void __launch_bounds__(256) k_gram_dirs(int64_t n, const R *m1, const R *m2, const double *sums,
                                                   R *l1, R *l2, double *part) {
    __shared__ double red[32];
    const double a11 = sums[0], a22 = sums[1], a12 = sums[2];
    const R c11 = (R)a11, c22 = (R)a22, c12 = (R)a12;
    const R ratio = a11 > 0 ? (R)(a12 / a11) : R(0);
    R res = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R x = m1[i], y = m2[i];
        if (l1) l1[i] = c22 * x - c12 * y;
        if (l2) l2[i] = c11 * y - c12 * x;
        const R d = y - ratio * x;
        res += d * d;
    }
    const double s = block_sum((double)res, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_gram_value(int nb, const double *part, const double *sums, double *S) {
    __shared__ double red[32];
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) t += part[b];
    t = block_sum(t, red);
    if (threadIdx.x == 0) *S = sums[0] > 0 ? sums[0] * t : 0.0;
}

template <typename R>
static gj_status gramian_launch(int64_t n, const void *m1, const void *m2, double *S, void *l1, void *l2,
                                cudaStream_t st) {
    const int nb = (int)std::min<int64_t>(4 * 152, std::max<int64_t>(1, (n + 255) / 256));
    double *scratch = nullptr;
    GJ_CUDA(cudaMallocAsync(&scratch, (3 * nb + 3) * sizeof(double), st));
    double *part = scratch, *sums = scratch + 3 * nb;
    k_gram_dots<R><<<nb, 256, 0, st>>>(n, (const R *)m1, (const R *)m2, part);
    k_gram_finish<<<1, 256, 0, st>>>(nb, part, sums);
    k_gram_dirs<R><<<nb, 256, 0, st>>>(n, (const R *)m1, (const R *)m2, sums, (R *)l1, (R *)l2, part);
    k_gram_value<<<1, 256, 0, st>>>(nb, part, sums, S);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "gramian launch");
    return GJ_OK;
}

}  // namespace gj

// Pearson coefficient of two vectors: means in a first pass, centred sums in a
// second (FP64 accumulation), the ratio in one thread.
namespace gj {
template <typename R>
__global__ void __launch_bounds__(256) k_sums2(int64_t n, const R *a, const R *b, double *part) {
    __shared__ double red[32];
    double sa = 0, sb = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        sa += (double)a[i];
        sb += (double)b[i];
    }
    sa = block_sum(sa, red);
    sb = block_sum(sb, red);
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = sa; part[2 * blockIdx.x + 1] = sb; }
}
template <typename R>
__global__ void __launch_bounds__(256) k_centred3(int64_t n, const R *a, const R *b, const double *part, int nb,
                                                  double *part2) {
    __shared__ double red[32];
    __shared__ double mean[2];
    if (threadIdx.x < 2) {
        double t = 0;
        for (int k = 0; k < nb; ++k) t += part[2 * k + threadIdx.x];
        mean[threadIdx.x] = t / (double)n;
    }
    __syncthreads();
    const double ma = mean[0], mb = mean[1];
    double saa = 0, sbb = 0, sab = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = (double)a[i] - ma, y = (double)b[i] - mb;
        saa += x * x; sbb += y * y; sab += x * y;
    }
    saa = block_sum(saa, red);
    sbb = block_sum(sbb, red);
    sab = block_sum(sab, red);
    if (threadIdx.x == 0) { part2[3 * blockIdx.x] = saa; part2[3 * blockIdx.x + 1] = sbb; part2[3 * blockIdx.x + 2] = sab; }
}
__global__ void k_pearson_finish(int nb, const double *part2, double *r) {
    double saa = 0, sbb = 0, sab = 0;
    for (int k = 0; k < nb; ++k) { saa += part2[3 * k]; sbb += part2[3 * k + 1]; sab += part2[3 * k + 2]; }
    const double den = sqrt(saa * sbb);
    *r = den > 0 ? sab / den : 0.0;
}
template <typename R>
static gj_status pearson_launch(int64_t n, const void *a, const void *b, double *r, cudaStream_t st) {
    const int nb = (int)std::min<int64_t>(2 * 152, std::max<int64_t>(1, (n + 255) / 256));
    double *scratch = nullptr;
    GJ_CUDA(cudaMallocAsync(&scratch, 5 * (size_t)nb * sizeof(double), st));
    k_sums2<R><<<nb, 256, 0, st>>>(n, (const R *)a, (const R *)b, scratch);
    k_centred3<R><<<nb, 256, 0, st>>>(n, (const R *)a, (const R *)b, scratch, nb, scratch + 2 * nb);
    k_pearson_finish<<<1, 1, 0, st>>>(nb, scratch + 2 * nb, r);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(scratch, st);
    return e == cudaSuccess ? GJ_OK : cuda_fail(e, "pearson launch");
}
}  // namespace gj

extern "C" gj_status gj_pearson(int64_t n, gj_precision prec, const void *a, const void *b, double *r,
                                gj_stream_t stream) {
    if (n < 1 || !a || !b || !r) { gj::set_error("gj_pearson: bad argument"); return GJ_ERR_ARG; }
    if (prec != GJ_FP64 && prec != GJ_FP32_MIXED) { gj::set_error("gj_pearson: bad precision"); return GJ_ERR_ARG; }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return prec == GJ_FP64 ? gj::pearson_launch<double>(n, a, b, r, st) : gj::pearson_launch<float>(n, a, b, r, st);
}

extern "C" gj_status gj_gramian_value_grad(int64_t n, gj_precision prec, const void *m1, const void *m2,
                                           double *S, void *l1, void *l2, gj_stream_t stream) {
    if (n < 1 || !m1 || !m2 || !S) { gj::set_error("gj_gramian_value_grad: bad argument"); return GJ_ERR_ARG; }
    if (prec != GJ_FP64 && prec != GJ_FP32_MIXED) { gj::set_error("gj_gramian_value_grad: bad precision"); return GJ_ERR_ARG; }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return prec == GJ_FP64 ? gj::gramian_launch<double>(n, m1, m2, S, l1, l2, st)
                           : gj::gramian_launch<float>(n, m1, m2, S, l1, l2, st);
}

// ---------------------------------------------------------------------------
// Allocation-free variant.  The reduction scratch lives in a file-scope device
// array (every GPU that loads the library keeps it until exit) instead of a
// per-call cudaMallocAsync.  Host code never passes the array's name to a kernel
// (on the host it is only a stand-in symbol): its device address is looked up once
// per device with cudaGetSymbolAddress while that device is current.

namespace gj {
namespace {

constexpr int kNoAllocMaxBlocks = 4096;             // partial sums per call
constexpr int64_t kNoAllocChunk = 4096;             // elements per block
constexpr int64_t kNoAllocMaxN = (int64_t)kNoAllocMaxBlocks * kNoAllocChunk;  // 16,777,216
constexpr int kNoAllocDoubles = 3 * kNoAllocMaxBlocks + 3 + kNoAllocMaxBlocks;  // 131,096 bytes
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

std::mutex g_noalloc_mu;
double *g_noalloc_addr[kMaxDevices] = {};

gj_status noalloc_scratch(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "gj_gramian_value_grad_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("gj_gramian_value_grad_noalloc: device index above 63");
        return GJ_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "gj_gramian_value_grad_noalloc: cudaGetSymbolAddress");
        g_noalloc_addr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_addr[dev];
    return GJ_OK;
}

template <typename R>
gj_status gramian_launch_noalloc(int64_t n, const void *m1, const void *m2, double *S, void *l1, void *l2,
                                 cudaStream_t st) {
    double *scratch = nullptr;
    gj_status rc = noalloc_scratch(&scratch);
    if (rc != GJ_OK) return rc;
    const int nb = (int)((n + kNoAllocChunk - 1) / kNoAllocChunk);
    double *part = scratch;                                  // 3 per block
    double *sums = scratch + 3 * kNoAllocMaxBlocks;          // 3
    double *part2 = sums + 3;                                // 1 per block
    // every slot that is read is written earlier in the same call: nothing needs clearing
    k_gram_dots<R><<<nb, 256, 0, st>>>(n, (const R *)m1, (const R *)m2, part);
    k_gram_finish<<<1, 256, 0, st>>>(nb, part, sums);
    k_gram_dirs<R><<<nb, 256, 0, st>>>(n, (const R *)m1, (const R *)m2, sums, (R *)l1, (R *)l2, part2);
    k_gram_value<<<1, 256, 0, st>>>(nb, part2, sums, S);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GJ_OK : cuda_fail(e, "gramian (no allocation) launch");
}

}  // namespace
}  // namespace gj

extern "C" gj_status gj_gramian_value_grad_noalloc(int64_t n, gj_precision prec, const void *m1, const void *m2,
                                                   double *S, void *l1, void *l2, gj_stream_t stream) {
    if (n > gj::kNoAllocMaxN) {
        gj::set_error("gj_gramian_value_grad_noalloc: n = " + std::to_string(n) +
                      " exceeds the allocation-free limit of 16777216 elements (use gj_gramian_value_grad)");
        return GJ_ERR_ARG;
    }
    if (n < 1 || !m1 || !m2 || !S) { gj::set_error("gj_gramian_value_grad_noalloc: bad argument"); return GJ_ERR_ARG; }
    if (prec != GJ_FP64 && prec != GJ_FP32_MIXED) {
        gj::set_error("gj_gramian_value_grad_noalloc: bad precision");
        return GJ_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return prec == GJ_FP64 ? gj::gramian_launch_noalloc<double>(n, m1, m2, S, l1, l2, st)
                           : gj::gramian_launch_noalloc<float>(n, m1, m2, S, l1, l2, st);
}
