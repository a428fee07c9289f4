// Batched mixed-radix FFTs in shared memory (self-sorting Stockham form).
//
// A CTA transforms B interleaved lines of length N: element j of line b lives at
// buf[j * B + b], so consecutive threads touch consecutive addresses.  Each stage
// of radix R reads the R inputs j + r N/R (r < R) of butterfly j, applies the
// twiddles W_N^(r k N/(Ns R)) with k = j mod Ns, transforms them with a length-R
// DFT in registers and writes them to (j div Ns) Ns R + k + r Ns of the other
// buffer.  Radices 2, 3, 4, 5, 7, 8 and the odd primes 11, 13, 17 are supported.
// Forward transforms use exp(-2 pi i jk/N); inverse ones are unnormalised.
#pragma once
#include "common.cuh"

namespace gj {

constexpr int kMaxStages = 16;

struct FftPlanDev {
    int N;
    int nst;
    int radix[kMaxStages];
};

// sqrt(2)/2
template <typename R> __device__ __forceinline__ R rsqrt2() { return R(0.70710678118654752440084436210485); }

template <typename R, bool INV>
__device__ __forceinline__ void dft2(cpx<R> *v) {
    cpx<R> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <typename R, bool INV>
__device__ __forceinline__ void dft4(cpx<R> &a0, cpx<R> &a1, cpx<R> &a2, cpx<R> &a3) {
    using C = cpx<R>;
    C s02 = cadd(a0, a2), d02 = csub(a0, a2);
    C s13 = cadd(a1, a3), d13 = mul_mi<C, INV>(csub(a1, a3));
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd(d02, d13);
    a3 = csub(d02, d13);
}

template <typename R, bool INV>
__device__ __forceinline__ void dft8(cpx<R> *v) {
    using C = cpx<R>;
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<R, INV>(e0, e1, e2, e3);
    dft4<R, INV>(o0, o1, o2, o3);
    const R h = rsqrt2<R>();
    // w8^1 = h(1 -+ i), w8^2 = -+i, w8^3 = h(-1 -+ i)   (upper sign forward)
    C t1 = INV ? mk<C>(h * (o1.x - o1.y), h * (o1.x + o1.y)) : mk<C>(h * (o1.x + o1.y), h * (o1.y - o1.x));
    C t2 = mul_mi<C, INV>(o2);
    C t3 = INV ? mk<C>(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : mk<C>(h * (o3.y - o3.x), -h * (o3.x + o3.y));
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, t1); v[5] = csub(e1, t1);
    v[2] = cadd(e2, t2); v[6] = csub(e2, t2);
    v[3] = cadd(e3, t3); v[7] = csub(e3, t3);
}

// Generic length-RAD DFT with roots taken from the length-N twiddle table.
template <typename R, int RAD, bool INV>
__device__ __forceinline__ void dft_generic(cpx<R> *v, const cpx<R> *tw, int N) {
    using C = cpx<R>;
    C y[RAD];
    const int step = N / RAD;
#pragma unroll
    for (int q = 0; q < RAD; ++q) {
        C acc = v[0];
#pragma unroll
        for (int r = 1; r < RAD; ++r) {
            C w = tw[step * ((r * q) % RAD)];
            if (INV) w = cconj(w);
            acc = cadd(acc, cmul(v[r], w));
        }
        y[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < RAD; ++q) v[q] = y[q];
}

template <typename R, int RAD, bool INV>
__device__ __forceinline__ void dft_small(cpx<R> *v, const cpx<R> *tw, int N) {
    if constexpr (RAD == 2) {
        dft2<R, INV>(v);
    } else if constexpr (RAD == 4) {
        dft4<R, INV>(v[0], v[1], v[2], v[3]);
    } else if constexpr (RAD == 8) {
        dft8<R, INV>(v);
    } else {
        dft_generic<R, RAD, INV>(v, tw, N);
    }
}

// One Stockham stage over B interleaved lines.  Inputs j >= valid (first stage
// only) are taken as zero.
template <typename R, int RAD, bool INV>
__device__ __forceinline__ void fft_stage(const cpx<R> *__restrict__ in, cpx<R> *__restrict__ out,
                                          int N, int Ns, int B, const cpx<R> *tw, int valid) {
    using C = cpx<R>;
    const int M = N / RAD;
    const int tws = N / (Ns * RAD);
    const int total = M * B;
    for (int it = threadIdx.x; it < total; it += blockDim.x) {
        const int b = it % B;
        const int j = it / B;
        const int k = j % Ns;
        C v[RAD];
#pragma unroll
        for (int r = 0; r < RAD; ++r) {
            const int src = j + r * M;
            v[r] = (src < valid) ? in[src * B + b] : czero<C>();
        }
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                C w = tw[r * k * tws];
                v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
            }
        }
        dft_small<R, RAD, INV>(v, tw, N);
        const int d0 = (j / Ns) * Ns * RAD + k;
#pragma unroll
        for (int r = 0; r < RAD; ++r) out[(d0 + r * Ns) * B + b] = v[r];
    }
}

// Full transform of B interleaved lines held in buf0; buf1 is scratch of the
// same size.  Returns the buffer that holds the result.  Inputs with index
// >= valid are treated as zero (their memory is never read).
template <typename R, bool INV>
__device__ cpx<R> *fft_lines(cpx<R> *buf0, cpx<R> *buf1, const FftPlanDev &plan, int B,
                             const cpx<R> *tw, int valid) {
    cpx<R> *in = buf0, *out = buf1;
    int Ns = 1;
    const int N = plan.N;
    for (int s = 0; s < plan.nst; ++s) {
        const int rad = plan.radix[s];
        const int vld = (s == 0) ? valid : N;
        switch (rad) {
            case 2: fft_stage<R, 2, INV>(in, out, N, Ns, B, tw, vld); break;
            case 3: fft_stage<R, 3, INV>(in, out, N, Ns, B, tw, vld); break;
            case 4: fft_stage<R, 4, INV>(in, out, N, Ns, B, tw, vld); break;
            case 5: fft_stage<R, 5, INV>(in, out, N, Ns, B, tw, vld); break;
            case 7: fft_stage<R, 7, INV>(in, out, N, Ns, B, tw, vld); break;
            case 8: fft_stage<R, 8, INV>(in, out, N, Ns, B, tw, vld); break;
            case 11: fft_stage<R, 11, INV>(in, out, N, Ns, B, tw, vld); break;
            case 13: fft_stage<R, 13, INV>(in, out, N, Ns, B, tw, vld); break;
            case 17: fft_stage<R, 17, INV>(in, out, N, Ns, B, tw, vld); break;
            default: break;
        }
        __syncthreads();
        Ns *= rad;
        cpx<R> *t = in; in = out; out = t;
    }
    return in;
}

}  // namespace gj
