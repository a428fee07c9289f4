// Column passes for a 1024-row BCCB embedding (N_y = 1024, FP32, at most 512 prisms
// and 512 stations per column; the rows run on the general kernels for any N_x, which
// write and read the transposed intermediates these kernels stream).
//
// Warp FFT.  A pruned 1024-point transform of 512 inputs splits into its even and odd
// outputs, X[2k + h] = FFT512(x[n] W1024^(h n))[k]; half-warp h computes one of them.
// Each 512-point transform is 32 x 16: lane l holds x[l + 16 j] (j < 32), takes a
// 32-point DFT over j in registers (two 16-point DFTs and a radix-2 step), multiplies
// by W1024^((2a + h) l) (the parity factor folded in), transposes through a swizzled
// 16 x 32 shared-memory tile and takes two 16-point DFTs over l, for a = l' and
// a = l' + 16.  Lane (h, l') then holds X[lambda + 64 b] in register b and
// X[lambda + 32 + 64 b] in register 16 + b (b < 16), lambda = 2 l' + h.  The inverse
// runs the steps backwards and returns y[n], n < 512, with the two halves combined
// across the half-warps, each keeping 256 of the outputs.
//
// Layouts (per field): spectra St[r][kx][ky < 1024] (the even real gravity spectrum
// as [r][kx][ky <= 512], 516 values per column), row-pass output Zt[r][kx][iy < 512],
// inverse-column output Wt[kx][jy < 512] and residual-row spectra Vt[kx][jy < 512].
#pragma once
#include "fast512.cuh"

namespace gj {
namespace f1024 {

using f512::ColItem;
using f512::View2;

constexpr int N = 1024, H = 512;
constexpr int CWF = 6;  // warps per CTA of the forward column kernel (32 KB of shared memory each)
constexpr int CWA = 8;  // warps per CTA of the adjoint column kernel (24 KB each)
constexpr int ST = f512::CSTAGES;  // TMA ring depth per warp
constexpr int KE = even_spec_len(N), KEB = KE * (int)sizeof(float);

// cos(pi j / 32) for j = 0..16
__host__ __device__ constexpr double cos_pi32(int j) {
    return j == 0 ? 1.0
         : j == 1 ? 0.995184726672196886245
         : j == 2 ? 0.980785280403230449126
         : j == 3 ? 0.956940335732208864936
         : j == 4 ? 0.923879532511286756128
         : j == 5 ? 0.881921264348355029713
         : j == 6 ? 0.831469612302545237079
         : j == 7 ? 0.773010453362736960811
         : j == 8 ? 0.707106781186547524401
         : j == 9 ? 0.634393284163645498215
         : j == 10 ? 0.555570233019602224743
         : j == 11 ? 0.471396736825997648556
         : j == 12 ? 0.382683432365089771728
         : j == 13 ? 0.290284677254462367636
         : j == 14 ? 0.195090322016128267848
         : j == 15 ? 0.0980171403295606019942
                   : 0.0;
}

// W64^j = cos(2 pi j / 64) - i sin(2 pi j / 64) for 0 <= j < 32 (j known at compile time)
template <typename R>
__device__ __forceinline__ cpx<R> w64c(int j) {
    const double c = j <= 16 ? cos_pi32(j) : -cos_pi32(32 - j);
    const double sn = j <= 16 ? cos_pi32(16 - j) : cos_pi32(j - 16);
    return mk<cpx<R>>((R)c, (R)(-sn));
}

// 32-point DFT in place, natural order in and out: the even- and odd-indexed halves
// by 16-point DFTs, then X[a] = E[a] + W32^a O[a], X[a + 16] = E[a] - W32^a O[a].
template <typename R, bool INV>
__device__ __forceinline__ void dft32(cpx<R> (&x)[32]) {
    using C = cpx<R>;
    C e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) { e[i] = x[2 * i]; o[i] = x[2 * i + 1]; }
    f512::dft16<R, INV>(e);
    f512::dft16<R, INV>(o);
#pragma unroll
    for (int a = 0; a < 16; ++a) {
        const C w = w64c<R>(2 * a);
        const C t = a == 0 ? o[a] : (INV ? cmulc(o[a], w) : cmul(o[a], w));
        x[a] = cadd(e[a], t);
        x[a + 16] = mk<C>(e[a].x - t.x, e[a].y - t.y);
    }
}

// The per-lane twiddles of one CTA, rows of 32 lanes (h, l), read from shared memory:
//   [a < 32]        forward W1024^((2a + h) l)
//   [32 + a]        inverse W1024^(2 l a) (used conjugated)
//   [64 + jj < 80]  combine W1024^(l + 16 (16 h + jj)) (used conjugated)
// The entries are the operator's W1024 table itself, so they carry no product rounding.
template <typename R>
struct Tab1024 {
    static constexpr int WORDS = 80 * 32;
    __device__ static void build(cpx<R> *t, const cpx<R> *__restrict__ tw1024) {
        for (int i = threadIdx.x; i < WORDS; i += blockDim.x) {
            const int row = i >> 5, ln = i & 31, h = ln >> 4, l = ln & 15;
            const int e = row < 32 ? (2 * row + h) * l : (row < 64 ? 2 * l * (row - 32) : l + 16 * (16 * h + row - 64));
            t[i] = __ldg(tw1024 + (e & (N - 1)));
        }
    }
};

// swizzled 16 x 32 tile of one half-warp: entry (row, col) at row * 32 + (col ^ row)
__device__ __forceinline__ int swz32(int row, int col) { return row * 32 + (col ^ row); }

// Forward pruned 1024-point transform.  In: v[j] = x[l + 16 j] (both halves).
// Out: lane (h, l) v[b] = X[lambda + 64 b], v[16 + b] = X[lambda + 32 + 64 b].
// buf: this warp's 1024-entry tile; tab: the CTA's Tab1024 (shared).
template <typename R>
__device__ __forceinline__ void fwd1024(cpx<R> (&v)[32], cpx<R> *buf, const cpx<R> *tab) {
    using C = cpx<R>;
    const int lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    C *t = buf + h * 512;
    if (h) {  // W1024^(16 j) = W64^j of the odd outputs' input factor
#pragma unroll
        for (int j = 1; j < 32; ++j) v[j] = cmul(v[j], w64c<R>(j));
    }
    dft32<R, false>(v);  // over j -> index a
#pragma unroll
    for (int a = 0; a < 32; ++a) v[a] = cmul(v[a], tab[a * 32 + lane]);
    __syncwarp();
#pragma unroll
    for (int a = 0; a < 32; ++a) t[swz32(l, a)] = v[a];
    __syncwarp();
    C p[16], q[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        p[r] = t[swz32(r, l)];
        q[r] = t[swz32(r, l + 16)];
    }
    f512::dft16<R, false>(p);  // over l -> index b, for a = this lane's l
    f512::dft16<R, false>(q);  // and for a = l + 16
#pragma unroll
    for (int b = 0; b < 16; ++b) { v[b] = p[b]; v[16 + b] = q[b]; }
}

// Inverse (unnormalised).  In: lane (h, l) v[b] = Y[lambda + 64 b], v[16 + b] =
// Y[lambda + 32 + 64 b].  Out: every lane of both halves holds y[n] for n = l + 16 j
// with j in [16 h, 16 h + 16): out[jj] = y[l + 16 (16 h + jj)].
template <typename R>
__device__ __forceinline__ void inv1024(cpx<R> (&v)[32], cpx<R> *buf, const cpx<R> *tab, cpx<R> (&out)[16]) {
    using C = cpx<R>;
    const int lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    C *t = buf + h * 512;
    C p[16], q[16];
#pragma unroll
    for (int b = 0; b < 16; ++b) { p[b] = v[b]; q[b] = v[16 + b]; }
    f512::dft16<R, true>(p);  // over b -> index r, for a = this lane's l
    f512::dft16<R, true>(q);  // and for a = l + 16
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        t[swz32(r, l)] = p[r];
        t[swz32(r, l + 16)] = q[r];
    }
    __syncwarp();
#pragma unroll
    for (int a = 0; a < 32; ++a) v[a] = cmulc(t[swz32(l, a)], tab[(32 + a) * 32 + lane]);  // W512^-(l a)
    dft32<R, true>(v);  // over a -> index j: v[j] = z_h[l + 16 j]
    // y[n] = z_0[n] + W1024^-n z_1[n]
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        C o;
        o.x = __shfl_xor_sync(0xffffffffu, v[j].x, 16);
        o.y = __shfl_xor_sync(0xffffffffu, v[j].y, 16);
        if ((j >> 4) == h) {
            const C z0 = h ? o : v[j];
            const C z1 = h ? v[j] : o;
            out[j & 15] = cadd(z0, cmulc(z1, tab[(64 + (j & 15)) * 32 + lane]));
        }
    }
}

// Position of register i's spectrum index in an even real spectrum stored for
// ky <= 512 (ky = lambda + 64 i for i < 16, lambda + 32 + 64 (i - 16) beyond; the
// entry is min(ky, 1024 - ky), which i, a compile-time index, decides).
__device__ __forceinline__ int even_pos1024(int lam, int i) {
    return i < 16 ? (i < 8 ? lam + 64 * i : N - 64 * i - lam)
                  : (i < 24 ? lam + 32 + 64 * (i - 16) : N - 32 - 64 * (i - 16) - lam);
}
__device__ __forceinline__ int ky_of(int lam, int i) { return i < 16 ? lam + 64 * i : lam + 32 + 64 * (i - 16); }

// Every CTA copies the operator's Tab1024 into shared memory with one bulk copy.
template <typename R>
__device__ __forceinline__ void load_tab(cpx<R> *tab, const cpx<R> *src, uint64_t *bar) {
    if (threadIdx.x == 0) {
        f512::mbar_expect(bar, Tab1024<R>::WORDS * sizeof(cpx<R>));
        f512::bulk_load(tab, src, Tab1024<R>::WORDS * sizeof(cpx<R>), bar);
    }
}

template <typename R>
__global__ void k_build_tab1024(cpx<R> *tab, const cpx<R> *tw1024) {
    Tab1024<R>::build(tab, tw1024);
}

// Forward column pass: for each (field, kx), Y = sum_r St_r[kx] . FFT1024(Zt_r[kx]),
// then Wt[kx][jy] = IFFT1024(Y)[jy] for jy < sy.  Persistent warps take balanced
// contiguous segments of the (kx, field, r) sequence; a column split across warps is
// summed in segment order by the last warp to finish it (as in the 512 kernels).
template <typename R>
__global__ void __launch_bounds__(CWF * 32, 1) k_col_fwd1024(View2<R> V, const int *done) {
    using C = cpx<R>;
    if (stopped(done) || f512::op_failed(V.err)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int ZB = H * sizeof(C), TB = N * sizeof(C);
    constexpr size_t WB = (size_t)ST * (ZB + TB) + N * sizeof(C);  // bytes per warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    unsigned char *wbase = smem_raw + (size_t)warp * WB;
    C *zs = reinterpret_cast<C *>(wbase);                       // ST x 512
    C *ts = reinterpret_cast<C *>(wbase + ST * ZB);             // ST x 1024
    C *xbuf = reinterpret_cast<C *>(wbase + ST * (ZB + TB));    // 1024
    C *tab = reinterpret_cast<C *>(smem_raw + (size_t)CWF * WB);
    __shared__ __align__(8) uint64_t bars[CWF][ST];
    __shared__ __align__(8) uint64_t tabbar;
    if (lane == 0)
        for (int s = 0; s < ST; ++s) f512::mbar_init(&bars[warp][s]);
    if (threadIdx.x == 0) f512::mbar_init(&tabbar);
    f512::mbar_fence_init();
    __syncthreads();
    const int nz = V.op[0].nz, sy = V.op[0].sy, NC = V.op[0].ncol;
    const long long T = (long long)V.nfield * NC * nz;
    const long long Wt = f512::seg_warps((long long)gridDim.x * CWF, T);
    const long long w = (long long)blockIdx.x * CWF + warp;
    if ((long long)blockIdx.x * CWF < Wt) load_tab<R>(tab, V.twtab, &tabbar);
    if (w >= Wt) return;
    const int t0 = (int)f512::seg_begin(w, T, Wt), t1 = (int)f512::seg_begin(w + 1, T, Wt);
    const int lam = 2 * l + h;
    ColItem cu, ci;
    cu.set(t0, nz, V.nfield);
    ci = cu;
    int ti = t0;
    auto issue = [&]() {
        const int s = (ti - t0) % ST;
        const OpView<R> &op = V.op[ci.fld];
        const size_t off = (size_t)ci.r * NC + ci.kx;
        if (op.real_spec) {
            f512::mbar_expect(&bars[warp][s], ZB + KEB);
            f512::bulk_load(zs + s * H, op.Z + off * H, ZB, &bars[warp][s]);
            f512::bulk_load(ts + s * N, reinterpret_cast<const R *>(op.spec) + off * KE, KEB, &bars[warp][s]);
        } else {
            f512::mbar_expect(&bars[warp][s], ZB + TB);
            f512::bulk_load(zs + s * H, op.Z + off * H, ZB, &bars[warp][s]);
            f512::bulk_load(ts + s * N, op.spec + off * N, TB, &bars[warp][s]);
        }
        ++ti;
        ci.next(nz, V.nfield);
    };
    if (lane == 0)
        while (ti < t1 && ti < t0 + ST) issue();
    C acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] = czero<C>();
    bool ok = __all_sync(0xffffffffu, f512::mbar_wait(&tabbar, 0, V.err));
    int t_fail = ok ? t1 : t0;
    int seg_start = t0;
    for (int t = t0; t < t1 && ok; ++t, cu.next(nz, V.nfield)) {
        const int s = (t - t0) % ST;
        const uint32_t par = (uint32_t)(((t - t0) / ST) & 1);
        ok = __all_sync(0xffffffffu, f512::mbar_wait(&bars[warp][s], par, V.err));
        if (!ok) { t_fail = t; break; }
        C v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = zs[s * H + l + 16 * j];
        fwd1024<R>(v, xbuf, tab);
        if (V.op[cu.fld].real_spec) {
            const R *tr = reinterpret_cast<const R *>(ts + s * N);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const R tt = tr[even_pos1024(lam, i)];
                acc[i] = mk<C>(acc[i].x + v[i].x * tt, acc[i].y + v[i].y * tt);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const C tt = ts[s * N + ky_of(lam, i)];
                acc[i].x = fma(v[i].x, tt.x, acc[i].x);
                acc[i].x = fma(-v[i].y, tt.y, acc[i].x);
                acc[i].y = fma(v[i].x, tt.y, acc[i].y);
                acc[i].y = fma(v[i].y, tt.x, acc[i].y);
            }
        }
        __syncwarp();
        if (lane == 0 && ti < t1) issue();
        if (cu.r == nz - 1 || t == t1 - 1) {
            const int fld = cu.fld, kx = cu.kx;
            const long long col = cu.col;
            const OpView<R> &op = V.op[fld];
            const long long cb = col * nz, ce = cb + nz - 1;
            const bool whole = (seg_start <= cb) && (t == ce);
            if (!whole) {
                const long long wf = f512::seg_owner(cb, T, Wt), wl = f512::seg_owner(ce, T, Wt);
                const int slot = (int)(w - wf), nslots = (int)(wl - wf + 1);
                C *Pc = V.P[fld] + (size_t)kx * V.slots * N;
#pragma unroll
                for (int i = 0; i < 32; ++i) Pc[(size_t)slot * N + ky_of(lam, i)] = acc[i];
                __threadfence();
                __syncwarp();
                int old = 0;
                if (lane == 0) old = atomicAdd(V.cnt[fld] + kx, 1);
                old = __shfl_sync(0xffffffffu, old, 0);
                if (old == nslots - 1) {
                    __threadfence();
#pragma unroll
                    for (int i = 0; i < 32; ++i) acc[i] = czero<C>();
                    for (int sl = 0; sl < nslots; ++sl) {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            acc[i] = cadd(acc[i], __ldcg(Pc + (size_t)sl * N + ky_of(lam, i)));
                    }
                    if (lane == 0) V.cnt[fld][kx] = 0;
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) acc[i] = czero<C>();
                    seg_start = t + 1;
                    continue;
                }
            }
            C out[16];
            inv1024<R>(acc, xbuf, tab, out);
            C *Wc = op.W + (size_t)kx * H;
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
                const int n = l + 16 * (16 * h + jj);
                if (n < sy) Wc[n] = out[jj];
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) acc[i] = czero<C>();
            seg_start = t + 1;
        }
    }
    if (!ok) f512::drain(bars[warp], t_fail, t0, t1, V.err);
}

// Adjoint column pass: for each (field, kx, r),
// Zt_r[kx][iy] = IFFT1024(conj(St_r[kx]) . FFT1024(Vt[kx]))[iy], iy < ny.
template <typename R>
__global__ void __launch_bounds__(CWA * 32, 1) k_col_adj1024(View2<R> V, const int *done) {
    using C = cpx<R>;
    if (stopped(done) || f512::op_failed(V.err)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TB = N * sizeof(C);
    constexpr size_t WB = (size_t)ST * TB + N * sizeof(C);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    unsigned char *wbase = smem_raw + (size_t)warp * WB;
    C *ts = reinterpret_cast<C *>(wbase);
    C *xbuf = reinterpret_cast<C *>(wbase + ST * TB);
    C *tab = reinterpret_cast<C *>(smem_raw + (size_t)CWA * WB);
    __shared__ __align__(8) uint64_t bars[CWA][ST];
    __shared__ __align__(8) uint64_t tabbar;
    if (lane == 0)
        for (int s = 0; s < ST; ++s) f512::mbar_init(&bars[warp][s]);
    if (threadIdx.x == 0) f512::mbar_init(&tabbar);
    f512::mbar_fence_init();
    __syncthreads();
    const int nz = V.op[0].nz, ny = V.op[0].ny, NC = V.op[0].ncol;
    const long long T = (long long)V.nfield * NC * nz;
    const long long Wt = f512::seg_warps((long long)gridDim.x * CWA, T);
    const long long w = (long long)blockIdx.x * CWA + warp;
    if ((long long)blockIdx.x * CWA < Wt) load_tab<R>(tab, V.twtab, &tabbar);
    if (w >= Wt) return;
    const int t0 = (int)f512::seg_begin(w, T, Wt), t1 = (int)f512::seg_begin(w + 1, T, Wt);
    const int lam = 2 * l + h;
    ColItem cu, ci;
    cu.set(t0, nz, V.nfield);
    ci = cu;
    int ti = t0;
    auto issue = [&]() {
        const int s = (ti - t0) % ST;
        const OpView<R> &op = V.op[ci.fld];
        const size_t off = (size_t)ci.r * NC + ci.kx;
        if (op.real_spec) {
            f512::mbar_expect(&bars[warp][s], KEB);
            f512::bulk_load(ts + s * N, reinterpret_cast<const R *>(op.spec) + off * KE, KEB, &bars[warp][s]);
        } else {
            f512::mbar_expect(&bars[warp][s], TB);
            f512::bulk_load(ts + s * N, op.spec + off * N, TB, &bars[warp][s]);
        }
        ++ti;
        ci.next(nz, V.nfield);
    };
    if (lane == 0)
        while (ti < t1 && ti < t0 + ST) issue();
    C vh[32];
    bool ok = __all_sync(0xffffffffu, f512::mbar_wait(&tabbar, 0, V.err));
    int t_fail = ok ? t1 : t0;
    for (int t = t0; t < t1 && ok; ++t, cu.next(nz, V.nfield)) {
        const int r = cu.r, fld = cu.fld, kx = cu.kx;
        const OpView<R> &op = V.op[fld];
        if (t == t0 || r == 0) {  // a new column: V^ = FFT1024 of the residual column (rows >= sy are zero)
            const C *Vc = op.V + (size_t)kx * H;
#pragma unroll
            for (int j = 0; j < 32; ++j) vh[j] = Vc[l + 16 * j];
            fwd1024<R>(vh, xbuf, tab);
        }
        const int s = (t - t0) % ST;
        const uint32_t par = (uint32_t)(((t - t0) / ST) & 1);
        ok = __all_sync(0xffffffffu, f512::mbar_wait(&bars[warp][s], par, V.err));
        if (!ok) { t_fail = t; break; }
        C v[32];
        if (op.real_spec) {
            const R *tr = reinterpret_cast<const R *>(ts + s * N);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const R tt = tr[even_pos1024(lam, i)];
                v[i] = mk<C>(vh[i].x * tt, vh[i].y * tt);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = cmulc(vh[i], ts[s * N + ky_of(lam, i)]);
        }
        __syncwarp();
        if (lane == 0 && ti < t1) issue();
        C out[16];
        inv1024<R>(v, xbuf, tab, out);
        C *Zc = op.Z + ((size_t)r * NC + kx) * H;
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
            const int n = l + 16 * (16 * h + jj);
            if (n < ny) Zc[n] = out[jj];
        }
    }
    if (!ok) f512::drain(bars[warp], t_fail, t0, t1, V.err);
}

// ---------------------------------------------------------------------------
// Row passes for N_x = 1024 (with the N_y = 1024 column kernels): real lines <->
// half spectra in the transposed layout, through the general kernels' per-element
// functors.  A CTA of RW warps runs one complex transform per warp: two lines of one
// field (pair map, joint = 0) or one line of each field (joint = 1).  The half
// spectra of the CTA's lines meet in a shared tile [slot][k < 513] (slot stride 513,
// odd, so that a warp's 16 slots of one k fall in distinct bank pairs) and move to or
// from the transposed layout with consecutive lines in consecutive words; each thread
// keeps one slot, so its line's address is formed once.  The warps' transform buffers
// share the tile's memory (barriers separate the two uses), so that two CTAs fit an SM.

constexpr int RW = 8;                 // warps (transforms) per CTA
constexpr int RSLOT = 2 * RW;         // tile slots: two lines per transform
constexpr int NCR = N / 2 + 1;        // 513 bins
constexpr int TP = NCR;               // tile slot stride
static_assert((RW * 32) % RSLOT == 0, "a thread keeps one tile slot");

// register of spectrum index lambda + 32 m in the forward transform's lane layout
__host__ __device__ constexpr int reg_of(int m) { return (m & 1) ? 16 + (m >> 1) : (m >> 1); }

// tile slot s of the CTA -> its line and field, and whether it exists
__device__ __forceinline__ bool slot_line(const PairMap &pm, int base, int s, int &line, int &field) {
    const int np = pm.npairs();
    if (pm.joint) {
        field = s / RW;
        const int q = base + (s % RW);
        line = q;
        return q < np;
    }
    field = 0;
    const int q = base + (s >> 1);
    line = 2 * q + (s & 1);
    return q < np && line < pm.nlines;
}

// The operator's twiddle table into shared memory with 16-byte asynchronous copies,
// all in flight at once (committed as one group; the caller waits and synchronises).
template <typename R>
__device__ __forceinline__ void load_tab_async(cpx<R> *tab, const cpx<R> *src) {
    constexpr int CH = Tab1024<R>::WORDS * (int)sizeof(cpx<R>) / 16;
    const char *s = reinterpret_cast<const char *>(src);
    char *d = reinterpret_cast<char *>(tab);
    for (int i = threadIdx.x; i < CH; i += blockDim.x) f512::cp_async16(d + 16 * i, s + 16 * i);
    f512::cp_async_commit();
}

// words of the tile / transform-buffer overlay
constexpr int row_overlay_words() { return RSLOT * TP > RW * N ? RSLOT * TP : RW * N; }

template <typename R, class Pro>
__global__ void __launch_bounds__(RW * 32, 2) k_row_fwd1024(OpView<R> op, PairMap pm, int n_in, cpx<R> *out0,
                                                            cpx<R> *out1, const cpx<R> *tab_src, Pro pro,
                                                            const int *done) {
    using C = cpx<R>;
    if (stopped(done)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tab = reinterpret_cast<C *>(smem_raw);
    C *tile = tab + Tab1024<R>::WORDS;  // [RSLOT][TP], or the warps' buffers before it is filled
    __shared__ double red[128];
    pro.init();
    load_tab_async<R>(tab, tab_src);  // in flight while the lines are read
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    const int base = blockIdx.x * RW, q = base + warp;
    const bool act = q < pm.npairs();
    C *buf = tile + warp * N;
    C v[32];
    if (act) {
        int la, lb;
        bool hb;
        pm.lines(q, la, lb, hb);
        // every element through the functor once (all loads issued before the first
        // store), then the lane layout of the transform
        R a[16], b[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int e = lane + 32 * i;
            a[i] = b[i] = R(0);
            if (e < n_in) field_functor(pro, blockIdx.y).fetch(la, lb, hb, e, a[i], b[i]);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) buf[lane + 32 * i] = mk<C>(a[i], b[i]);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = buf[l + 16 * j];
        __syncwarp();
    }
    f512::cp_async_wait<0>();
    __syncthreads();  // the table is in
    if (act) fwd1024<R>(v, buf, tab);
    __syncthreads();  // the buffers become the tile
    if (act) {
        // Z = FFT(a + i b) -> A = (Z[k] + conj Z[N - k]) / 2, B = (Z[k] - conj Z[N - k]) / 2i,
        // k <= 512.  For lambda != 0, Z[N - k] sits in lane (h, 16 - l - h) at m' = 31 - m;
        // lane 0 (lambda = 0) holds it at m' = 32 - m.
        const int sa = pm.joint ? warp : 2 * warp, sb = pm.joint ? RW + warp : 2 * warp + 1;
        const int partner = h ? 31 - l : ((16 - l) & 15);
        const int lam = 2 * l + h;
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            C zm;
            zm.x = __shfl_sync(0xffffffffu, v[reg_of(31 - m)].x, partner);
            zm.y = __shfl_sync(0xffffffffu, v[reg_of(31 - m)].y, partner);
            if (lane == 0) zm = v[reg_of((32 - m) & 31)];
            const C zk = v[reg_of(m)];
            const int k = lam + 32 * m;
            tile[sa * TP + k] = mk<C>(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y));
            tile[sb * TP + k] = mk<C>(R(0.5) * (zk.y + zm.y), R(-0.5) * (zk.x - zm.x));
        }
        if (lane == 0) {  // k = 512 is its own partner
            tile[sa * TP + H] = mk<C>(v[reg_of(16)].x, R(0));
            tile[sb * TP + H] = mk<C>(v[reg_of(16)].y, R(0));
        }
    }
    __syncthreads();
    {
        const int s = threadIdx.x % RSLOT;
        int line, field;
        if (slot_line(pm, base, s, line, field)) {
            if (!pm.joint) field = blockIdx.y;  // pairs of one field: the launch's grid y
            C *o = (field ? out1 : out0) + pm.at(line, 0, op.ncol, op.tcol);
            const size_t step = op.tcol ? (size_t)op.tcol : 1;
            for (int k = threadIdx.x / RSLOT; k < NCR; k += blockDim.x / RSLOT) o[k * step] = tile[s * TP + k];
        }
    }
    pro.flush(red);
}

template <typename R, class Epi>
__global__ void __launch_bounds__(RW * 32, 2) k_row_inv1024(OpView<R> op, PairMap pm, int n_out, const cpx<R> *in0,
                                                            const cpx<R> *in1, const cpx<R> *tab_src, Epi epi,
                                                            const int *done) {
    using C = cpx<R>;
    if (stopped(done)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tab = reinterpret_cast<C *>(smem_raw);
    C *tile = tab + Tab1024<R>::WORDS;  // [RSLOT][TP], then the warps' buffers
    __shared__ double red[128];
    epi.init();
    load_tab_async<R>(tab, tab_src);
    const int base = blockIdx.x * RW;
    {
        const int s = threadIdx.x % RSLOT;
        int line, field;
        const bool ok = slot_line(pm, base, s, line, field);
        if (!pm.joint) field = blockIdx.y;  // pairs of one field: the launch's grid y
        const C *src = ok ? (field ? in1 : in0) + pm.at(line, 0, op.ncol, op.tcol) : nullptr;
        const size_t step = op.tcol ? (size_t)op.tcol : 1;
        // every copy of the CTA's half spectra in flight at once (asynchronous copies)
        for (int k = threadIdx.x / RSLOT; k < NCR; k += blockDim.x / RSLOT) {
            C *dst = tile + s * TP + k;
            if (!ok) *dst = czero<C>();
            else if constexpr (sizeof(C) == 8) f512::cp_async8(dst, src + k * step);
            else f512::cp_async16(dst, src + k * step);
        }
        f512::cp_async_commit();
        f512::cp_async_wait<0>();
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    const int q = base + warp;
    const bool act = q < pm.npairs();
    int la = 0, lb = 0;
    bool hb = false;
    C v[32];
    if (act) {
        pm.lines(q, la, lb, hb);
        const int sa = pm.joint ? warp : 2 * warp, sb = pm.joint ? RW + warp : 2 * warp + 1;
        const int lam = 2 * l + h;
        // Hermitian-extended A + i B in the lane layout (an absent second line reads as zero)
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            const int k = lam + 32 * m;
            const bool lo = k <= H;
            const int kk = lo ? k : N - k;
            C A = tile[sa * TP + kk], B = tile[sb * TP + kk];
            if (kk == 0 || kk == H) { A.y = 0; B.y = 0; }
            v[reg_of(m)] = lo ? mk<C>(A.x - B.y, A.y + B.x) : mk<C>(A.x + B.y, B.x - A.y);
        }
    }
    __syncthreads();  // the tile becomes the warps' buffers
    if (act) {
        C out[16];
        inv1024<R>(v, tile + warp * N, tab, out);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
            const int n = l + 16 * (16 * h + jj);
            if (n < n_out) field_functor(epi, blockIdx.y).store(la, lb, hb, n, out[jj].x, out[jj].y);
        }
    }
    epi.flush(red);
}

template <typename R> inline size_t smem_row() {
    return ((size_t)Tab1024<R>::WORDS + (size_t)row_overlay_words()) * sizeof(cpx<R>);
}

template <typename R> inline size_t smem_col_fwd() {
    return (size_t)CWF * ((size_t)ST * (H + N) + N) * sizeof(cpx<R>) + Tab1024<R>::WORDS * sizeof(cpx<R>);
}
template <typename R> inline size_t smem_col_adj() {
    return (size_t)CWA * ((size_t)ST * N + N) * sizeof(cpx<R>) + Tab1024<R>::WORDS * sizeof(cpx<R>);
}

}  // namespace f1024
}  // namespace gj
