// Specialised kernels for a 512 x 512 BCCB embedding with at most 256 prisms and
// 256 stations per direction (the zero-padded half of every transform is never
// read or computed).
//
// Warp FFT.  A pruned 512-point transform of 256 inputs x[n] splits into its even
// and odd outputs, X[2k + h] = FFT256(x[n] W512^(h n))[k]; half-warp h computes one
// of them.  Each 256-point transform is 16 x 16: lane l holds x[l + 16 j]
// (j < 16), takes a 16-point DFT over j, multiplies by W256^(l k2), transposes
// through a swizzled shared-memory tile and takes a second 16-point DFT over l.
// Lane (h, k2) then holds X[2(k2 + 16 k1) + h] = X[lambda + 32 k1] in register k1,
// lambda = 2 k2 + h.  The inverse runs the same steps backwards and returns
// y[n], n < 256, with the even/odd halves combined across the two half-warps.
//
// Layouts (per field): row-pass output Zt[r][kx][iy] (kx < 257, iy < 256),
// spectra St[r][kx][ky] (ky < 512), inverse-column output Wt[kx][jy].  Every
// column a warp streams is contiguous (2 KB or 4 KB), fetched with 1-D TMA bulk
// copies into a per-warp ring completed by mbarriers.
#pragma once
#include "bttb_kernels.cuh"
#include "gj.h"

namespace gj {
namespace f512 {

constexpr int N = 512, H = 256, NC = 257;
constexpr int CWARPS = 12;        // warps per CTA of the persistent column kernels (one CTA per SM)
constexpr int CSTAGES = 2;        // TMA ring depth per warp of the column kernels
constexpr long long kSpinLimit = 1LL << 26;  // bounded mbarrier waits

// ---------------------------------------------------------------------------
// small DFTs in registers

template <typename R> struct K16;
template <> struct K16<float> {
    static __device__ __forceinline__ float c1() { return 0.92387953251128675613f; }
    static __device__ __forceinline__ float s1() { return 0.38268343236508977173f; }
    static __device__ __forceinline__ float r2() { return 0.70710678118654752440f; }
};
template <> struct K16<double> {
    static __device__ __forceinline__ double c1() { return 0.92387953251128675613; }
    static __device__ __forceinline__ double s1() { return 0.38268343236508977173; }
    static __device__ __forceinline__ double r2() { return 0.70710678118654752440; }
};

// multiply by W16^e (forward) or W16^-e (inverse) for e in {0,1,2,3,4,6,9}
template <typename R, bool INV, int E>
__device__ __forceinline__ cpx<R> w16(cpx<R> a) {
    using C = cpx<R>;
    const R c1 = K16<R>::c1(), s1 = K16<R>::s1(), r2 = K16<R>::r2();
    const R sg = INV ? R(1) : R(-1);  // sign of the imaginary part of the root
    if constexpr (E == 0) return a;
    else if constexpr (E == 1) { const R wr = c1, wi = sg * s1; return mk<C>(a.x * wr - a.y * wi, a.x * wi + a.y * wr); }
    else if constexpr (E == 2) { const R wr = r2, wi = sg * r2; return mk<C>(a.x * wr - a.y * wi, a.x * wi + a.y * wr); }
    else if constexpr (E == 3) { const R wr = s1, wi = sg * c1; return mk<C>(a.x * wr - a.y * wi, a.x * wi + a.y * wr); }
    else if constexpr (E == 4) return mul_mi<C, INV>(a);
    else if constexpr (E == 6) { const R wr = -r2, wi = sg * r2; return mk<C>(a.x * wr - a.y * wi, a.x * wi + a.y * wr); }
    else { static_assert(E == 9, "w16"); const R wr = -c1, wi = -sg * s1; return mk<C>(a.x * wr - a.y * wi, a.x * wi + a.y * wr); }
}

template <typename R, bool INV, int N2>
__device__ __forceinline__ void tw_col(cpx<R> (&y)[16]) {
    // y[n2 + 4 k1] *= W16^(n2 k1)
    y[N2 + 4] = w16<R, INV, N2 * 1>(y[N2 + 4]);
    y[N2 + 8] = w16<R, INV, N2 * 2>(y[N2 + 8]);
    y[N2 + 12] = w16<R, INV, N2 * 3>(y[N2 + 12]);
}

// 16-point DFT in place, natural order in and out.
template <typename R, bool INV>
__device__ __forceinline__ void dft16(cpx<R> (&x)[16]) {
    using C = cpx<R>;
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<R, INV>(x[n2], x[n2 + 4], x[n2 + 8], x[n2 + 12]);
    tw_col<R, INV, 1>(x);
    tw_col<R, INV, 2>(x);
    tw_col<R, INV, 3>(x);
    // now x[n2 + 4 k1] = Y[n2][k1]; DFT4 over n2 gives X[k1 + 4 k2]
    C o[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        C a0 = x[4 * k1 + 0], a1 = x[4 * k1 + 1], a2 = x[4 * k1 + 2], a3 = x[4 * k1 + 3];
        dft4<R, INV>(a0, a1, a2, a3);
        o[k1 + 0] = a0; o[k1 + 4] = a1; o[k1 + 8] = a2; o[k1 + 12] = a3;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = o[i];
}

// cos(pi j / 16) for j = 0..8 (W32^j = cos(pi j/16) - i sin(pi j/16))
__host__ __device__ constexpr double cos_pi16(int j) {
    return j == 0 ? 1.0
         : j == 1 ? 0.98078528040323044913
         : j == 2 ? 0.92387953251128675613
         : j == 3 ? 0.83146961230254523708
         : j == 4 ? 0.70710678118654752440
         : j == 5 ? 0.55557023301960222474
         : j == 6 ? 0.38268343236508977173
         : j == 7 ? 0.19509032201612826785
                  : 0.0;
}

template <typename R>
__device__ __forceinline__ cpx<R> w32c(int j) {  // W32^j for 0 <= j < 16 (j known at compile time)
    const double c = j <= 8 ? cos_pi16(j) : -cos_pi16(16 - j);
    const double sn = j <= 8 ? cos_pi16(8 - j) : cos_pi16(j - 8);
    return mk<cpx<R>>((R)c, (R)(-sn));
}

// Per-lane twiddles, l = lane & 15.  Inverse form (load_inv): W256^(l k) =
// lo[k & 3] * hi[k >> 2] and pre = W512^l.  Forward form (load_fwd): the odd
// half-warp's factor W512^l is folded into hi, so that
// lo[k & 3] * hi[k >> 2] = W512^(h l) W256^(l k) and the odd half only needs the
// constant factors W32^j before its first DFT (W512^(l + 16 j) = W512^l W32^j).
template <typename R>
struct LaneTw {
    cpx<R> lo[4], hi[4], pre;
    __device__ void load_inv(const cpx<R> *__restrict__ tw512) {  // tw512[k] = W512^k (global, read-only)
        const int l = threadIdx.x & 15;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            lo[k] = __ldg(tw512 + ((2 * l * k) & 511));
            hi[k] = __ldg(tw512 + ((8 * l * k) & 511));
        }
        pre = __ldg(tw512 + l);
    }
    __device__ void load_fwd(const cpx<R> *__restrict__ tw512) {
        load_inv(tw512);
        if (threadIdx.x & 16) {
#pragma unroll
            for (int k = 0; k < 4; ++k) hi[k] = cmul(hi[k], pre);
        }
    }
    // twiddle of output k of the first DFT: W256^(l k) (times W512^(h l) in the forward form)
    template <bool INV> __device__ __forceinline__ cpx<R> mul256(cpx<R> a, int k) const {
        const cpx<R> w = (k >> 2) == 0 ? lo[k & 3] : ((k & 3) == 0 ? hi[k >> 2] : cmul(lo[k & 3], hi[k >> 2]));
        return INV ? cmulc(a, w) : cmul(a, w);
    }
    __device__ __forceinline__ cpx<R> fwd_tw(cpx<R> a, int k) const {  // forward form, includes k = 0
        const cpx<R> w = (k & 3) == 0 ? hi[k >> 2] : cmul(lo[k & 3], hi[k >> 2]);
        return cmul(a, w);
    }
};

// Parity-split position of spectrum index k (0 <= k < 512) in a staging row, so
// that the lanes of a half-warp (one parity, consecutive k/2) hit consecutive words.
__device__ __forceinline__ int ppos(int k) { return ((k & 1) << 8) | (k >> 1); }
// and of column kx (0 <= kx <= 256) in the inverse passes' staging tile
__device__ __forceinline__ int kpos(int kx) { return (kx & 1) ? 129 + (kx >> 1) : (kx >> 1); }

// swizzled 16 x 16 tile of one half-warp: entry (row, col) at row*16 + (col ^ row)
__device__ __forceinline__ int swz(int row, int col) { return row * 16 + (col ^ row); }

// Forward pruned 512-point transform.  In: v[j] = x[l + 16 j] (both halves).
// Out: lane (h, k2) v[k1] = X[lambda + 32 k1].  buf: this warp's 512-entry tile.
// tw must hold the forward form (load_fwd).
template <typename R>
__device__ __forceinline__ void fwd512(cpx<R> (&v)[16], cpx<R> *buf, const LaneTw<R> &tw) {
    const int lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    cpx<R> *t = buf + h * 256;
    if (h) {
#pragma unroll
        for (int j = 1; j < 16; ++j) v[j] = cmul(v[j], w32c<R>(j));
    }
    dft16<R, false>(v);
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = tw.fwd_tw(v[k], k);
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 16; ++k) t[swz(l, k)] = v[k];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = t[swz(r, l)];
    dft16<R, false>(v);
}

// Inverse (tw in the inverse form, load_inv): in lane (h, k2) v[k1] = Y[lambda + 32 k1].  Out (unnormalised): every
// lane of both halves holds y[n] for n = l + 16 j with j in [8h, 8h + 8):
// out[jj] = y[l + 16 (8h + jj)], jj < 8.
template <typename R>
__device__ __forceinline__ void inv512(cpx<R> (&v)[16], cpx<R> *buf, const LaneTw<R> &tw, cpx<R> (&out)[8]) {
    const int lane = threadIdx.x & 31, h = lane >> 4, k2 = lane & 15;
    cpx<R> *t = buf + h * 256;
    dft16<R, true>(v);  // over k1 -> index l
#pragma unroll
    for (int l = 1; l < 16; ++l) v[l] = tw.template mul256<true>(v[l], l);
    __syncwarp();
#pragma unroll
    for (int l = 0; l < 16; ++l) t[swz(k2, l)] = v[l];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = t[swz(r, k2)];
    dft16<R, true>(v);  // over k2 -> j ; now v[j] = z_h[k2 + 16 j] (this lane's l = k2)
    // y[n] = z_0[n] + W512^-n z_1[n]
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        cpx<R> o;
        o.x = __shfl_xor_sync(0xffffffffu, v[j].x, 16);
        o.y = __shfl_xor_sync(0xffffffffu, v[j].y, 16);
        const bool mine = (j >> 3) == h;
        if (mine) {
            const cpx<R> z0 = h ? o : v[j];
            const cpx<R> z1 = h ? v[j] : o;
            const cpx<R> w = cmul(tw.pre, w32c<R>(j));  // W512^(l + 16 j)
            out[j & 7] = cadd(z0, cmulc(z1, w));
        }
    }
}

// ---------------------------------------------------------------------------
// TMA bulk copies and mbarriers

__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(s_addr(dst)),
        "l"(src), "r"(bytes), "r"(s_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(s_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait; returns false (and records an error) if the phase never completes.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err) {
    for (long long i = 0; i < kSpinLimit; ++i)
        if (mbar_test(bar, parity)) return true;
    if (err) atomicExch(err, GJ_ERR_TIMEOUT);
    return false;
}

// After a timed-out wait at item t_fail, wait (bounded) for the copies this warp
// issued and has not consumed (items t_fail .. t_fail + CSTAGES - 1) so that no
// bulk copy lands in shared memory after the CTA exits.
__device__ __forceinline__ void drain(uint64_t *bars, long long t_fail, long long t0, long long t1, int *err) {
    for (long long t = t_fail; t < t1 && t < t_fail + CSTAGES; ++t) {
        const int s = (int)((t - t0) % CSTAGES);
        const uint32_t par = (uint32_t)(((t - t0) / CSTAGES) & 1);
        mbar_wait(bars + s, par, err);
    }
}

// ---------------------------------------------------------------------------
// Segmentation of the flattened (field, kx, layer) sequence over the warps of a
// persistent grid: warp w takes [T w / Wt, T (w+1) / Wt).

__device__ __host__ __forceinline__ long long seg_warps(long long warps, long long T) { return warps < T ? warps : T; }
__device__ __host__ __forceinline__ long long seg_begin(long long w, long long T, long long Wt) { return (w * T) / Wt; }
// the warp whose segment contains item t
__device__ __host__ __forceinline__ long long seg_owner(long long t, long long T, long long Wt) {
    return ((t + 1) * Wt + T - 1) / T - 1;
}

template <typename R>
struct View2 {  // the two fields of a launch (field 1 unused in single-field launches)
    OpView<R> op[2];
    cpx<R> *P[2];   // [NC][slots][512] layer-sum partials
    int *cnt[2];    // [NC] arrival counters (zero between launches)
    int slots;      // partial slots per column
    int nfield;
    int *err;
};

// ---------------------------------------------------------------------------
// Row pass (x direction), real lines -> half spectra in the transposed layout.
// A CTA of NW warps runs FPW complex transforms per warp (FFTS = NW * FPW per CTA).
// Joint mode: transform f packs line (base + f) of field 0 (real part) and field 1
// (imaginary part); single mode: lines (base + 2f, base + 2f + 1) of field 0.
// lpl = lines per layer (ny for model lines, sy for data lines).

__device__ __forceinline__ void pair_lines(int joint, int base, int f, int nlines, int &la, int &lb, bool &ha,
                                           bool &hb) {
    if (joint) { la = lb = base + f; ha = hb = la < nlines; }
    else { la = base + 2 * f; lb = la + 1; ha = la < nlines; hb = lb < nlines; }
}

// Splits the staged spectra of FFTS transforms into the two real half spectra and
// writes them to out[r][kx][iy] (the transposed layout), iy fastest.
template <typename R, int FFTS>
__device__ __forceinline__ void write_half_spectra(const cpx<R> *tile, const View2<R> &V, int joint, int base,
                                                   int nlines, int lpl, int out_sel) {
    using C = cpx<R>;
    static_assert((FFTS & (FFTS - 1)) == 0, "FFTS must be a power of two");
    // blockDim is a multiple of FFTS, so this thread always serves transform f
    const int f = threadIdx.x % FFTS;
    int la, lb;
    bool ha, hb;
    pair_lines(joint, base, f, nlines, la, lb, ha, hb);
    const int fb = joint ? 1 : 0;
    const int ra = ha ? la / lpl : 0, rb = hb ? lb / lpl : 0;
    C *oa = (out_sel == 0 ? V.op[0].Z : (out_sel == 1 ? V.op[0].W : V.op[0].V)) + (size_t)ra * NC * H + (la - ra * lpl);
    C *ob = (out_sel == 0 ? V.op[fb].Z : (out_sel == 1 ? V.op[fb].W : V.op[fb].V)) + (size_t)rb * NC * H + (lb - rb * lpl);
    const C *row = tile + f * (N + 1);
    const int kstep = blockDim.x / FFTS;
    for (int kx = threadIdx.x / FFTS; kx < NC; kx += kstep) {
        const C zk = row[ppos(kx)];
        const C zm = row[ppos((N - kx) & (N - 1))];
        if (ha) oa[kx * H] = mk<C>(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y));
        if (hb) ob[kx * H] = mk<C>(R(0.5) * (zk.y + zm.y), R(-0.5) * (zk.x - zm.x));
    }
}

// Real input a + i b held as a[i], b[i] for elements lane + 32 i: redistribute
// through the warp tile and run the forward transform.  Result in v (lane layout).
template <typename R>
__device__ __forceinline__ void fwd512_from_lines(const R (&a)[8], const R (&b)[8], cpx<R> *buf, const LaneTw<R> &tw,
                                                  cpx<R> (&v)[16]) {
    using C = cpx<R>;
    const int lane = threadIdx.x & 31, l = lane & 15;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i) buf[lane + 32 * i] = mk<C>(a[i], b[i]);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = buf[l + 16 * j];
    fwd512<R>(v, buf, tw);
}

template <typename R, class Pro, int NW, int FPW>
__global__ void __launch_bounds__(NW * 32, 2) k_row_fwd512(View2<R> V, int joint, int nlines, int lpl, int n_in,
                                                           int out_sel, Pro pro, const int *done) {
    using C = cpx<R>;
    constexpr int FFTS = NW * FPW;
    if (stopped(done)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tile = reinterpret_cast<C *>(smem_raw);  // [FFTS][N + 1]
    C *xb = tile + FFTS * (N + 1);              // per warp 512
    C *tws = xb + NW * N;                       // W512 table
    __shared__ double red[128];
    pro.init();
    __syncthreads();
    LaneTw<R> tw;
    tw.load_fwd(V.op[0].twx);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    const int base = blockIdx.x * (joint ? FFTS : 2 * FFTS);
    C *buf = xb + warp * N;
    for (int s = 0; s < FPW; ++s) {
        const int f = warp * FPW + s;
        int la, lb;
        bool ha, hb;
        pair_lines(joint, base, f, nlines, la, lb, ha, hb);
        R a[8], b[8];
        if (ha) {
            // two batches of four keep the prologue's registers below the spill point
            R a0[4], b0[4], a1[4], b1[4];
            pro.template fetch_batch<4>(la, lb, hb, lane, 32, n_in, a0, b0);
            pro.template fetch_batch<4>(la, lb, hb, lane + 128, 32, n_in, a1, b1);
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = a0[i]; b[i] = b0[i]; a[4 + i] = a1[i]; b[4 + i] = b1[i]; }
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = b[i] = R(0);
        }
        C v[16];
        fwd512_from_lines<R>(a, b, buf, tw, v);
        const int lam = 2 * l + h;
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) tile[f * (N + 1) + ppos(lam + 32 * k1)] = v[k1];
    }
    __syncthreads();
    write_half_spectra<R, FFTS>(tile, V, joint, base, nlines, lpl, out_sel);
    pro.flush(red);
}

// Stages the half spectra of the CTA's lines: source column s < 2 FFTS holds
// (joint) field s / FFTS, line base + s % FFTS, or (single) line base + s.
template <typename R, int FFTS>
__device__ __forceinline__ void stage_half_spectra(cpx<R> *tile, const View2<R> &V, int joint, int base, int nlines,
                                                   int lpl, int in_sel) {
    using C = cpx<R>;
    constexpr int SRC = 2 * FFTS, P = SRC + 1;
    const int s = threadIdx.x % SRC;
    const int fld = joint ? (s / FFTS) : 0;
    const int line = joint ? base + (s % FFTS) : base + s;
    const bool ok = line < nlines;
    const int r = ok ? line / lpl : 0, iy = ok ? line - r * lpl : 0;
    const C *src = in_sel == 0 ? V.op[fld].Z : (in_sel == 1 ? V.op[fld].W : V.op[fld].V);
    const C *in = src + (size_t)r * NC * H + iy;
    const int kx0 = threadIdx.x / SRC, kstep = blockDim.x / SRC;
    for (int kb = kx0; kb < NC; kb += 8 * kstep) {
        C val[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int kx = kb + u * kstep;
            val[u] = (ok && kx < NC) ? in[(size_t)kx * H] : czero<C>();
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int kx = kb + u * kstep;
            if (kx < NC) tile[kpos(kx) * P + s] = val[u];
        }
    }
}

// Gathers transform f (sources sa, sb: Hermitian-extended A + i B) in the lane
// layout and runs the inverse transform; returns y[lane + 32 i] in a[i] + i b[i].
template <typename R, int FFTS>
__device__ __forceinline__ void inv512_to_lines(const cpx<R> *tile, int sa, int sb, cpx<R> *buf, const LaneTw<R> &tw,
                                                R (&a)[8], R (&b)[8]) {
    using C = cpx<R>;
    constexpr int P = 2 * FFTS + 1;
    const int lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    const int lam = 2 * l + h;
    C v[16];
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) {
        const int k = lam + 32 * k1;
        const bool lo = k <= H;
        const int kk = lo ? k : N - k;
        C A = tile[kpos(kk) * P + sa], B = tile[kpos(kk) * P + sb];
        if (kk == 0 || kk == H) { A.y = 0; B.y = 0; }
        v[k1] = lo ? mk<C>(A.x - B.y, A.y + B.x) : mk<C>(A.x + B.y, B.x - A.y);
    }
    C out[8];
    inv512<R>(v, buf, tw, out);
    __syncwarp();
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) buf[l + 16 * (8 * h + jj)] = out[jj];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const C y = buf[lane + 32 * i];
        a[i] = y.x;
        b[i] = y.y;
    }
}

// Inverse row pass: half spectra in[r][kx][iy] -> real lines, cropped to n_out,
// through the epilogue functor.
template <typename R, class Epi, int NW, int FPW>
__global__ void __launch_bounds__(NW * 32, 2) k_row_inv512(View2<R> V, int joint, int nlines, int lpl, int n_out,
                                                           int in_sel, Epi epi, const int *done) {
    using C = cpx<R>;
    constexpr int FFTS = NW * FPW;
    if (stopped(done)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tile = reinterpret_cast<C *>(smem_raw);  // [NC][2 FFTS + 1]
    C *xb = tile + NC * (2 * FFTS + 1);
    C *tws = xb + NW * N;
    __shared__ double red[128];
    epi.init();
    const int base = blockIdx.x * (joint ? FFTS : 2 * FFTS);
    stage_half_spectra<R, FFTS>(tile, V, joint, base, nlines, lpl, in_sel);
    __syncthreads();
    LaneTw<R> tw;
    tw.load_inv(V.op[0].twx);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C *buf = xb + warp * N;
    for (int s2 = 0; s2 < FPW; ++s2) {
        const int f = warp * FPW + s2;
        const int sa = joint ? f : 2 * f;
        const int sb = joint ? FFTS + f : 2 * f + 1;
        R a[8], b[8];
        inv512_to_lines<R, FFTS>(tile, sa, sb, buf, tw, a, b);
        int la, lb;
        bool ha, hb;
        pair_lines(joint, base, f, nlines, la, lb, ha, hb);
        if (ha) {
            R a0[4], b0[4], a1[4], b1[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a0[i] = a[i]; b0[i] = b[i]; a1[i] = a[4 + i]; b1[i] = b[4 + i]; }
            epi.template store_batch<4>(la, lb, hb, lane, 32, n_out, a0, b0);
            epi.template store_batch<4>(la, lb, hb, lane + 128, 32, n_out, a1, b1);
        }
    }
    epi.flush(red);
}

// ---------------------------------------------------------------------------
// Persistent joint row passes (both fields in one complex transform per line).
// A team of four warps takes a balanced contiguous range of the aligned four-line
// groups of the layers (warp k of the team transforms line 4q + k of group q), so
// that no launch ends in a partial wave.  The half spectra of a group sit in a
// double-buffered team tile stage[field][slot][kq(kx)] and move to or from the
// transposed layout out[r][kx][iy] as whole 32-byte sectors (four lines of one
// column).  kq puts even columns first and odd ones from 136 on; with the slot
// stride LS = 274 (2 mod 16), a half-warp's 16 consecutive columns of one line, and
// its 4 x 4 (column, slot) pairs of a group, each fall in 16 distinct bank pairs.
// One named barrier per group and team.  The rows the functor reads in every
// launch (m, p, l) are staged one line ahead with asynchronous copies.

constexpr int TEAM = 4;                 // warps per team = lines per group
constexpr int LS = 274, FS = TEAM * LS;  // slot and field strides of a team tile (complex words)

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() {  // at most NPEND of the newest groups still in flight
    asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory");
}
__device__ __forceinline__ void team_barrier(int team) {  // barrier 0 stays with __syncthreads
    asm volatile("bar.sync %0, %1;\n" ::"r"(1 + team), "r"(TEAM * 32) : "memory");
}

__device__ __forceinline__ int kq(int kx) { return (kx & 1) ? 136 + (kx >> 1) : (kx >> 1); }

// Z = FFT(a + i b) in the lane layout (v[k1] = Z[lambda + 32 k1]) -> the half
// spectra A = (Z[kx] + conj Z[N - kx]) / 2 and B = (Z[kx] - conj Z[N - kx]) / 2i,
// kx = 0..256, into slot g of a team tile.  For lambda != 0, Z[N - kx] sits in
// lane (h, 16 - l - h) at k1' = 15 - k1; lane 0 (lambda = 0) holds it at 16 - k1.
template <typename R>
__device__ __forceinline__ void split_to_stage(const cpx<R> (&v)[16], cpx<R> *stage, int g) {
    using C = cpx<R>;
    const int lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    const int partner = h ? 31 - l : ((16 - l) & 15);
    C *sa = stage + g * LS, *sb = sa + FS;
    const int q0 = h * 136 + l;  // kq(lambda + 32 k1) = q0 + 16 k1
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
        C zm;
        zm.x = __shfl_sync(0xffffffffu, v[15 - k1].x, partner);
        zm.y = __shfl_sync(0xffffffffu, v[15 - k1].y, partner);
        if (lane == 0) zm = v[(16 - k1) & 15];
        const C zk = v[k1];
        sa[q0 + 16 * k1] = mk<C>(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y));
        sb[q0 + 16 * k1] = mk<C>(R(0.5) * (zk.y + zm.y), R(-0.5) * (zk.x - zm.x));
    }
    if (lane == 0) {  // kx = 256 is its own partner
        sa[kq(H)] = mk<C>(v[8].x, R(0));
        sb[kq(H)] = mk<C>(v[8].y, R(0));
    }
}

// Slot g < ng of a team tile -> oa[kx * H + g], ob[kx * H + g]; the team's 128
// threads each take (g, kx) = (tid % 4, tid / 4 + 32 i).
template <typename R>
__device__ __forceinline__ void team_store(const cpx<R> *stage, cpx<R> *oa, cpx<R> *ob, int ng, int tid) {
    const int g = tid % TEAM;
    if (g >= ng) return;
    const cpx<R> *sa = stage + g * LS, *sb = sa + FS;
    for (int kx = tid / TEAM; kx < NC; kx += 32) {
        oa[(size_t)kx * H + g] = sa[kq(kx)];
        ob[(size_t)kx * H + g] = sb[kq(kx)];
    }
}

// ia[kx * H + g], ib[kx * H + g] -> slot g < ng of a team tile (asynchronous copies).
template <typename R>
__device__ __forceinline__ void team_load(cpx<R> *stage, const cpx<R> *ia, const cpx<R> *ib, int ng, int tid) {
    const int g = tid % TEAM;
    if (g >= ng) return;
    cpx<R> *sa = stage + g * LS, *sb = sa + FS;
    for (int kx = tid / TEAM; kx < NC; kx += 32) {
        cp_async8(sa + kq(kx), ia + (size_t)kx * H + g);
        cp_async8(sb + kq(kx), ib + (size_t)kx * H + g);
    }
}

// Slot g of a team tile (A + i B, Hermitian-extended) -> inverse transform ->
// y[lane + 32 i] in a[i] + i b[i].
template <typename R>
__device__ __forceinline__ void stage_to_lines(const cpx<R> *stage, int g, cpx<R> *buf, const LaneTw<R> &tw,
                                               R (&a)[8], R (&b)[8]) {
    using C = cpx<R>;
    const int lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    const int lam = 2 * l + h;
    const C *sa = stage + g * LS, *sb = sa + FS;
    C v[16];
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) {
        const int k = lam + 32 * k1;
        const bool lo = k <= H;
        const int kk = lo ? k : N - k;
        C A = sa[kq(kk)], B = sb[kq(kk)];
        if (kk == 0 || kk == H) { A.y = 0; B.y = 0; }
        v[k1] = lo ? mk<C>(A.x - B.y, A.y + B.x) : mk<C>(A.x + B.y, B.x - A.y);
    }
    C out[8];
    inv512<R>(v, buf, tw, out);
    __syncwarp();
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) buf[l + 16 * (8 * h + jj)] = out[jj];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const C y = buf[lane + 32 * i];
        a[i] = y.x;
        b[i] = y.y;
    }
}

// Stages the functor's rows of line t (n elements each) into pre[a][field][H]: 16-byte
// copies where the rows allow them, else 4-byte ones.  Does not commit.
template <typename R, class Fn>
__device__ __forceinline__ void prefetch_rows(const Fn &fn, R *pre, int t, int n) {
    constexpr int V4 = 16 / sizeof(R);
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int a = 0; a < Fn::NPRE; ++a)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const R *src = fn.pre_src(a, i);
            if (!src) continue;
            src += (size_t)t * n;
            R *dst = pre + (a * 2 + i) * H;
            if (n % V4 == 0 && ((uintptr_t)src & 15) == 0) {
                for (int q = lane; q < n / V4; q += 32) cp_async16(dst + q * V4, src + q * V4);
            } else {
                for (int j = lane; j < n; j += 32) cp_async4(dst + j, src + j);
            }
        }
}

template <typename R>
__device__ __forceinline__ cpx<R> *sel_buf(const OpView<R> &o, int sel) {  // 0 = Z, 1 = W, 2 = V
    return sel == 0 ? o.Z : (sel == 1 ? o.W : o.V);
}

// Shared memory of the persistent row passes (complex words): per team two tiles,
// per warp a transform buffer and the staged functor rows.
template <typename R, int NPRE>
constexpr int row_warp_words() {
    return N + (NPRE * 2 * H * (int)sizeof(R) + (int)sizeof(cpx<R>) - 1) / (int)sizeof(cpx<R>);
}
template <typename R, int NW, int NPRE>
constexpr int row_t_words() {
    return (NW / TEAM) * 2 * 2 * FS + NW * row_warp_words<R, NPRE>();
}

// Group q of a layer-major sequence (gpl groups per layer): layer, first line.
__device__ __forceinline__ void group_lines(int q, int gpl, int lpl, int &r, int &iy0, int &ng) {
    r = q / gpl;
    iy0 = (q - r * gpl) * TEAM;
    ng = min(TEAM, lpl - iy0);
}

// Forward joint row pass: line r lpl + iy of both fields (through the prologue
// functor) -> half spectra out[r][kx][iy].
template <typename R, class Pro, int NW>
__global__ void __launch_bounds__(NW * 32, 1) k_row_fwd512t(View2<R> V, int nz, int lpl, int n_in, int out_sel,
                                                            Pro pro, const int *done) {
    using C = cpx<R>;
    static_assert(NW % TEAM == 0, "whole teams");
    constexpr int NT = NW / TEAM;
    if (stopped(done)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int team = warp / TEAM, k = warp % TEAM, tid = threadIdx.x - team * TEAM * 32;
    C *tiles = reinterpret_cast<C *>(smem_raw) + (size_t)team * 2 * 2 * FS;
    C *buf = reinterpret_cast<C *>(smem_raw) + (size_t)NT * 2 * 2 * FS + (size_t)warp * row_warp_words<R, Pro::NPRE>();
    R *pre = reinterpret_cast<R *>(buf + N);
    __shared__ double red[128];
    pro.init();
    LaneTw<R> tw;
    tw.load_fwd(V.op[0].twx);
    const int gpl = (lpl + TEAM - 1) / TEAM;
    const long long NG = (long long)nz * gpl;
    const long long Tt = seg_warps((long long)gridDim.x * NT, NG);
    const long long tm = (long long)blockIdx.x * NT + team;
    if (tm < Tt) {
        const int q0 = (int)seg_begin(tm, NG, Tt), q1 = (int)seg_begin(tm + 1, NG, Tt);
        C *out0 = sel_buf(V.op[0], out_sel), *out1 = sel_buf(V.op[1], out_sel);
        int r, iy0, ng;
        group_lines(q0, gpl, lpl, r, iy0, ng);
        if (k < ng) prefetch_rows(pro, pre, r * lpl + iy0 + k, n_in);
        cp_async_commit();
        for (int q = q0; q < q1; ++q) {
            group_lines(q, gpl, lpl, r, iy0, ng);
            C *tile = tiles + (q & 1) * 2 * FS;
            const bool act = k < ng;  // this warp has a line in group q
            R a[8], b[8];
            if (act) {
                const int t = r * lpl + iy0 + k;
                cp_async_wait<0>();
                __syncwarp();
                R a0[4], b0[4], a1[4], b1[4];
                pro.template fetch_batch<4, true>(t, t, true, lane, 32, n_in, a0, b0, pre);
                pro.template fetch_batch<4, true>(t, t, true, lane + 128, 32, n_in, a1, b1, pre);
#pragma unroll
                for (int i = 0; i < 4; ++i) { a[i] = a0[i]; b[i] = b0[i]; a[4 + i] = a1[i]; b[4 + i] = b1[i]; }
                __syncwarp();
            }
            if (q + 1 < q1) {  // the rows of this warp's line in the next group
                int r2, iy2, ng2;
                group_lines(q + 1, gpl, lpl, r2, iy2, ng2);
                if (k < ng2) prefetch_rows(pro, pre, r2 * lpl + iy2 + k, n_in);
            }
            cp_async_commit();
            if (act) {
                C v[16];
                fwd512_from_lines<R>(a, b, buf, tw, v);
                split_to_stage<R>(v, tile, k);
            }
            team_barrier(team);  // the group's tile is complete; the other tile is free again
            const size_t off = (size_t)r * NC * H + iy0;
            team_store<R>(tile, out0 + off, out1 + off, ng, tid);
        }
    }
    pro.flush(red);
}

// Inverse joint row pass: half spectra in[r][kx][iy] -> line r lpl + iy of both
// fields, cropped to n_out, through the epilogue functor.  Copy groups in flight
// at the top of group q: [tile of q], [rows of q's line].
template <typename R, class Epi, int NW>
__global__ void __launch_bounds__(NW * 32, 1) k_row_inv512t(View2<R> V, int nz, int lpl, int n_out, int in_sel,
                                                            Epi epi, const int *done) {
    using C = cpx<R>;
    static_assert(NW % TEAM == 0, "whole teams");
    constexpr int NT = NW / TEAM;
    if (stopped(done)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int team = warp / TEAM, k = warp % TEAM, tid = threadIdx.x - team * TEAM * 32;
    C *tiles = reinterpret_cast<C *>(smem_raw) + (size_t)team * 2 * 2 * FS;
    C *buf = reinterpret_cast<C *>(smem_raw) + (size_t)NT * 2 * 2 * FS + (size_t)warp * row_warp_words<R, Epi::NPRE>();
    R *pre = reinterpret_cast<R *>(buf + N);
    __shared__ double red[128];
    epi.init();
    LaneTw<R> tw;
    tw.load_inv(V.op[0].twx);
    const int gpl = (lpl + TEAM - 1) / TEAM;
    const long long NG = (long long)nz * gpl;
    const long long Tt = seg_warps((long long)gridDim.x * NT, NG);
    const long long tm = (long long)blockIdx.x * NT + team;
    if (tm < Tt) {
        const int q0 = (int)seg_begin(tm, NG, Tt), q1 = (int)seg_begin(tm + 1, NG, Tt);
        const C *in0 = sel_buf(V.op[0], in_sel), *in1 = sel_buf(V.op[1], in_sel);
        int r, iy0, ng;
        group_lines(q0, gpl, lpl, r, iy0, ng);
        {
            const size_t off = (size_t)r * NC * H + iy0;
            team_load<R>(tiles + (q0 & 1) * 2 * FS, in0 + off, in1 + off, ng, tid);
            cp_async_commit();
            if (k < ng) prefetch_rows(epi, pre, r * lpl + iy0 + k, n_out);
            cp_async_commit();
        }
        for (int q = q0; q < q1; ++q) {
            group_lines(q, gpl, lpl, r, iy0, ng);
            cp_async_wait<1>();  // this thread's copies of the tile of q
            team_barrier(team);  // everyone's copies of q; the other tile is free again
            if (q + 1 < q1) {
                int r2, iy2, ng2;
                group_lines(q + 1, gpl, lpl, r2, iy2, ng2);
                const size_t off = (size_t)r2 * NC * H + iy2;
                team_load<R>(tiles + ((q + 1) & 1) * 2 * FS, in0 + off, in1 + off, ng2, tid);
            }
            cp_async_commit();
            if (k < ng) {
                const int t = r * lpl + iy0 + k;
                R a[8], b[8];
                stage_to_lines<R>(tiles + (q & 1) * 2 * FS, k, buf, tw, a, b);
                cp_async_wait<1>();  // the rows of line t
                __syncwarp();
                R a0[4], b0[4], a1[4], b1[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) { a0[i] = a[i]; b0[i] = b[i]; a1[i] = a[4 + i]; b1[i] = b[4 + i]; }
                epi.template store_batch<4, true>(t, t, true, lane, 32, n_out, a0, b0, pre);
                epi.template store_batch<4, true>(t, t, true, lane + 128, 32, n_out, a1, b1, pre);
                __syncwarp();
            }
            if (q + 1 < q1) {
                int r2, iy2, ng2;
                group_lines(q + 1, gpl, lpl, r2, iy2, ng2);
                if (k < ng2) prefetch_rows(epi, pre, r2 * lpl + iy2 + k, n_out);
            }
            cp_async_commit();
        }
    }
    epi.flush(red);
}

// Fused data-line pass of the solver: for station row jy of both fields, inverse
// row transform of W (the cropped forward product), the residual epilogue
// (r~ = W_d (A m - d), v = W_d r~, Phi partials), then the forward row transform
// of v written to V[kx][jy] for the adjoint's column pass.
template <typename R, class Epi, int NW>
__global__ void __launch_bounds__(NW * 32, 2) k_row_resid512(View2<R> V, int nlines, int n_out, Epi epi,
                                                             const int *done) {
    using C = cpx<R>;
    constexpr int FFTS = NW;  // one joint transform per warp
    if (stopped(done)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tile = reinterpret_cast<C *>(smem_raw);  // [NC][2 NW + 1], later [NW][N + 1]
    C *xb = tile + (NC * (2 * FFTS + 1) > FFTS * (N + 1) ? NC * (2 * FFTS + 1) : FFTS * (N + 1));
    C *tws = xb + NW * N;
    __shared__ double red[128];
    epi.init();
    const int base = blockIdx.x * FFTS;
    stage_half_spectra<R, FFTS>(tile, V, 1, base, nlines, nlines, 1);
    __syncthreads();
    LaneTw<R> tw;
    tw.load_inv(V.op[0].twx);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    C *buf = xb + warp * N;
    const int f = warp;
    R a[8], b[8];
    inv512_to_lines<R, FFTS>(tile, f, FFTS + f, buf, tw, a, b);
    tw.load_fwd(V.op[0].twx);
    const int line = base + f;
    const bool ok = line < nlines;
    if (ok) {
        epi.template resid_batch<8>(line, lane, 32, n_out, a, b);  // a, b <- v of both fields
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = b[i] = R(0);
    }
    C v[16];
    fwd512_from_lines<R>(a, b, buf, tw, v);
    __syncthreads();  // every warp is done reading the staged input
    const int lam = 2 * l + h;
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) tile[f * (N + 1) + ppos(lam + 32 * k1)] = v[k1];
    __syncthreads();
    write_half_spectra<R, FFTS>(tile, V, 1, base, nlines, nlines, 2);
    epi.flush(red);
}

// ---------------------------------------------------------------------------
// Item t = (field NC + kx) nz + r of the column passes, set once by division and
// then advanced by increments.
struct ColItem {
    int fld, kx, r;
    __device__ __forceinline__ void set(int t, int nz) {
        const int col = t / nz;
        r = t - col * nz;
        fld = col / NC;
        kx = col - fld * NC;
    }
    __device__ __forceinline__ void next(int nz) {
        if (++r == nz) {
            r = 0;
            if (++kx == NC) { kx = 0; ++fld; }
        }
    }
};

// Forward column pass: for each (field, kx), Y = sum_r St_r[kx] . FFT512(Zt_r[kx]),
// then W[kx][jy] = IFFT512(Y)[jy] for jy < sy.  Persistent warps take balanced
// contiguous segments of the (field, kx, r) sequence; a column split across warps
// is summed in segment order by the last warp to finish it.
template <typename R>
__global__ void __launch_bounds__(CWARPS * 32, 1) k_col_fwd512(View2<R> V, const int *done) {
    using C = cpx<R>;
    if (stopped(done)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int ZB = H * sizeof(C), TB = N * sizeof(C);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    unsigned char *wbase = smem_raw + (size_t)warp * (CSTAGES * (ZB + TB) + N * sizeof(C));
    C *zs = reinterpret_cast<C *>(wbase);                          // CSTAGES x 256
    C *ts = reinterpret_cast<C *>(wbase + CSTAGES * ZB);            // CSTAGES x 512
    C *xbuf = reinterpret_cast<C *>(wbase + CSTAGES * (ZB + TB));   // 512
    __shared__ __align__(8) uint64_t bars[CWARPS][CSTAGES];
    if (lane == 0)
        for (int s = 0; s < CSTAGES; ++s) mbar_init(&bars[warp][s]);
    mbar_fence_init();
    __syncthreads();
    LaneTw<R> tw;
    tw.load_fwd(V.op[0].twy);
    const int nz = V.op[0].nz, sy = V.op[0].sy;
    const long long T = (long long)V.nfield * NC * nz;
    // at most T warps take part, so that every segment holds at least one item
    const long long Wt = seg_warps((long long)gridDim.x * CWARPS, T);
    const long long w = (long long)blockIdx.x * CWARPS + warp;
    if (w >= Wt) return;
    const int t0 = (int)seg_begin(w, T, Wt), t1 = (int)seg_begin(w + 1, T, Wt);
    const int lam = 2 * l + h;
    ColItem cu, ci;  // the item being consumed; (lane 0) the next one to issue
    cu.set(t0, nz);
    ci = cu;
    int ti = t0;
    auto issue = [&]() {  // item ti into stage (ti - t0) % CSTAGES
        const int s = (ti - t0) % CSTAGES;
        const OpView<R> &op = V.op[ci.fld];
        const size_t off = (size_t)ci.r * NC + ci.kx;
        if (op.real_spec) {
            mbar_expect(&bars[warp][s], ZB + TB / 2);
            bulk_load(zs + s * H, op.Z + off * H, ZB, &bars[warp][s]);
            bulk_load(ts + s * N, reinterpret_cast<const R *>(op.spec) + off * N, TB / 2, &bars[warp][s]);
        } else {
            mbar_expect(&bars[warp][s], ZB + TB);
            bulk_load(zs + s * H, op.Z + off * H, ZB, &bars[warp][s]);
            bulk_load(ts + s * N, op.spec + off * N, TB, &bars[warp][s]);
        }
        ++ti;
        ci.next(nz);
    };
    if (lane == 0)
        while (ti < t1 && ti < t0 + CSTAGES) issue();
    C acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = czero<C>();
    bool ok = true;
    int t_fail = t1;
    int seg_start = t0;
    for (int t = t0; t < t1 && ok; ++t, cu.next(nz)) {
        const int s = (t - t0) % CSTAGES;
        const uint32_t par = (uint32_t)(((t - t0) / CSTAGES) & 1);
        ok = __all_sync(0xffffffffu, mbar_wait(&bars[warp][s], par, V.err));
        if (!ok) { t_fail = t; break; }
        C v[16];
        const bool real_t = V.op[cu.fld].real_spec;
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = zs[s * H + l + 16 * j];
        fwd512<R>(v, xbuf, tw);
        // multiply by the layer's spectrum straight from the stage, then release it
        if (real_t) {
            const R *tr = reinterpret_cast<const R *>(ts + s * N);
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {
                const R tt = tr[lam + 32 * k1];
                acc[k1] = mk<C>(acc[k1].x + v[k1].x * tt, acc[k1].y + v[k1].y * tt);
            }
        } else {
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) acc[k1] = cadd(acc[k1], cmul(v[k1], ts[s * N + lam + 32 * k1]));
        }
        __syncwarp();
        if (lane == 0 && ti < t1) issue();
        if (cu.r == nz - 1 || t == t1 - 1) {
            // end of this warp's part of column `col`
            const int fld = cu.fld, kx = cu.kx;
            const long long col = (long long)fld * NC + kx;
            const OpView<R> &op = V.op[fld];
            const long long cb = col * nz, ce = cb + nz - 1;
            const bool whole = (seg_start <= cb) && (t == ce);
            if (!whole) {
                const long long wf = seg_owner(cb, T, Wt), wl = seg_owner(ce, T, Wt);
                const int slot = (int)(w - wf), nslots = (int)(wl - wf + 1);
                C *Pc = V.P[fld] + (size_t)kx * V.slots * N;
#pragma unroll
                for (int k1 = 0; k1 < 16; ++k1) Pc[(size_t)slot * N + lam + 32 * k1] = acc[k1];
                __threadfence();
                __syncwarp();
                int old = 0;
                if (lane == 0) old = atomicAdd(V.cnt[fld] + kx, 1);
                old = __shfl_sync(0xffffffffu, old, 0);
                if (old == nslots - 1) {
                    __threadfence();
#pragma unroll
                    for (int k1 = 0; k1 < 16; ++k1) acc[k1] = czero<C>();
                    for (int sl = 0; sl < nslots; ++sl) {
#pragma unroll
                        for (int k1 = 0; k1 < 16; ++k1)
                            acc[k1] = cadd(acc[k1], __ldcg(Pc + (size_t)sl * N + lam + 32 * k1));
                    }
                    if (lane == 0) V.cnt[fld][kx] = 0;
                } else {
#pragma unroll
                    for (int k1 = 0; k1 < 16; ++k1) acc[k1] = czero<C>();
                    seg_start = t + 1;
                    continue;
                }
            }
            C out[8];
            tw.load_inv(V.op[0].twy);
            inv512<R>(acc, xbuf, tw, out);
            tw.load_fwd(V.op[0].twy);
            C *Wc = op.W + (size_t)kx * H;
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                const int n = l + 16 * (8 * h + jj);
                if (n < sy) Wc[n] = out[jj];
            }
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) acc[k1] = czero<C>();
            seg_start = t + 1;
        }
    }
    if (!ok) drain(bars[warp], t_fail, t0, t1, V.err);
}

// ---------------------------------------------------------------------------
// Adjoint column pass: for each (field, kx, r),
// Zt_r[kx][iy] = IFFT512(conj(St_r[kx]) . FFT512(Wt[kx]))[iy], iy < ny.
template <typename R>
__global__ void __launch_bounds__(CWARPS * 32, 1) k_col_adj512(View2<R> V, const int *done) {
    using C = cpx<R>;
    if (stopped(done)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TB = N * sizeof(C);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    unsigned char *wbase = smem_raw + (size_t)warp * (CSTAGES * TB + N * sizeof(C));
    C *ts = reinterpret_cast<C *>(wbase);
    C *xbuf = reinterpret_cast<C *>(wbase + CSTAGES * TB);
    __shared__ __align__(8) uint64_t bars[CWARPS][CSTAGES];
    if (lane == 0)
        for (int s = 0; s < CSTAGES; ++s) mbar_init(&bars[warp][s]);
    mbar_fence_init();
    __syncthreads();
    LaneTw<R> tw;
    tw.load_inv(V.op[0].twy);
    const int nz = V.op[0].nz, ny = V.op[0].ny;
    const long long T = (long long)V.nfield * NC * nz;
    // at most T warps take part, so that every segment holds at least one item
    const long long Wt = seg_warps((long long)gridDim.x * CWARPS, T);
    const long long w = (long long)blockIdx.x * CWARPS + warp;
    if (w >= Wt) return;
    const int t0 = (int)seg_begin(w, T, Wt), t1 = (int)seg_begin(w + 1, T, Wt);
    const int lam = 2 * l + h;
    ColItem cu, ci;  // the item being consumed; (lane 0) the next one to issue
    cu.set(t0, nz);
    ci = cu;
    int ti = t0;
    auto issue = [&]() {  // item ti into stage (ti - t0) % CSTAGES
        const int s = (ti - t0) % CSTAGES;
        const size_t off = (size_t)ci.r * NC + ci.kx;
        if (V.op[ci.fld].real_spec) {
            mbar_expect(&bars[warp][s], TB / 2);
            bulk_load(ts + s * N, reinterpret_cast<const R *>(V.op[ci.fld].spec) + off * N, TB / 2, &bars[warp][s]);
        } else {
            mbar_expect(&bars[warp][s], TB);
            bulk_load(ts + s * N, V.op[ci.fld].spec + off * N, TB, &bars[warp][s]);
        }
        ++ti;
        ci.next(nz);
    };
    if (lane == 0)
        while (ti < t1 && ti < t0 + CSTAGES) issue();
    C vh[16];
    bool ok = true;
    int t_fail = t1;
    for (int t = t0; t < t1 && ok; ++t, cu.next(nz)) {
        const int r = cu.r, fld = cu.fld, kx = cu.kx;
        const OpView<R> &op = V.op[fld];
        if (t == t0 || r == 0) {  // a new column
            // V^ = FFT512 of the residual column (rows >= sy are zero)
            const C *Wc = op.V + (size_t)kx * H;
#pragma unroll
            for (int j = 0; j < 16; ++j) vh[j] = Wc[l + 16 * j];
            tw.load_fwd(V.op[0].twy);
            fwd512<R>(vh, xbuf, tw);
            tw.load_inv(V.op[0].twy);
        }
        const int s = (t - t0) % CSTAGES;
        const uint32_t par = (uint32_t)(((t - t0) / CSTAGES) & 1);
        ok = __all_sync(0xffffffffu, mbar_wait(&bars[warp][s], par, V.err));
        if (!ok) { t_fail = t; break; }
        C v[16];
        if (op.real_spec) {
            const R *tr = reinterpret_cast<const R *>(ts + s * N);
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {
                const R tt = tr[lam + 32 * k1];
                v[k1] = mk<C>(vh[k1].x * tt, vh[k1].y * tt);
            }
        } else {
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) v[k1] = cmulc(vh[k1], ts[s * N + lam + 32 * k1]);
        }
        __syncwarp();
        if (lane == 0 && ti < t1) issue();
        C out[8];
        inv512<R>(v, xbuf, tw, out);
        C *Zc = op.Z + ((size_t)r * NC + kx) * H;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            const int n = l + 16 * (8 * h + jj);
            if (n < ny) Zc[n] = out[jj];
        }
    }
    if (!ok) drain(bars[warp], t_fail, t0, t1, V.err);
}

// shared-memory bytes of each kernel
template <typename R, int NW, int FPW> inline size_t smem_row_fwd() {
    return (size_t)(NW * FPW * (N + 1) + NW * N + N) * sizeof(cpx<R>);
}
template <typename R, int NW, int FPW> inline size_t smem_row_inv() {
    return (size_t)(NC * (2 * NW * FPW + 1) + NW * N + N) * sizeof(cpx<R>);
}
template <typename R, int NW> inline size_t smem_row_resid() {
    const size_t t = (size_t)NC * (2 * NW + 1) > (size_t)NW * (N + 1) ? (size_t)NC * (2 * NW + 1) : (size_t)NW * (N + 1);
    return (t + NW * N + N) * sizeof(cpx<R>);
}
template <typename R, int NW, int NPRE> inline size_t smem_row_t() {
    return (size_t)row_t_words<R, NW, NPRE>() * sizeof(cpx<R>);
}
template <typename R> inline size_t smem_col_fwd() {
    return (size_t)CWARPS * (CSTAGES * (H + N) + N) * sizeof(cpx<R>);
}
template <typename R> inline size_t smem_col_adj() {
    return (size_t)CWARPS * (CSTAGES * N + N) * sizeof(cpx<R>);
}

}  // namespace f512
}  // namespace gj
