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
// Bounded mbarrier waits give up after this long (read from %globaltimer, checked
// every eight polls), record GJ_ERR_TIMEOUT in the operator's error word and
// let the kernel return; a healthy 2-4 KB bulk copy completes in microseconds.
constexpr unsigned long long kWaitLimitNs = 200ull * 1000ull * 1000ull;

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
    // combine twiddle of the inverse, W512^(l + 16 j) (j known at compile time)
    __device__ __forceinline__ cpx<R> cmb(int j) const { return cmul(pre, w32c<R>(j)); }
};

// The same twiddles read from a per-CTA shared-memory table (no per-lane products,
// no twiddle registers), rows of 32 lanes (h, l):
//   [k < 16]       forward W512^(h l + 2 l k)  (fwd_tw)
//   [16 + k]       inverse W256^(l k) = W512^(2 l k)  (mul256)
//   [32 + jj < 40] combine W512^(l + 16 (8 h + jj))  (cmb)
// The entries are the operator's W512 table itself, so they carry no product rounding.
template <typename R>
struct TabTw {
    static constexpr int WORDS = 40 * 32;
    const cpx<R> *t;  // shared
    int lane;
    // every thread of the CTA, followed by a barrier before first use
    __device__ static void build(cpx<R> *t, const cpx<R> *__restrict__ tw512) {
        for (int i = threadIdx.x; i < WORDS; i += blockDim.x) {
            const int row = i >> 5, ln = i & 31, h = ln >> 4, l = ln & 15;
            const int e = row < 16 ? h * l + 2 * l * row : (row < 32 ? 2 * l * (row - 16) : l + 16 * (8 * h + row - 32));
            t[i] = __ldg(tw512 + (e & 511));
        }
    }
    __device__ void bind(const cpx<R> *tab) { t = tab; lane = threadIdx.x & 31; }
    template <bool INV> __device__ __forceinline__ cpx<R> mul256(cpx<R> a, int k) const {
        const cpx<R> w = t[(16 + k) * 32 + lane];
        return INV ? cmulc(a, w) : cmul(a, w);
    }
    __device__ __forceinline__ cpx<R> fwd_tw(cpx<R> a, int k) const { return cmul(a, t[k * 32 + lane]); }
    __device__ __forceinline__ cpx<R> cmb(int j) const { return t[(32 + (j & 7)) * 32 + lane]; }
};

// Parity-split position of spectrum index k (0 <= k < 512) in a staging row, so
// that the lanes of a half-warp (one parity, consecutive k/2) hit consecutive words.
__device__ __forceinline__ int ppos(int k) { return ((k & 1) << 8) | (k >> 1); }
// and of column kx (0 <= kx <= 256) in the inverse passes' staging tile
__device__ __forceinline__ int kpos(int kx) { return (kx & 1) ? 129 + (kx >> 1) : (kx >> 1); }

// Real, even spectra (the gravity table over stations that cover the prisms) keep
// ky <= N/2 only: KE values per column (a multiple of four, so that columns start on
// 16 bytes).  Spectrum index ky = lambda + 32 k1 of the 512 transform's lane layout
// reads entry min(ky, 512 - ky), which k1 (a compile-time index) decides.
constexpr int KE = even_spec_len(N), KEB = KE * (int)sizeof(float);  // FP32, the fast path's precision
__device__ __forceinline__ int even_pos512(int lam, int k1) { return k1 < 8 ? lam + 32 * k1 : N - 32 * k1 - lam; }

// swizzled 16 x 16 tile of one half-warp: entry (row, col) at row*16 + (col ^ row)
__device__ __forceinline__ int swz(int row, int col) { return row * 16 + (col ^ row); }

// Forward pruned 512-point transform.  In: v[j] = x[l + 16 j] (both halves).
// Out: lane (h, k2) v[k1] = X[lambda + 32 k1].  buf: this warp's 512-entry tile.
// tw: LaneTw in the forward form (load_fwd), or TabTw.
template <typename R, class TW>
__device__ __forceinline__ void fwd512(cpx<R> (&v)[16], cpx<R> *buf, const TW &tw) {
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
template <typename R, class TW>
__device__ __forceinline__ void inv512(cpx<R> (&v)[16], cpx<R> *buf, const TW &tw, cpx<R> (&out)[8]) {
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
            const cpx<R> w = tw.cmb(j);  // W512^(l + 16 j)
            out[j & 7] = cadd(z0, cmulc(z1, w));
        }
    }
}

// ---------------------------------------------------------------------------
// TMA bulk copies and mbarriers

__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// asynchronous global -> shared copies (cp.async), completed per thread by groups
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
// The same copy with an L2 policy (createpolicy): the column passes read each layer
// spectrum once per product, so its lines go first when L2 needs room and the
// row passes' intermediates stay longer.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void bulk_load_hint(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                               uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            s_addr(dst)),
        "l"(src), "r"(bytes), "r"(s_addr(bar)), "l"(pol)
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
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: returns false (and records GJ_ERR_TIMEOUT in *err) if the phase
// has not completed limit_ns after the first poll.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err,
                                          unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
#pragma unroll 1
        for (int i = 0; i < 8; ++i)
            if (mbar_test(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) break;
    }
    if (err) atomicExch(err, GJ_ERR_TIMEOUT);
    return false;
}

// An operator whose column kernel gave up on a wait is unusable until the error
// is read and cleared (gj_op_status): its layer-sum counters may be off, so every
// fast-path kernel of it returns at once while the error word is set.
__device__ __forceinline__ bool op_failed(const int *err) {
    return err != nullptr && *(volatile const int *)err != 0;
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
// Segmentation of the flattened (kx, field, layer) sequence over the warps of a
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
    const cpx<R> *twtab;  // the column kernels' twiddle table (TabTw layout), built once per operator
    int hy;               // column stride of Zt, Wt and Vt: Ny / 2 (256 or 128)
};

// Every CTA of a column kernel copies the operator's twiddle table into shared
// memory with one bulk copy (thread 0, barrier `bar`), issued before the first
// items' copies so that both arrive together.
template <typename R>
__device__ __forceinline__ void load_twtab(cpx<R> *tab, const cpx<R> *src, uint64_t *bar) {
    if (threadIdx.x == 0) {
        mbar_expect(bar, TabTw<R>::WORDS * sizeof(cpx<R>));
        bulk_load(tab, src, TabTw<R>::WORDS * sizeof(cpx<R>), bar);
    }
}

// Fills the table once (one block; setup).
template <typename R>
__global__ void k_build_twtab(cpx<R> *tab, const cpx<R> *tw512) {
    TabTw<R>::build(tab, tw512);
}

// ---------------------------------------------------------------------------
// Item t = col nz + r of the column passes, column col = kx nf + fld: the fields
// alternate column by column, so every warp's segment mixes the cheaper gravity
// columns (real spectrum) with the magnetic ones.  Set once by division, then
// advanced by increments.
struct ColItem {
    int fld, kx, r, col;
    __device__ __forceinline__ void set(int t, int nz, int nf) {
        col = t / nz;
        r = t - col * nz;
        kx = col / nf;
        fld = col - kx * nf;
    }
    __device__ __forceinline__ void next(int nz, int nf) {
        if (++r == nz) {
            r = 0;
            ++col;
            if (++fld == nf) { fld = 0; ++kx; }
        }
    }
};

// Forward column pass: for each (field, kx), Y = sum_r St_r[kx] . FFT512(Zt_r[kx]),
// then W[kx][jy] = IFFT512(Y)[jy] for jy < sy.  Persistent warps take balanced
// contiguous segments of the (kx, field, r) sequence; a column split across warps
// is summed in segment order by the last warp to finish it.
template <typename R>
__global__ void __launch_bounds__(CWARPS * 32, 1) k_col_fwd512(View2<R> V, const int *done) {
    using C = cpx<R>;
    if (stopped(done) || op_failed(V.err)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int ZB = H * sizeof(C), TB = N * sizeof(C);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    unsigned char *wbase = smem_raw + (size_t)warp * (CSTAGES * (ZB + TB) + N * sizeof(C));
    C *zs = reinterpret_cast<C *>(wbase);                          // CSTAGES x 256
    C *ts = reinterpret_cast<C *>(wbase + CSTAGES * ZB);            // CSTAGES x 512
    C *xbuf = reinterpret_cast<C *>(wbase + CSTAGES * (ZB + TB));   // 512
    C *tab = reinterpret_cast<C *>(smem_raw + (size_t)CWARPS * (CSTAGES * (ZB + TB) + N * sizeof(C)));
    __shared__ __align__(8) uint64_t bars[CWARPS][CSTAGES];
    __shared__ __align__(8) uint64_t tabbar;
    if (lane == 0)
        for (int s = 0; s < CSTAGES; ++s) mbar_init(&bars[warp][s]);
    if (threadIdx.x == 0) mbar_init(&tabbar);
    mbar_fence_init();
    __syncthreads();
    TabTw<R> tw;
    tw.bind(tab);
    const int nz = V.op[0].nz, sy = V.op[0].sy;
    const long long T = (long long)V.nfield * NC * nz;
    // at most T warps take part, so that every segment holds at least one item
    const long long Wt = seg_warps((long long)gridDim.x * CWARPS, T);
    const long long w = (long long)blockIdx.x * CWARPS + warp;
    // a CTA with work fetches the table; its warp 0 has work and waits for the copy,
    // so the CTA outlives it
    if ((long long)blockIdx.x * CWARPS < Wt) load_twtab<R>(tab, V.twtab, &tabbar);
    if (w >= Wt) return;
    const int t0 = (int)seg_begin(w, T, Wt), t1 = (int)seg_begin(w + 1, T, Wt);
    const int lam = 2 * l + h;
    ColItem cu, ci;  // the item being consumed; (lane 0) the next one to issue
    cu.set(t0, nz, V.nfield);
    ci = cu;
    int ti = t0;
    const uint64_t pol = l2_evict_first();
    auto issue = [&]() {  // item ti into stage (ti - t0) % CSTAGES
        const int s = (ti - t0) % CSTAGES;
        const OpView<R> &op = V.op[ci.fld];
        const size_t off = (size_t)ci.r * NC + ci.kx;
        if (op.real_spec) {
            mbar_expect(&bars[warp][s], ZB + KEB);
            bulk_load(zs + s * H, op.Z + off * H, ZB, &bars[warp][s]);
            bulk_load_hint(ts + s * N, reinterpret_cast<const R *>(op.spec) + off * KE, KEB, &bars[warp][s], pol);
        } else {
            mbar_expect(&bars[warp][s], ZB + TB);
            bulk_load(zs + s * H, op.Z + off * H, ZB, &bars[warp][s]);
            bulk_load_hint(ts + s * N, op.spec + off * N, TB, &bars[warp][s], pol);
        }
        ++ti;
        ci.next(nz, V.nfield);
    };
    if (lane == 0)
        while (ti < t1 && ti < t0 + CSTAGES) issue();
    C acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = czero<C>();
    bool ok = __all_sync(0xffffffffu, mbar_wait(&tabbar, 0, V.err));
    int t_fail = ok ? t1 : t0;
    int seg_start = t0;
    for (int t = t0; t < t1 && ok; ++t, cu.next(nz, V.nfield)) {
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
                const R tt = tr[even_pos512(lam, k1)];
                acc[k1] = mk<C>(acc[k1].x + v[k1].x * tt, acc[k1].y + v[k1].y * tt);
            }
        } else {
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {  // acc += v * t, four fused multiply-adds
                const C t = ts[s * N + lam + 32 * k1];
                acc[k1].x = fma(v[k1].x, t.x, acc[k1].x);
                acc[k1].x = fma(-v[k1].y, t.y, acc[k1].x);
                acc[k1].y = fma(v[k1].x, t.y, acc[k1].y);
                acc[k1].y = fma(v[k1].y, t.x, acc[k1].y);
            }
        }
        __syncwarp();
        if (lane == 0 && ti < t1) issue();
        if (cu.r == nz - 1 || t == t1 - 1) {
            // end of this warp's part of column `col`
            const int fld = cu.fld, kx = cu.kx;
            const long long col = cu.col;
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
            inv512<R>(acc, xbuf, tw, out);
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
    if (stopped(done) || op_failed(V.err)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TB = N * sizeof(C);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    unsigned char *wbase = smem_raw + (size_t)warp * (CSTAGES * TB + N * sizeof(C));
    C *ts = reinterpret_cast<C *>(wbase);
    C *xbuf = reinterpret_cast<C *>(wbase + CSTAGES * TB);
    C *tab = reinterpret_cast<C *>(smem_raw + (size_t)CWARPS * (CSTAGES * TB + N * sizeof(C)));
    __shared__ __align__(8) uint64_t bars[CWARPS][CSTAGES];
    __shared__ __align__(8) uint64_t tabbar;
    if (lane == 0)
        for (int s = 0; s < CSTAGES; ++s) mbar_init(&bars[warp][s]);
    if (threadIdx.x == 0) mbar_init(&tabbar);
    mbar_fence_init();
    __syncthreads();
    TabTw<R> tw;
    tw.bind(tab);
    const int nz = V.op[0].nz, ny = V.op[0].ny;
    const long long T = (long long)V.nfield * NC * nz;
    // at most T warps take part, so that every segment holds at least one item
    const long long Wt = seg_warps((long long)gridDim.x * CWARPS, T);
    const long long w = (long long)blockIdx.x * CWARPS + warp;
    // a CTA with work fetches the table; its warp 0 has work and waits for the copy,
    // so the CTA outlives it
    if ((long long)blockIdx.x * CWARPS < Wt) load_twtab<R>(tab, V.twtab, &tabbar);
    if (w >= Wt) return;
    const int t0 = (int)seg_begin(w, T, Wt), t1 = (int)seg_begin(w + 1, T, Wt);
    const int lam = 2 * l + h;
    ColItem cu, ci;  // the item being consumed; (lane 0) the next one to issue
    cu.set(t0, nz, V.nfield);
    ci = cu;
    int ti = t0;
    const uint64_t pol = l2_evict_first();
    auto issue = [&]() {  // item ti into stage (ti - t0) % CSTAGES
        const int s = (ti - t0) % CSTAGES;
        const size_t off = (size_t)ci.r * NC + ci.kx;
        if (V.op[ci.fld].real_spec) {
            mbar_expect(&bars[warp][s], KEB);
            bulk_load_hint(ts + s * N, reinterpret_cast<const R *>(V.op[ci.fld].spec) + off * KE, KEB, &bars[warp][s],
                           pol);
        } else {
            mbar_expect(&bars[warp][s], TB);
            bulk_load_hint(ts + s * N, V.op[ci.fld].spec + off * N, TB, &bars[warp][s], pol);
        }
        ++ti;
        ci.next(nz, V.nfield);
    };
    if (lane == 0)
        while (ti < t1 && ti < t0 + CSTAGES) issue();
    C vh[16];
    bool ok = __all_sync(0xffffffffu, mbar_wait(&tabbar, 0, V.err));
    int t_fail = ok ? t1 : t0;
    for (int t = t0; t < t1 && ok; ++t, cu.next(nz, V.nfield)) {
        const int r = cu.r, fld = cu.fld, kx = cu.kx;
        const OpView<R> &op = V.op[fld];
        if (t == t0 || r == 0) {  // a new column
            // V^ = FFT512 of the residual column (rows >= sy are zero)
            const C *Wc = op.V + (size_t)kx * H;
#pragma unroll
            for (int j = 0; j < 16; ++j) vh[j] = Wc[l + 16 * j];
            fwd512<R>(vh, xbuf, tw);
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
                const R tt = tr[even_pos512(lam, k1)];
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

// ---------------------------------------------------------------------------
// Column passes of the 256-row embedding (N_y = 256, at most 128 prisms and 128
// stations per column; the rows keep N_x = 512).  Each half-warp runs a pruned
// 256-point transform of its own (inputs n < 128, the rest zero) on the 16 x 16
// steps of the 512 transform without the parity split: lane (h, l) holds
// x_h[l + 16 j], and after the second 16-point DFT lane (h, k2) holds
// X_h[k2 + 16 k1] in register k1.  The two half-warps take two layers of the same
// column, so an item is a layer pair (2 rp, 2 rp + 1) and the register, stage and
// transpose footprint equals the 512 kernels'.  Layouts: Zt[r][kx][iy < 128],
// St[r][kx][ky < 256], Wt/Vt[kx][jy < 128].

constexpr int N2 = 256, H2 = 128;
// even spectra at N_y = 256: ky <= 128 kept; index ky = l + 16 k1 reads min(ky, 256 - ky)
constexpr int KE2 = even_spec_len(N2), KEB2 = KE2 * (int)sizeof(float);
__device__ __forceinline__ int even_pos256(int l, int k1) { return k1 < 8 ? l + 16 * k1 : N2 - 16 * k1 - l; }

// Forward pruned 256-point transform of this half-warp's column.  In: v[j] =
// x[l + 16 j] for j < 8 (v[8..15] ignored, taken as zero).  Out: v[k1] = X[k2 + 16 k1].
template <typename R, class TW>
__device__ __forceinline__ void fwd256h(cpx<R> (&v)[16], cpx<R> *buf, const TW &tw) {
    const int lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    cpx<R> *t = buf + h * 256;
#pragma unroll
    for (int j = 8; j < 16; ++j) v[j] = czero<cpx<R>>();
    dft16<R, false>(v);  // over j -> index a; the zero half folds away
#pragma unroll
    for (int k = 1; k < 16; ++k) v[k] = tw.template mul256<false>(v[k], k);  // W256^(l a)
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 16; ++k) t[swz(l, k)] = v[k];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = t[swz(r, l)];
    dft16<R, false>(v);  // over l -> index b: X[a + 16 b], a = this lane's l
}

// Inverse 256-point transform of this half-warp's column (unnormalised).
// In: v[k1] = Y[k2 + 16 k1].  Out: v[j] = y[l + 16 j], j < 16.
template <typename R, class TW>
__device__ __forceinline__ void inv256h(cpx<R> (&v)[16], cpx<R> *buf, const TW &tw) {
    const int lane = threadIdx.x & 31, h = lane >> 4, k2 = lane & 15;
    cpx<R> *t = buf + h * 256;
    dft16<R, true>(v);  // over k1 -> index l
#pragma unroll
    for (int l = 1; l < 16; ++l) v[l] = tw.template mul256<true>(v[l], l);  // W256^-(l k2)
    __syncwarp();
#pragma unroll
    for (int l = 0; l < 16; ++l) t[swz(k2, l)] = v[l];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = t[swz(r, k2)];
    dft16<R, true>(v);  // over k2 -> index j
}

// Forward column pass, N_y = 256: for each (field, kx), Y = sum_r St_r[kx] . FFT256(Zt_r[kx]),
// then W[kx][jy] = IFFT256(Y)[jy] for jy < sy.  Items are (kx, field, layer pair) in
// the order of k_col_fwd512; the two half-warps' sums meet at the end of a column.
template <typename R>
__global__ void __launch_bounds__(CWARPS * 32, 1) k_col_fwd256(View2<R> V, const int *done) {
    using C = cpx<R>;
    if (stopped(done) || op_failed(V.err)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int ZB = H2 * sizeof(C), TB = N2 * sizeof(C);  // one layer's column of Zt / St
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    unsigned char *wbase = smem_raw + (size_t)warp * (CSTAGES * 2 * (ZB + TB) + N * sizeof(C));
    C *zs = reinterpret_cast<C *>(wbase);                              // CSTAGES x 2 x 128
    C *ts = reinterpret_cast<C *>(wbase + CSTAGES * 2 * ZB);           // CSTAGES x 2 x 256
    C *xbuf = reinterpret_cast<C *>(wbase + CSTAGES * 2 * (ZB + TB));  // 512
    C *tab = reinterpret_cast<C *>(smem_raw + (size_t)CWARPS * (CSTAGES * 2 * (ZB + TB) + N * sizeof(C)));
    __shared__ __align__(8) uint64_t bars[CWARPS][CSTAGES];
    __shared__ __align__(8) uint64_t tabbar;
    if (lane == 0)
        for (int s = 0; s < CSTAGES; ++s) mbar_init(&bars[warp][s]);
    if (threadIdx.x == 0) mbar_init(&tabbar);
    mbar_fence_init();
    __syncthreads();
    TabTw<R> tw;
    tw.bind(tab);
    const int nz = V.op[0].nz, sy = V.op[0].sy, nzp = (nz + 1) >> 1;
    const long long T = (long long)V.nfield * NC * nzp;
    const long long Wt = seg_warps((long long)gridDim.x * CWARPS, T);
    const long long w = (long long)blockIdx.x * CWARPS + warp;
    if ((long long)blockIdx.x * CWARPS < Wt) load_twtab<R>(tab, V.twtab, &tabbar);
    if (w >= Wt) return;
    const int t0 = (int)seg_begin(w, T, Wt), t1 = (int)seg_begin(w + 1, T, Wt);
    ColItem cu, ci;  // r counts layer pairs
    cu.set(t0, nzp, V.nfield);
    ci = cu;
    int ti = t0;
    auto issue = [&]() {  // the layer pair of item ti into stage (ti - t0) % CSTAGES
        const int s = (ti - t0) % CSTAGES;
        const OpView<R> &op = V.op[ci.fld];
        const int r0 = 2 * ci.r, nl = r0 + 1 < nz ? 2 : 1;
        const size_t off = (size_t)r0 * NC + ci.kx;
        const uint32_t tb = op.real_spec ? KEB2 : TB;
        mbar_expect(&bars[warp][s], nl * (ZB + tb));
        for (int i = 0; i < nl; ++i) {
            const size_t o = off + (size_t)i * NC;
            bulk_load(zs + (s * 2 + i) * H2, op.Z + o * H2, ZB, &bars[warp][s]);
            if (op.real_spec)
                bulk_load(reinterpret_cast<R *>(ts + s * 2 * N2) + i * KE2, reinterpret_cast<const R *>(op.spec) + o * KE2,
                          tb, &bars[warp][s]);
            else
                bulk_load(ts + (s * 2 + i) * N2, op.spec + o * N2, tb, &bars[warp][s]);
        }
        ++ti;
        ci.next(nzp, V.nfield);
    };
    if (lane == 0)
        while (ti < t1 && ti < t0 + CSTAGES) issue();
    C acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = czero<C>();
    bool ok = __all_sync(0xffffffffu, mbar_wait(&tabbar, 0, V.err));
    int t_fail = ok ? t1 : t0;
    int seg_start = t0;
    for (int t = t0; t < t1 && ok; ++t, cu.next(nzp, V.nfield)) {
        const int s = (t - t0) % CSTAGES;
        const uint32_t par = (uint32_t)(((t - t0) / CSTAGES) & 1);
        ok = __all_sync(0xffffffffu, mbar_wait(&bars[warp][s], par, V.err));
        if (!ok) { t_fail = t; break; }
        const bool mine = 2 * cu.r + h < nz;  // this half-warp's layer exists
        C v[16];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = zs[(s * 2 + h) * H2 + l + 16 * j];
        fwd256h<R>(v, xbuf, tw);
        if (mine) {
            if (V.op[cu.fld].real_spec) {
                const R *tr = reinterpret_cast<const R *>(ts + s * 2 * N2) + h * KE2;
#pragma unroll
                for (int k1 = 0; k1 < 16; ++k1) {
                    const R tt = tr[even_pos256(l, k1)];
                    acc[k1] = mk<C>(acc[k1].x + v[k1].x * tt, acc[k1].y + v[k1].y * tt);
                }
            } else {
                const C *tc = ts + (s * 2 + h) * N2;
#pragma unroll
                for (int k1 = 0; k1 < 16; ++k1) {
                    const C tt = tc[l + 16 * k1];
                    acc[k1].x = fma(v[k1].x, tt.x, acc[k1].x);
                    acc[k1].x = fma(-v[k1].y, tt.y, acc[k1].x);
                    acc[k1].y = fma(v[k1].x, tt.y, acc[k1].y);
                    acc[k1].y = fma(v[k1].y, tt.x, acc[k1].y);
                }
            }
        }
        __syncwarp();
        if (lane == 0 && ti < t1) issue();
        if (cu.r == nzp - 1 || t == t1 - 1) {
            // end of this warp's part of column `col`: the half-warps' layer sums meet
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {
                acc[k1].x += __shfl_xor_sync(0xffffffffu, acc[k1].x, 16);
                acc[k1].y += __shfl_xor_sync(0xffffffffu, acc[k1].y, 16);
            }
            const int fld = cu.fld, kx = cu.kx;
            const long long col = cu.col;
            const OpView<R> &op = V.op[fld];
            const long long cb = col * nzp, ce = cb + nzp - 1;
            const bool whole = (seg_start <= cb) && (t == ce);
            if (!whole) {
                const long long wf = seg_owner(cb, T, Wt), wl = seg_owner(ce, T, Wt);
                const int slot = (int)(w - wf), nslots = (int)(wl - wf + 1);
                C *Pc = V.P[fld] + (size_t)kx * V.slots * N2;
#pragma unroll
                for (int k1 = 0; k1 < 8; ++k1)  // registers chosen by selects, not by a runtime index
                    Pc[(size_t)slot * N2 + l + 16 * (8 * h + k1)] = h ? acc[8 + k1] : acc[k1];
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
                            acc[k1] = cadd(acc[k1], __ldcg(Pc + (size_t)sl * N2 + l + 16 * k1));
                    }
                    if (lane == 0) V.cnt[fld][kx] = 0;
                } else {
#pragma unroll
                    for (int k1 = 0; k1 < 16; ++k1) acc[k1] = czero<C>();
                    seg_start = t + 1;
                    continue;
                }
            }
            // both half-warps hold the column's sum; each writes half of the rows
            inv256h<R>(acc, xbuf, tw);
            C *Wc = op.W + (size_t)kx * H2;
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int n = l + 16 * (4 * h + jj);
                if (n < sy) Wc[n] = h ? acc[4 + jj] : acc[jj];
            }
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) acc[k1] = czero<C>();
            seg_start = t + 1;
        }
    }
    if (!ok) drain(bars[warp], t_fail, t0, t1, V.err);
}

// Adjoint column pass, N_y = 256: for each (field, kx, r),
// Zt_r[kx][iy] = IFFT256(conj(St_r[kx]) . FFT256(Vt[kx]))[iy], iy < ny; half-warp h
// takes layer 2 rp + h of item (kx, field, rp).
template <typename R>
__global__ void __launch_bounds__(CWARPS * 32, 1) k_col_adj256(View2<R> V, const int *done) {
    using C = cpx<R>;
    if (stopped(done) || op_failed(V.err)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TB = N2 * sizeof(C);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    unsigned char *wbase = smem_raw + (size_t)warp * (CSTAGES * 2 * TB + N * sizeof(C));
    C *ts = reinterpret_cast<C *>(wbase);                      // CSTAGES x 2 x 256
    C *xbuf = reinterpret_cast<C *>(wbase + CSTAGES * 2 * TB);  // 512
    C *tab = reinterpret_cast<C *>(smem_raw + (size_t)CWARPS * (CSTAGES * 2 * TB + N * sizeof(C)));
    __shared__ __align__(8) uint64_t bars[CWARPS][CSTAGES];
    __shared__ __align__(8) uint64_t tabbar;
    if (lane == 0)
        for (int s = 0; s < CSTAGES; ++s) mbar_init(&bars[warp][s]);
    if (threadIdx.x == 0) mbar_init(&tabbar);
    mbar_fence_init();
    __syncthreads();
    TabTw<R> tw;
    tw.bind(tab);
    const int nz = V.op[0].nz, ny = V.op[0].ny, nzp = (nz + 1) >> 1;
    const long long T = (long long)V.nfield * NC * nzp;
    const long long Wt = seg_warps((long long)gridDim.x * CWARPS, T);
    const long long w = (long long)blockIdx.x * CWARPS + warp;
    if ((long long)blockIdx.x * CWARPS < Wt) load_twtab<R>(tab, V.twtab, &tabbar);
    if (w >= Wt) return;
    const int t0 = (int)seg_begin(w, T, Wt), t1 = (int)seg_begin(w + 1, T, Wt);
    ColItem cu, ci;  // r counts layer pairs
    cu.set(t0, nzp, V.nfield);
    ci = cu;
    int ti = t0;
    auto issue = [&]() {
        const int s = (ti - t0) % CSTAGES;
        const OpView<R> &op = V.op[ci.fld];
        const int r0 = 2 * ci.r, nl = r0 + 1 < nz ? 2 : 1;
        const size_t off = (size_t)r0 * NC + ci.kx;
        const uint32_t tb = op.real_spec ? KEB2 : TB;
        mbar_expect(&bars[warp][s], nl * tb);
        for (int i = 0; i < nl; ++i) {
            const size_t o = off + (size_t)i * NC;
            if (op.real_spec)
                bulk_load(reinterpret_cast<R *>(ts + s * 2 * N2) + i * KE2, reinterpret_cast<const R *>(op.spec) + o * KE2,
                          tb, &bars[warp][s]);
            else
                bulk_load(ts + (s * 2 + i) * N2, op.spec + o * N2, tb, &bars[warp][s]);
        }
        ++ti;
        ci.next(nzp, V.nfield);
    };
    if (lane == 0)
        while (ti < t1 && ti < t0 + CSTAGES) issue();
    C vh[16];
    bool ok = __all_sync(0xffffffffu, mbar_wait(&tabbar, 0, V.err));
    int t_fail = ok ? t1 : t0;
    for (int t = t0; t < t1 && ok; ++t, cu.next(nzp, V.nfield)) {
        const int fld = cu.fld, kx = cu.kx, r = 2 * cu.r + h;
        const OpView<R> &op = V.op[fld];
        if (t == t0 || cu.r == 0) {  // a new column: both half-warps transform it
            const C *Vc = op.V + (size_t)kx * H2;
#pragma unroll
            for (int j = 0; j < 8; ++j) vh[j] = Vc[l + 16 * j];
            fwd256h<R>(vh, xbuf, tw);
        }
        const int s = (t - t0) % CSTAGES;
        const uint32_t par = (uint32_t)(((t - t0) / CSTAGES) & 1);
        ok = __all_sync(0xffffffffu, mbar_wait(&bars[warp][s], par, V.err));
        if (!ok) { t_fail = t; break; }
        const bool mine = r < nz;
        C v[16];
        if (!mine) {  // the stage holds no spectrum for this half-warp
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) v[k1] = czero<C>();
        } else if (op.real_spec) {
            const R *tr = reinterpret_cast<const R *>(ts + s * 2 * N2) + h * KE2;
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {
                const R tt = tr[even_pos256(l, k1)];
                v[k1] = mk<C>(vh[k1].x * tt, vh[k1].y * tt);
            }
        } else {
            const C *tc = ts + (s * 2 + h) * N2;
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) v[k1] = cmulc(vh[k1], tc[l + 16 * k1]);
        }
        __syncwarp();
        if (lane == 0 && ti < t1) issue();
        inv256h<R>(v, xbuf, tw);
        if (mine) {
            C *Zc = op.Z + ((size_t)r * NC + kx) * H2;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int n = l + 16 * j;
                if (n < ny) Zc[n] = v[j];
            }
        }
    }
    if (!ok) drain(bars[warp], t_fail, t0, t1, V.err);
}

// shared-memory bytes of each kernel
template <typename R> inline size_t smem_col_fwd() {
    return ((size_t)CWARPS * (CSTAGES * (H + N) + N) + TabTw<R>::WORDS) * sizeof(cpx<R>);
}
template <typename R> inline size_t smem_col_adj() {
    return ((size_t)CWARPS * (CSTAGES * N + N) + TabTw<R>::WORDS) * sizeof(cpx<R>);
}
// the 256-row kernels stage two layers of half the length: the same bytes
template <typename R> inline size_t smem_col_fwd256() {
    return ((size_t)CWARPS * (CSTAGES * 2 * (H2 + N2) + N) + TabTw<R>::WORDS) * sizeof(cpx<R>);
}
template <typename R> inline size_t smem_col_adj256() {
    return ((size_t)CWARPS * (CSTAGES * 2 * N2 + N) + TabTw<R>::WORDS) * sizeof(cpx<R>);
}

}  // namespace f512
}  // namespace gj
