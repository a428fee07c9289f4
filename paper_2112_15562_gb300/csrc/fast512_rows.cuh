// Row passes of the 512 x 512 fast path (x direction): real lines <-> half spectra
// in the transposed layout Zt[r][kx][iy] that the column passes of fast512.cuh
// stream.  The warp FFT, the TMA helpers and the segmentation live there.
#pragma once
#include "fast512.cuh"

namespace gj {
namespace f512 {

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
// (single mode: the lines are field `field`'s)
template <typename R, int FFTS>
__device__ __forceinline__ void write_half_spectra(const cpx<R> *tile, const View2<R> &V, int joint, int base,
                                                   int nlines, int lpl, int out_sel, int field = 0) {
    using C = cpx<R>;
    static_assert((FFTS & (FFTS - 1)) == 0, "FFTS must be a power of two");
    // blockDim is a multiple of FFTS, so this thread always serves transform f
    const int f = threadIdx.x % FFTS;
    int la, lb;
    bool ha, hb;
    pair_lines(joint, base, f, nlines, la, lb, ha, hb);
    const int fa = joint ? 0 : field, fb = joint ? 1 : field;
    const int ra = ha ? la / lpl : 0, rb = hb ? lb / lpl : 0;
    const int hy = V.hy;
    C *oa = (out_sel == 0 ? V.op[fa].Z : (out_sel == 1 ? V.op[fa].W : V.op[fa].V)) + (size_t)ra * NC * hy + (la - ra * lpl);
    C *ob = (out_sel == 0 ? V.op[fb].Z : (out_sel == 1 ? V.op[fb].W : V.op[fb].V)) + (size_t)rb * NC * hy + (lb - rb * lpl);
    const C *row = tile + f * (N + 1);
    const int kstep = blockDim.x / FFTS;
    for (int kx = threadIdx.x / FFTS; kx < NC; kx += kstep) {
        const C zk = row[ppos(kx)];
        const C zm = row[ppos((N - kx) & (N - 1))];
        if (ha) oa[kx * hy] = mk<C>(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y));
        if (hb) ob[kx * hy] = mk<C>(R(0.5) * (zk.y + zm.y), R(-0.5) * (zk.x - zm.x));
    }
}

// Real input a + i b held as a[i], b[i] for elements lane + 32 i: redistribute
// through the warp tile and run the forward transform.  Result in v (lane layout).
template <typename R, class TW>
__device__ __forceinline__ void fwd512_from_lines(const R (&a)[8], const R (&b)[8], cpx<R> *buf, const TW &tw,
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
    const int field = blockIdx.y;  // single mode: the field of this CTA's lines (grid y = fields)
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
            field_functor(pro, field).template fetch_batch<4>(la, lb, hb, lane, 32, n_in, a0, b0);
            field_functor(pro, field).template fetch_batch<4>(la, lb, hb, lane + 128, 32, n_in, a1, b1);
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
    write_half_spectra<R, FFTS>(tile, V, joint, base, nlines, lpl, out_sel, field);
    pro.flush(red);
}

// Stages the half spectra of the CTA's lines: source column s < 2 FFTS holds
// (joint) field s / FFTS, line base + s % FFTS, or (single) line base + s.
// The caller synchronises the block before reading the tile.
template <typename R, int FFTS>
__device__ __forceinline__ void stage_half_spectra(cpx<R> *tile, const View2<R> &V, int joint, int base, int nlines,
                                                   int lpl, int in_sel, int field = 0) {
    using C = cpx<R>;
    constexpr int SRC = 2 * FFTS, P = SRC + 1;
    const int s = threadIdx.x % SRC;
    const int fld = joint ? (s / FFTS) : field;
    const int line = joint ? base + (s % FFTS) : base + s;
    const bool ok = line < nlines;
    const int r = ok ? line / lpl : 0, iy = ok ? line - r * lpl : 0;
    const C *src = in_sel == 0 ? V.op[fld].Z : (in_sel == 1 ? V.op[fld].W : V.op[fld].V);
    const int hy = V.hy;
    const C *in = src + (size_t)r * NC * hy + iy;
    const int kx0 = threadIdx.x / SRC, kstep = blockDim.x / SRC;
    // every copy in flight at once; sources past the last line read as zero (their
    // lane may pair with a valid line in the same complex transform)
    for (int kx = kx0; kx < NC; kx += kstep) {
        C *dst = tile + kpos(kx) * P + s;
        if (ok) cp_async8(dst, in + (size_t)kx * hy);
        else *dst = czero<C>();
    }
    cp_async_commit();
    cp_async_wait<0>();  // the caller's barrier publishes the tile
}

// Gathers transform f (sources sa, sb: Hermitian-extended A + i B) in the lane
// layout and runs the inverse transform; returns y[lane + 32 i] in a[i] + i b[i].
template <typename R, int FFTS, class TW>
__device__ __forceinline__ void inv512_to_lines(const cpx<R> *tile, int sa, int sb, cpx<R> *buf, const TW &tw,
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
    const int field = blockIdx.y;  // single mode: the field of this CTA's lines (grid y = fields)
    stage_half_spectra<R, FFTS>(tile, V, joint, base, nlines, lpl, in_sel, field);
    __syncthreads();
    LaneTw<R> tw;
    tw.load_inv(V.op[0].twx);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C *buf = xb + warp * N;
    for (int s2 = 0; s2 < FPW; ++s2) {
        const int f = warp * FPW + s2;
        const int sa = joint ? f : 2 * f;
        const int sb = joint ? FFTS + f : 2 * f + 1;
        int la, lb;
        bool ha, hb;
        pair_lines(joint, base, f, nlines, la, lb, ha, hb);
        if (ha) field_functor(epi, field).prefetch(la, lb, hb, lane, n_out);  // rows load during the transform
        R a[8], b[8];
        inv512_to_lines<R, FFTS>(tile, sa, sb, buf, tw, a, b);
        if (ha) {
            R a0[4], b0[4], a1[4], b1[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a0[i] = a[i]; b0[i] = b[i]; a1[i] = a[4 + i]; b1[i] = b[4 + i]; }
            field_functor(epi, field).template store_batch<4>(la, lb, hb, lane, 32, n_out, a0, b0);
            field_functor(epi, field).template store_batch<4>(la, lb, hb, lane + 128, 32, n_out, a1, b1);
        }
    }
    epi.flush(red);
}

// ---------------------------------------------------------------------------
// Persistent row passes in teams of four warps.  A team takes a balanced contiguous
// range of the aligned groups of the layers (a layer's last group may hold fewer
// lines), so that no launch ends in a partial wave.  Two modes:
//   joint: both fields of a line in one complex transform; a group is four lines,
//          warp k takes line k; the tile is stage[field][slot < 4][kq(kx)] with slot
//          stride 274 (2 mod 16);
//   pair:  one field, two lines per transform (warp k: lines 2k and 2k + 1); a group
//          is eight lines; the tile is stage[slot < 8][kq(kx)] with slot stride 273
//          (1 mod 16).
// The half spectra of a group sit in a double-buffered team tile and move to or from
// the transposed layout out[r][kx][iy] as whole 32-byte sectors.  kq puts even
// columns first and odd ones from 136 on; with these strides a half-warp's 16
// consecutive columns of one slot, and its (column, slot) pairs of a group store or
// load, each fall in 16 distinct bank pairs.  One named barrier per group and team.
// The functor rows read in every launch are staged one transform ahead with
// asynchronous copies.

constexpr int TEAM = 4;                  // warps per team
constexpr int LS = 274, FS = TEAM * LS;  // joint tile: slot and field strides (complex words)
constexpr int LSP = 273;                 // pair tile: slot stride (8 slots fit in 2 FS)
template <bool PAIR> struct TeamMode {
    static constexpr int LPG = PAIR ? 2 * TEAM : TEAM;  // lines per group
    static constexpr int GPT = PAIR ? 8 : 4;            // slots one thread row of a store covers
};

__device__ __forceinline__ void team_barrier(int team) {  // barrier 0 stays with __syncthreads
    asm volatile("bar.sync %0, %1;\n" ::"r"(1 + team), "r"(TEAM * 32) : "memory");
}

__device__ __forceinline__ int kq(int kx) { return (kx & 1) ? 136 + (kx >> 1) : (kx >> 1); }

// Z = FFT(a + i b) in the lane layout (v[k1] = Z[lambda + 32 k1]) -> the half
// spectra A = (Z[kx] + conj Z[N - kx]) / 2 and B = (Z[kx] - conj Z[N - kx]) / 2i,
// kx = 0..256, at sa[kq(kx)] and sb[kq(kx)].  For lambda != 0, Z[N - kx] sits in
// lane (h, 16 - l - h) at k1' = 15 - k1; lane 0 (lambda = 0) holds it at 16 - k1.
template <typename R>
__device__ __forceinline__ void split_to_stage(const cpx<R> (&v)[16], cpx<R> *sa, cpx<R> *sb) {
    using C = cpx<R>;
    const int lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    const int partner = h ? 31 - l : ((16 - l) & 15);
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

// Slots g < ng of a team tile -> out[kx * hy + g] (joint: field 0 to oa, field 1 to
// ob; pair: eight slots to oa; hy = the column stride).  The team's 128 threads take (g, kx) =
// (tid % GPT, tid / GPT + (128 / GPT) i): kx advances by 32 or 16, keeping its parity,
// so kq(kx) advances by half of that.
template <typename R, bool PAIR>
__device__ __forceinline__ void team_store(const cpx<R> *stage, cpx<R> *oa, cpx<R> *ob, int ng, int tid, int hy) {
    constexpr int GPT = TeamMode<PAIR>::GPT, KS = 128 / GPT;
    const int g = tid % GPT;
    if (g >= ng) return;
    int kx = tid / GPT;
    const cpx<R> *sa = stage + g * (PAIR ? LSP : LS) + kq(kx);
    size_t o = (size_t)kx * hy + g;
    for (; kx < NC; kx += KS, sa += KS / 2, o += (size_t)KS * hy) {
        oa[o] = sa[0];
        if (!PAIR) ob[o] = sa[FS];
    }
}

// in[kx * hy + g] -> slots g < ng of a team tile (asynchronous copies; layout as in
// team_store).
template <typename R, bool PAIR>
__device__ __forceinline__ void team_load(cpx<R> *stage, const cpx<R> *ia, const cpx<R> *ib, int ng, int tid,
                                          int hy) {
    constexpr int GPT = TeamMode<PAIR>::GPT, KS = 128 / GPT;
    const int g = tid % GPT;
    if (g >= ng) return;
    int kx = tid / GPT;
    cpx<R> *sa = stage + g * (PAIR ? LSP : LS) + kq(kx);
    size_t o = (size_t)kx * hy + g;
    for (; kx < NC; kx += KS, sa += KS / 2, o += (size_t)KS * hy) {
        cp_async8(sa, ia + o);
        if (!PAIR) cp_async8(sa + FS, ib + o);
    }
}

// A at sa, B at sb (B taken as zero when has_b is false; Hermitian-extended A + i B)
// -> inverse transform -> y[lane + 32 i] in a[i] + i b[i].
template <typename R, class TW>
__device__ __forceinline__ void stage_to_lines(const cpx<R> *sa, const cpx<R> *sb, bool has_b, cpx<R> *buf,
                                               const TW &tw, R (&a)[8], R (&b)[8]) {
    using C = cpx<R>;
    const int lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    const int lam = 2 * l + h;
    C v[16];
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) {
        const int k = lam + 32 * k1;
        const bool lo = k <= H;
        const int kk = lo ? k : N - k;
        C A = sa[kq(kk)], B = has_b ? sb[kq(kk)] : czero<C>();
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

// Stages the functor's rows into pre[a][i][H] (n elements each): source i = 0 from
// row ta, i = 1 from row tb (skipped when tb < 0); 16-byte copies where the rows
// allow them, else 4-byte ones.  Does not commit.
template <typename R, class Fn>
__device__ __forceinline__ void prefetch_rows(const Fn &fn, R *pre, int ta, int tb, int n) {
    constexpr int V4 = 16 / sizeof(R);
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int a = 0; a < Fn::NPRE; ++a)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const R *src = fn.pre_src(a, i);
            const int t = i == 0 ? ta : tb;
            if (!src || t < 0) continue;
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

// Group q of a layer-major sequence (gpl groups of lpg lines per layer): layer, first
// line, lines in the group.
__device__ __forceinline__ void group_lines(int q, int gpl, int lpl, int lpg, int &r, int &iy0, int &ng) {
    r = q / gpl;
    iy0 = (q - r * gpl) * lpg;
    ng = min(lpg, lpl - iy0);
}

// Warp k's transform in a group (layer r, first line iy0, ng lines): its lines la
// (always) and lb (when hb), active when the group reaches la.
template <bool PAIR>
__device__ __forceinline__ bool warp_lines(int k, int r, int iy0, int ng, int lpl, int &la, int &lb, bool &hb) {
    const int s = PAIR ? 2 * k : k;
    la = r * lpl + iy0 + s;
    lb = PAIR ? la + 1 : la;
    hb = PAIR ? s + 1 < ng : true;
    return s < ng;
}

// Forward row pass: lines r lpl + iy (both fields, or pairs of one field's lines)
// through the prologue functor -> half spectra out[r][kx][iy].
template <typename R, class Pro, int NW, bool PAIR>
__global__ void __launch_bounds__(NW * 32, 1) k_row_fwd512t(View2<R> V, int nz, int lpl, int n_in, int out_sel,
                                                            Pro pro, const int *done) {
    using C = cpx<R>;
    static_assert(NW % TEAM == 0, "whole teams");
    constexpr int NT = NW / TEAM, LPG = TeamMode<PAIR>::LPG;
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
    const int gpl = (lpl + LPG - 1) / LPG;
    // pair mode with both fields in V: the groups of field 0, then those of field 1
    const long long NG1 = (long long)nz * gpl;
    const int nfl = (PAIR && V.nfield == 2) ? 2 : 1;
    const long long NG = NG1 * nfl;
    auto fgroup = [&](int q, int &f, int &r, int &iy0, int &ng) {
        f = (nfl == 2 && q >= NG1) ? 1 : 0;
        group_lines(q - (int)(f * NG1), gpl, lpl, LPG, r, iy0, ng);
    };
    const long long Tt = seg_warps((long long)gridDim.x * NT, NG);
    const long long tm = (long long)blockIdx.x * NT + team;
    if (tm < Tt) {
        const int q0 = (int)seg_begin(tm, NG, Tt), q1 = (int)seg_begin(tm + 1, NG, Tt);
        C *out0 = sel_buf(V.op[0], out_sel), *out1 = sel_buf(V.op[1], out_sel);
        int fq, r, iy0, ng, la, lb;
        bool hb;
        fgroup(q0, fq, r, iy0, ng);
        if (warp_lines<PAIR>(k, r, iy0, ng, lpl, la, lb, hb))
            prefetch_rows(field_functor(pro, fq), pre, la, hb ? lb : -1, n_in);
        cp_async_commit();
        for (int q = q0; q < q1; ++q) {
            fgroup(q, fq, r, iy0, ng);
            C *tile = tiles + (q & 1) * 2 * FS;
            const bool act = warp_lines<PAIR>(k, r, iy0, ng, lpl, la, lb, hb);  // this warp has a transform in q
            R a[8], b[8];
            if (act) {
                cp_async_wait<0>();
                __syncwarp();
                R a0[4], b0[4], a1[4], b1[4];
                field_functor(pro, fq).template fetch_batch<4, true>(la, lb, hb, lane, 32, n_in, a0, b0, pre);
                field_functor(pro, fq).template fetch_batch<4, true>(la, lb, hb, lane + 128, 32, n_in, a1, b1, pre);
#pragma unroll
                for (int i = 0; i < 4; ++i) { a[i] = a0[i]; b[i] = b0[i]; a[4 + i] = a1[i]; b[4 + i] = b1[i]; }
                __syncwarp();
            }
            if (q + 1 < q1) {  // the rows of this warp's transform in the next group
                int f2, r2, iy2, ng2, la2, lb2;
                bool hb2;
                fgroup(q + 1, f2, r2, iy2, ng2);
                if (warp_lines<PAIR>(k, r2, iy2, ng2, lpl, la2, lb2, hb2))
                    prefetch_rows(field_functor(pro, f2), pre, la2, hb2 ? lb2 : -1, n_in);
            }
            cp_async_commit();
            if (act) {
                C v[16];
                fwd512_from_lines<R>(a, b, buf, tw, v);
                if (PAIR) split_to_stage<R>(v, tile + 2 * k * LSP, tile + (2 * k + 1) * LSP);
                else split_to_stage<R>(v, tile + k * LS, tile + FS + k * LS);
            }
            team_barrier(team);  // the group's tile is complete; the other tile is free again
            const size_t off = (size_t)r * NC * V.hy + iy0;
            team_store<R, PAIR>(tile, (fq ? out1 : out0) + off, out1 + off, ng, tid, V.hy);
        }
    }
    pro.flush(red);
}

// Inverse row pass: half spectra in[r][kx][iy] -> lines r lpl + iy (both fields, or
// pairs of one field's lines), cropped to n_out, through the epilogue functor.  Copy
// groups in flight at the top of group q: [tile of q], [rows of q's transform].
template <typename R, class Epi, int NW, bool PAIR>
__global__ void __launch_bounds__(NW * 32, 1) k_row_inv512t(View2<R> V, int nz, int lpl, int n_out, int in_sel,
                                                            Epi epi, const int *done) {
    using C = cpx<R>;
    static_assert(NW % TEAM == 0, "whole teams");
    constexpr int NT = NW / TEAM, LPG = TeamMode<PAIR>::LPG;
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
    const int gpl = (lpl + LPG - 1) / LPG;
    // pair mode with both fields in V: the groups of field 0, then those of field 1
    const long long NG1 = (long long)nz * gpl;
    const int nfl = (PAIR && V.nfield == 2) ? 2 : 1;
    const long long NG = NG1 * nfl;
    auto fgroup = [&](int q, int &f, int &r, int &iy0, int &ng) {
        f = (nfl == 2 && q >= NG1) ? 1 : 0;
        group_lines(q - (int)(f * NG1), gpl, lpl, LPG, r, iy0, ng);
    };
    const long long Tt = seg_warps((long long)gridDim.x * NT, NG);
    const long long tm = (long long)blockIdx.x * NT + team;
    if (tm < Tt) {
        const int q0 = (int)seg_begin(tm, NG, Tt), q1 = (int)seg_begin(tm + 1, NG, Tt);
        const C *in0 = sel_buf(V.op[0], in_sel), *in1 = sel_buf(V.op[1], in_sel);
        int fq, r, iy0, ng, la, lb;
        bool hb;
        fgroup(q0, fq, r, iy0, ng);
        {
            const size_t off = (size_t)r * NC * V.hy + iy0;
            team_load<R, PAIR>(tiles + (q0 & 1) * 2 * FS, (fq ? in1 : in0) + off, in1 + off, ng, tid, V.hy);
            cp_async_commit();
            if (warp_lines<PAIR>(k, r, iy0, ng, lpl, la, lb, hb))
                prefetch_rows(field_functor(epi, fq), pre, la, hb ? lb : -1, n_out);
            cp_async_commit();
        }
        for (int q = q0; q < q1; ++q) {
            fgroup(q, fq, r, iy0, ng);
            cp_async_wait<1>();  // this thread's copies of the tile of q
            team_barrier(team);  // everyone's copies of q; the other tile is free again
            if (q + 1 < q1) {
                int f2, r2, iy2, ng2;
                fgroup(q + 1, f2, r2, iy2, ng2);
                const size_t off = (size_t)r2 * NC * V.hy + iy2;
                team_load<R, PAIR>(tiles + ((q + 1) & 1) * 2 * FS, (f2 ? in1 : in0) + off, in1 + off, ng2, tid, V.hy);
            }
            cp_async_commit();
            if (warp_lines<PAIR>(k, r, iy0, ng, lpl, la, lb, hb)) {
                const C *tile = tiles + (q & 1) * 2 * FS;
                R a[8], b[8];
                if (PAIR) stage_to_lines<R>(tile + 2 * k * LSP, tile + (2 * k + 1) * LSP, hb, buf, tw, a, b);
                else stage_to_lines<R>(tile + k * LS, tile + FS + k * LS, true, buf, tw, a, b);
                cp_async_wait<1>();  // the rows of this transform
                __syncwarp();
                R a0[4], b0[4], a1[4], b1[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) { a0[i] = a[i]; b0[i] = b[i]; a1[i] = a[4 + i]; b1[i] = b[4 + i]; }
                field_functor(epi, fq).template store_batch<4, true>(la, lb, hb, lane, 32, n_out, a0, b0, pre);
                field_functor(epi, fq).template store_batch<4, true>(la, lb, hb, lane + 128, 32, n_out, a1, b1, pre);
                __syncwarp();
            }
            if (q + 1 < q1) {
                int f2, r2, iy2, ng2, la2, lb2;
                bool hb2;
                fgroup(q + 1, f2, r2, iy2, ng2);
                if (warp_lines<PAIR>(k, r2, iy2, ng2, lpl, la2, lb2, hb2))
                    prefetch_rows(field_functor(epi, f2), pre, la2, hb2 ? lb2 : -1, n_out);
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
    const int line = base + f;
    const bool ok = line < nlines;
    R wv[2][8], dv[2][8];  // W_d and d of the line, loaded during the transform
    if (ok) epi.template resid_load<8>(line, lane, 32, n_out, wv, dv);
    R a[8], b[8];
    inv512_to_lines<R, FFTS>(tile, f, FFTS + f, buf, tw, a, b);
    tw.load_fwd(V.op[0].twx);
    if (ok) {
        epi.template resid_apply<8>(lane, 32, n_out, wv, dv, a, b);  // a, b <- v of both fields
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

// shared-memory bytes of each row kernel
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

}  // namespace f512
}  // namespace gj
