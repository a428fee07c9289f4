// Kernels of the BTTB/BCCB sensitivity products (Sec. 2.7.1).
//
// A 2-D transform of an Ny x Nx layer is split into a row pass (length Nx, along x)
// and a column pass (length Ny, along y).  Real rows are transformed two at a time
// as one complex sequence (a + i b); the half spectrum of each is recovered from
// Z[k] and Z[N-k].  Only ncol = Nx/2 + 1 columns are kept.  Zero padding is never
// stored: the first stage of each transform skips the inputs beyond the data.
//
// Forward product of one field:  rows (m -> Z) -> columns with the layer spectra
// multiplied and summed over layers (Z -> Y) -> inverse columns (Y -> W) ->
// inverse rows cropped to the stations (W -> d).  Adjoint: rows (r -> W) ->
// columns (W -> Y = V^) -> per layer conj(T^_r) V^ and inverse columns (Y -> Z)
// -> inverse rows cropped to the prisms (Z -> g).
#pragma once
#include "fft.cuh"

namespace gj {

template <typename R>
struct OpView {
    int sx, sy, nx, ny, nz, Nx, Ny, ncol;
    FftPlanDev px, py;
    const cpx<R> *twx;   // W_Nx^k, k < Nx
    const cpx<R> *twy;   // W_Ny^k, k < Ny
    const cpx<R> *spec;  // [nz][Ny][ncol] layer spectra / (Nx Ny)
    cpx<R> *Z;           // [nz*ny][ncol]  row-pass output / adjoint column output
    cpx<R> *Y;           // [Ny][ncol]     summed spectrum / residual spectrum
    cpx<R> *W;           // [max(sy, ...)][ncol]  inverse-column output / residual rows
    cpx<R> *V;           // fast path: residual-row spectra [ncol][256] (unused otherwise)
    int real_spec;       // fast path: spec holds the real, even spectrum of an even table for
                         // ky <= Ny/2 only, R[nz][ncol][even_spec_len(Ny)]
    int rbase;           // first layer of a column launch (per-layer launches of the recompute mode)
    int spec_r0;         // layer held at spec index 0 (0 when all layers are stored)
    int tcol;            // 0: Z, W, V row-major ([line][ncol]); > 0: transposed, line iy of layer r and
                         // bin k at ((r * ncol + k) * tcol + iy) (the N_y = 1024 column kernels' layout)
};

// Stored entries per column of a real, even spectrum (fast path): ky = 0 .. Ny/2,
// padded to a multiple of four values so that every column starts on 16 bytes.
__host__ __device__ constexpr int even_spec_len(int Ny) { return Ny / 2 + 4; }

// How real lines are paired into complex transforms.
struct PairMap {
    int nlines;  // lines per side
    int joint;   // 1: pair q = (line q of op0, line q of op1); 0: lines (2q, 2q+1) of op0
    int lpl;     // lines per layer (0: one layer), for the transposed layout
    __device__ __forceinline__ int npairs() const { return joint ? nlines : (nlines + 1) >> 1; }
    __device__ __forceinline__ void lines(int q, int &la, int &lb, bool &hasb) const {
        if (joint) { la = q; lb = q; hasb = true; }
        else { la = 2 * q; lb = 2 * q + 1; hasb = lb < nlines; }
    }
    // element (line, bin k) of a row pass's output or input
    __device__ __forceinline__ size_t at(int line, int k, int ncol, int tcol) const {
        if (!tcol) return (size_t)line * ncol + k;
        const int L = lpl > 0 ? lpl : nlines;
        const int r = line / L;
        return ((size_t)r * ncol + k) * tcol + (line - r * L);
    }
};

__device__ __forceinline__ bool stopped(const int *done) {
    return done != nullptr && *(volatile const int *)done != 0;
}

// Block-strided loop over it < total in batches of U elements per thread: the U
// loads of a batch are issued before any of its stores, so that a thread keeps U
// global reads in flight instead of one.
template <int U, class Load, class Store>
__device__ __forceinline__ void staged_loop(int total, Load load, Store store) {
    for (int it0 = threadIdx.x; it0 < total; it0 += U * blockDim.x) {
        decltype(load(0)) v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int it = it0 + u * (int)blockDim.x;
            if (it < total) v[u] = load(it);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int it = it0 + u * (int)blockDim.x;
            if (it < total) store(it, v[u]);
        }
    }
}
constexpr int kStageU = 8;  // loads in flight per thread in the general kernels' staging loops
// Batch of a row functor's staging loop: Pro::STAGE_U where the functor states it
// (a functor whose fetch is long arithmetic keeps 1, so that its code is not
// replicated), else 4.
template <class F, class = void> struct StageU { static constexpr int value = 4; };
template <class F> struct StageU<F, decltype((void)F::STAGE_U)> { static constexpr int value = F::STAGE_U; };

// ---------------------------------------------------------------------------
// Row pass, real -> half spectrum.  Pro::fetch(la, lb, hasb, j, a, b) supplies the
// two real inputs of element j (< n_in); Pro::flush(scratch) runs once per block.
template <typename R, class Pro>
__global__ void __launch_bounds__(256) k_row_fwd(OpView<R> op, PairMap pm, int n_in, int P,
                                                 cpx<R> *out0, cpx<R> *out1, Pro pro, const int *done) {
    using C = cpx<R>;
    if (stopped(done)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = op.Nx, ncol = op.ncol;
    C *buf0 = reinterpret_cast<C *>(smem_raw);
    C *buf1 = buf0 + N * P;
    C *tw = buf1 + N * P;
    __shared__ double red[128];
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = op.twx[i];
    pro.init();
    const int q0 = blockIdx.x * P;
    const int np = pm.npairs();
    staged_loop<StageU<Pro>::value>(
        n_in * P,
        [&](int it) {
            const int p = it % P, j = it / P, q = q0 + p;
            R a = 0, b = 0;
            if (q < np) {
                int la, lb; bool hb;
                pm.lines(q, la, lb, hb);
                pro.fetch(la, lb, hb, j, a, b);
            }
            return mk<C>(a, b);
        },
        [&](int it, C z) { buf0[it] = z; });
    __syncthreads();
    C *X = fft_lines<R, false>(buf0, buf1, op.px, P, tw, n_in);
    for (int it = threadIdx.x; it < ncol * P; it += blockDim.x) {
        const int p = it % P, k = it / P, q = q0 + p;
        if (q >= np) continue;
        const C zk = X[k * P + p];
        const C zm = X[((N - k) % N) * P + p];
        int la, lb; bool hb;
        pm.lines(q, la, lb, hb);
        out0[pm.at(la, k, ncol, op.tcol)] = mk<C>(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y));
        if (hb) out1[pm.at(lb, k, ncol, op.tcol)] = mk<C>(R(0.5) * (zk.y + zm.y), R(-0.5) * (zk.x - zm.x));
    }
    pro.flush(red);
}

// ---------------------------------------------------------------------------
// Row pass, half spectrum -> real, cropped to n_out.  Epi::store(la, lb, hasb, j, a, b).
template <typename R, class Epi>
__global__ void __launch_bounds__(256) k_row_inv(OpView<R> op, PairMap pm, int n_out, int P,
                                                 const cpx<R> *in0, const cpx<R> *in1, Epi epi,
                                                 const int *done) {
    using C = cpx<R>;
    if (stopped(done)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = op.Nx, ncol = op.ncol;
    C *buf0 = reinterpret_cast<C *>(smem_raw);
    C *buf1 = buf0 + N * P;
    C *tw = buf1 + N * P;
    __shared__ double red[128];
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = op.twx[i];
    epi.init();
    const int q0 = blockIdx.x * P;
    const int np = pm.npairs();
    staged_loop<kStageU>(
        N * P,
        [&](int it) {
            const int p = it % P, k = it / P, q = q0 + p;
            C z = czero<C>();
            if (q < np) {
                int la, lb; bool hb;
                pm.lines(q, la, lb, hb);
                const bool lo = k < ncol;
                const int kk = lo ? k : N - k;
                C A = in0[pm.at(la, kk, ncol, op.tcol)];
                C B = hb ? in1[pm.at(lb, kk, ncol, op.tcol)] : czero<C>();
                if (kk == 0 || 2 * kk == N) { A.y = 0; B.y = 0; }
                z = lo ? mk<C>(A.x - B.y, A.y + B.x) : mk<C>(A.x + B.y, B.x - A.y);
            }
            return z;
        },
        [&](int it, C z) { buf0[it] = z; });
    __syncthreads();
    C *X = fft_lines<R, true>(buf0, buf1, op.px, P, tw, N);
    for (int it = threadIdx.x; it < n_out * P; it += blockDim.x) {
        const int p = it % P, j = it / P, q = q0 + p;
        if (q >= np) continue;
        int la, lb; bool hb;
        pm.lines(q, la, lb, hb);
        const C z = X[j * P + p];
        epi.store(la, lb, hb, j, z.x, z.y);
    }
    epi.flush(red);
}

// ---------------------------------------------------------------------------
// Column pass of the forward product: for a tile of C columns and a group of
// layers, Y += sum_r T^_r . FFT_y(Z_r).  Y must be zeroed before the launch.
template <typename R>
__global__ void __launch_bounds__(256) k_col_fwd_mac(OpView<R> op0, OpView<R> op1, int C, int L,
                                                     const int *done) {
    using Cx = cpx<R>;
    if (stopped(done)) return;
    const OpView<R> &op = blockIdx.z ? op1 : op0;
    const int c0 = blockIdx.x * C;
    const int r0 = op.rbase + blockIdx.y * L;
    if (r0 >= op.nz || c0 >= op.ncol) return;
    const int r1 = min(r0 + L, op.nz);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ny = op.Ny, ny = op.ny, ncol = op.ncol;
    Cx *buf0 = reinterpret_cast<Cx *>(smem_raw);
    Cx *buf1 = buf0 + Ny * C;
    Cx *acc = buf1 + Ny * C;
    Cx *tw = acc + Ny * C;
    for (int i = threadIdx.x; i < Ny; i += blockDim.x) tw[i] = op.twy[i];
    for (int it = threadIdx.x; it < Ny * C; it += blockDim.x) acc[it] = czero<Cx>();
    for (int r = r0; r < r1; ++r) {
        const Cx *Zr = op.Z + (size_t)r * ny * ncol;
        staged_loop<kStageU>(
            ny * C,
            [&](int it) {
                const int c = it % C, iy = it / C;
                return (c0 + c < ncol) ? Zr[(size_t)iy * ncol + c0 + c] : czero<Cx>();
            },
            [&](int it, Cx z) { buf0[it] = z; });
        __syncthreads();
        const Cx *X = fft_lines<R, false>(buf0, buf1, op.py, C, tw, ny);
        const Cx *Tr = op.spec + (size_t)(r - op.spec_r0) * Ny * ncol;
        staged_loop<kStageU>(
            Ny * C,
            [&](int it) {
                const int c = it % C, ky = it / C;
                return (c0 + c < ncol) ? Tr[(size_t)ky * ncol + c0 + c] : czero<Cx>();
            },
            [&](int it, Cx t) {
                if (c0 + it % C < ncol) acc[it] = cadd(acc[it], cmul(X[it], t));
            });
        __syncthreads();
    }
    for (int it = threadIdx.x; it < Ny * C; it += blockDim.x) {
        const int c = it % C, ky = it / C;
        if (c0 + c < ncol) {
            R *y = reinterpret_cast<R *>(op.Y + (size_t)ky * ncol + c0 + c);
            atomicAdd(y, acc[it].x);
            atomicAdd(y + 1, acc[it].y);
        }
    }
}

// Inverse column pass of the forward product: W[jy] = IFFT_y(Y)[jy], jy < sy.
template <typename R>
__global__ void __launch_bounds__(256) k_col_inv(OpView<R> op0, OpView<R> op1, int C, const int *done) {
    using Cx = cpx<R>;
    if (stopped(done)) return;
    const OpView<R> &op = blockIdx.y ? op1 : op0;
    const int c0 = blockIdx.x * C;
    if (c0 >= op.ncol) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ny = op.Ny, ncol = op.ncol;
    Cx *buf0 = reinterpret_cast<Cx *>(smem_raw);
    Cx *buf1 = buf0 + Ny * C;
    Cx *tw = buf1 + Ny * C;
    for (int i = threadIdx.x; i < Ny; i += blockDim.x) tw[i] = op.twy[i];
    staged_loop<kStageU>(
        Ny * C,
        [&](int it) {
            const int c = it % C, ky = it / C;
            return (c0 + c < ncol) ? op.Y[(size_t)ky * ncol + c0 + c] : czero<Cx>();
        },
        [&](int it, Cx z) { buf0[it] = z; });
    __syncthreads();
    const Cx *X = fft_lines<R, true>(buf0, buf1, op.py, C, tw, Ny);
    for (int it = threadIdx.x; it < op.sy * C; it += blockDim.x) {
        const int c = it % C, jy = it / C;
        if (c0 + c < ncol) op.W[(size_t)jy * ncol + c0 + c] = X[it];
    }
}

// Forward column pass of the residual (adjoint preparation): Y = FFT_y(W), W has
// sy nonzero rows.
template <typename R>
__global__ void __launch_bounds__(256) k_col_fft(OpView<R> op0, OpView<R> op1, int C, const int *done) {
    using Cx = cpx<R>;
    if (stopped(done)) return;
    const OpView<R> &op = blockIdx.y ? op1 : op0;
    const int c0 = blockIdx.x * C;
    if (c0 >= op.ncol) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ny = op.Ny, ncol = op.ncol;
    Cx *buf0 = reinterpret_cast<Cx *>(smem_raw);
    Cx *buf1 = buf0 + Ny * C;
    Cx *tw = buf1 + Ny * C;
    for (int i = threadIdx.x; i < Ny; i += blockDim.x) tw[i] = op.twy[i];
    staged_loop<kStageU>(
        op.sy * C,
        [&](int it) {
            const int c = it % C, iy = it / C;
            return (c0 + c < ncol) ? op.W[(size_t)iy * ncol + c0 + c] : czero<Cx>();
        },
        [&](int it, Cx z) { buf0[it] = z; });
    __syncthreads();
    const Cx *X = fft_lines<R, false>(buf0, buf1, op.py, C, tw, op.sy);
    for (int it = threadIdx.x; it < Ny * C; it += blockDim.x) {
        const int c = it % C, ky = it / C;
        if (c0 + c < ncol) op.Y[(size_t)ky * ncol + c0 + c] = X[it];
    }
}

// Column pass of the adjoint product: for layer r, Z_r = IFFT_y(conj(T^_r) . Y),
// rows iy < ny.
template <typename R>
__global__ void __launch_bounds__(256) k_col_adj(OpView<R> op0, OpView<R> op1, int C, const int *done) {
    using Cx = cpx<R>;
    if (stopped(done)) return;
    const OpView<R> &op = blockIdx.z ? op1 : op0;
    const int c0 = blockIdx.x * C;
    const int r = op.rbase + blockIdx.y;
    if (c0 >= op.ncol || r >= op.nz) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ny = op.Ny, ncol = op.ncol, ny = op.ny;
    Cx *buf0 = reinterpret_cast<Cx *>(smem_raw);
    Cx *buf1 = buf0 + Ny * C;
    Cx *tw = buf1 + Ny * C;
    for (int i = threadIdx.x; i < Ny; i += blockDim.x) tw[i] = op.twy[i];
    const Cx *Tr = op.spec + (size_t)(r - op.spec_r0) * Ny * ncol;
    staged_loop<kStageU>(
        Ny * C,
        [&](int it) {
            const int c = it % C, ky = it / C;
            return (c0 + c < ncol) ? cmulc(op.Y[(size_t)ky * ncol + c0 + c], Tr[(size_t)ky * ncol + c0 + c])
                                   : czero<Cx>();
        },
        [&](int it, Cx z) { buf0[it] = z; });
    __syncthreads();
    const Cx *X = fft_lines<R, true>(buf0, buf1, op.py, C, tw, Ny);
    Cx *Zr = op.Z + (size_t)r * ny * ncol;
    for (int it = threadIdx.x; it < ny * C; it += blockDim.x) {
        const int c = it % C, iy = it / C;
        if (c0 + c < ncol) Zr[(size_t)iy * ncol + c0 + c] = X[it];
    }
}

// ---------------------------------------------------------------------------
// Plain functors.

// row length of the staged functor rows of the 512 row passes (pre[a][i][kStageRow])
constexpr int kStageRow = 256;

template <typename R>
struct LoadPlain {  // a = x0[la*pitch + j], b = x1[lb*pitch + j]
    const R *x0;
    const R *x1;
    int pitch;
    static constexpr int NPRE = 1;  // rows la of x0 and lb of x1, staged by the 512 team passes
    static constexpr int STAGE_U = 8;
    __device__ const R *pre_src(int, int i) const { return i == 0 ? x0 : x1; }
    __device__ void init() {}
    __device__ __forceinline__ void fetch(int la, int lb, bool hb, int j, R &a, R &b) const {
        a = x0[(size_t)la * pitch + j];
        b = hb ? x1[(size_t)lb * pitch + j] : R(0);
    }
    // elements j0 + k * stride (k < K) below n; zero beyond
    template <int K, bool PRE = false>
    __device__ __forceinline__ void fetch_batch(int la, int lb, bool hb, int j0, int stride, int n, R (&a)[K],
                                                R (&b)[K], const R *pre = nullptr) const {
        const R *pa = PRE ? pre : x0 + (size_t)la * pitch;
        const R *pb = PRE ? pre + kStageRow : x1 + (size_t)lb * pitch;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + k * stride;
            a[k] = j < n ? pa[j] : R(0);
            b[k] = (hb && j < n) ? pb[j] : R(0);
        }
    }
    __device__ __forceinline__ void flush(double *) const {}
};

template <typename R>
struct StorePlain {
    R *y0;
    R *y1;
    int pitch;
    static constexpr int NPRE = 0;  // reads nothing
    __device__ const R *pre_src(int, int) const { return nullptr; }
    __device__ __forceinline__ void prefetch(int, int, bool, int, int) const {}
    __device__ void init() {}
    __device__ __forceinline__ void store(int la, int lb, bool hb, int j, R a, R b) const {
        y0[(size_t)la * pitch + j] = a;
        if (hb) y1[(size_t)lb * pitch + j] = b;
    }
    template <int K, bool PRE = false>
    __device__ __forceinline__ void store_batch(int la, int lb, bool hb, int j0, int stride, int n, const R (&a)[K],
                                                const R (&b)[K], const R * = nullptr) const {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + k * stride;
            if (j < n) {
                y0[(size_t)la * pitch + j] = a[k];
                if (hb) y1[(size_t)lb * pitch + j] = b[k];
            }
        }
    }
    __device__ __forceinline__ void flush(double *) const {}
};

// ---------------------------------------------------------------------------
// Two fields' single-field products in one launch (the pair calls): a functor per
// field, the one of field f taken with field_functor(pro, f).  Every other functor
// serves its launch's lines as it is.
template <typename R>
struct LoadPlain2 {  // field f: lines la and lb of x[f]
    const R *x[2];
    int pitch;
    static constexpr int NPRE = LoadPlain<R>::NPRE;
    __device__ void init() {}
    __device__ void flush(double *) const {}
    __device__ LoadPlain<R> of(int f) const {  // a select, not an indexed load
        const R *p = f ? x[1] : x[0];
        return LoadPlain<R>{p, p, pitch};
    }
};
template <typename R>
struct StorePlain2 {  // field f: lines la and lb of y[f]
    R *y[2];
    int pitch;
    static constexpr int NPRE = StorePlain<R>::NPRE;
    __device__ void init() {}
    __device__ void flush(double *) const {}
    __device__ StorePlain<R> of(int f) const {  // a select, not an indexed load
        R *p = f ? y[1] : y[0];
        return StorePlain<R>{p, p, pitch};
    }
};
template <class P>
__device__ __forceinline__ P &field_functor(P &p, int) { return p; }
template <typename R>
__device__ __forceinline__ LoadPlain<R> field_functor(const LoadPlain2<R> &p, int f) { return p.of(f); }
template <typename R>
__device__ __forceinline__ StorePlain<R> field_functor(const StorePlain2<R> &p, int f) { return p.of(f); }
template <typename R>
__device__ __forceinline__ LoadPlain<R> field_functor(LoadPlain2<R> &p, int f) { return p.of(f); }
template <typename R>
__device__ __forceinline__ StorePlain<R> field_functor(StorePlain2<R> &p, int f) { return p.of(f); }

}  // namespace gj
