// Operator setup (Sec. 2.7.1): prism kernel tables of every depth layer, their
// BCCB embedding and 2-D spectra.  All geometry arithmetic runs in FP64.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "fast1024.cuh"
#include "fast512.cuh"
#include "view.cuh"

namespace gj {

// ---------------------------------------------------------------------------
// Closed-form prism fields as corner sums of antiderivatives (Sec. 2.1 cites
// Haaz for the vertical gravity and Rao & Babu for the total-field anomaly).
// u = x' - x0, v = y' - y0, w = z' - z0 (z down) with w >= 0 at every corner;
// u and v are never zero because corners sit half a cell from the stations.

// ln(a + R) for R = sqrt(a^2 + b^2 + c^2); for a < 0 use (b^2 + c^2) / (R - a).
__device__ __forceinline__ double log_a_plus_r(double a, double R, double b, double c) {
    return a >= 0.0 ? log(a + R) : log((b * b + c * c) / (R - a));
}

// Antiderivative whose mixed third derivative is w / R^3.
__device__ __forceinline__ double gravity_corner(double u, double v, double w) {
    const double R = sqrt(u * u + v * v + w * w);
    return -(u * log_a_plus_r(v, R, u, w) + v * log_a_plus_r(u, R, v, w) - w * atan2(u * v, w * R));
}

// t^T H t with H the antiderivatives of the second derivatives of 1/R, weights
// c = (txx, tyy, tzz, 2txy, 2txz, 2tyz).
struct MagCoef { double c[6]; };

__device__ __forceinline__ double magnetic_corner(double u, double v, double w, const MagCoef &k) {
    const double R = sqrt(u * u + v * v + w * w);
    const double hxx = -atan(v * w / (u * R));
    const double hyy = -atan(u * w / (v * R));
    const double hzz = -atan2(u * v, w * R);
    const double hxy = log_a_plus_r(w, R, u, v);
    const double hxz = log_a_plus_r(v, R, u, w);
    const double hyz = log_a_plus_r(u, R, v, w);
    return k.c[0] * hxx + k.c[1] * hyy + k.c[2] * hzz + k.c[3] * hxy + k.c[4] * hxz + k.c[5] * hyz;
}

struct Lattice {
    int nbx1, nby1, nz1;     // lattice points in u, v, w
    int a_max, b_max;
    double dx, dy;
    const double *zw;        // nz + 1 values of w
};

__global__ void k_corner_lattice(Lattice L, int magnetic, MagCoef mc, double *out) {
    const size_t total = (size_t)L.nbx1 * L.nby1 * L.nz1;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(i % L.nbx1);
        const int f = (int)((i / L.nbx1) % L.nby1);
        const int k = (int)(i / ((size_t)L.nbx1 * L.nby1));
        const double u = (-(double)L.b_max - 0.5 + e) * L.dx;
        const double v = (-(double)L.a_max - 0.5 + f) * L.dy;
        const double w = L.zw[k];
        out[i] = magnetic ? magnetic_corner(u, v, w, mc) : gravity_corner(u, v, w);
    }
}

// Far from the station the 8-corner sums cancel (their terms grow like R log R
// while the field falls like 1/R^2): a prism whose centre is at least kFar times its
// largest side away is integrated by tensor Gauss-Legendre cubature of the smooth
// integrand instead, 5 points per axis up to 3 kFar sides, 4 up to 8 kFar and 3
// beyond (relative error at most about 5e-13 there, against 1e-7 for the corner
// sums at 100 sides).
constexpr double kFar = 8.0;
// Gauss-Legendre nodes and weights on [-1, 1]
__constant__ double kGL5x[5] = {-0.90617984593866399280, -0.53846931010568309104, 0.0, 0.53846931010568309104,
                                0.90617984593866399280};
__constant__ double kGL5w[5] = {0.23692688505618908751, 0.47862867049936646804, 0.56888888888888888889,
                                0.47862867049936646804, 0.23692688505618908751};
__constant__ double kGL4x[4] = {-0.86113631159405257522, -0.33998104358485626480, 0.33998104358485626480,
                                0.86113631159405257522};
__constant__ double kGL4w[4] = {0.34785484513745385737, 0.65214515486254614263, 0.65214515486254614263,
                                0.34785484513745385737};
__constant__ double kGL3x[3] = {-0.77459666924148337704, 0.0, 0.77459666924148337704};
__constant__ double kGL3w[3] = {0.55555555555555555556, 0.88888888888888888889, 0.55555555555555555556};

// The integral over [u1, u2] x [v1, v2] x [w1, w2] of w / R^3 (gravity) or of
// t^T (d2(1/R)/dr dr) t = (c0 (3u^2 - R^2) + c1 (3v^2 - R^2) + c2 (3w^2 - R^2)
// + 3 (c3 uv + c4 uw + c5 vw)) / R^5 (magnetic), by an n-point tensor rule in
// precision F.  The integrand is smooth there and the sum has no cancellation to
// speak of, so for an FP32 operator (whose spectra are rounded to FP32) the rule runs
// in FP32, some 30 times the FP64 rate; FP64 operators keep FP64.
template <typename F> __device__ __forceinline__ F rsqrt_t(F x);
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }

template <int NP, typename F>
__device__ double far_cubature(double uc_, double hu_, double vc_, double hv_, double wc_, double hw_, int magnetic,
                               const MagCoef &k) {
    const double *x = NP == 5 ? kGL5x : (NP == 4 ? kGL4x : kGL3x);
    const double *wt = NP == 5 ? kGL5w : (NP == 4 ? kGL4w : kGL3w);
    const F uc = (F)uc_, hu = (F)hu_, vc = (F)vc_, hv = (F)hv_, wc = (F)wc_, hw = (F)hw_;
    const F c0 = (F)k.c[0], c1 = (F)k.c[1], c2 = (F)k.c[2], c3 = (F)k.c[3], c4 = (F)k.c[4], c5 = (F)k.c[5];
    F s = 0;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
        const F u = uc + hu * (F)x[a];
#pragma unroll
        for (int b = 0; b < NP; ++b) {
            const F v = vc + hv * (F)x[b];
            F sw = 0;
#pragma unroll
            for (int c = 0; c < NP; ++c) {
                const F w = wc + hw * (F)x[c];
                const F r2 = u * u + v * v + w * w;
                const F ir = rsqrt_t<F>(r2);
                const F ir3 = ir * ir * ir;
                F f;
                if (magnetic) {
                    const F q = c0 * (F(3) * u * u - r2) + c1 * (F(3) * v * v - r2) + c2 * (F(3) * w * w - r2) +
                                F(3) * (c3 * u * v + c4 * u * w + c5 * v * w);
                    f = q * ir3 * ir * ir;
                } else {
                    f = w * ir3;
                }
                sw += (F)wt[c] * f;
            }
            s += (F)(wt[a] * wt[b]) * sw;
        }
    }
    return (double)s * hu_ * hv_ * hw_;
}

// Row-pass input of the setup: the circulant embedding of layer r's table,
// T[c_y mod Ny][c_x mod Nx] = K(c_y + off_y, c_x + off_x) for c in
// [-(n-1), s-1], zero elsewhere; K is the 8-corner sum of the lattice, or the
// far-field cubature.
struct LoadTable {
    static constexpr int STAGE_U = 1;  // the fetch is the corner differences and the far-field cubature
    const double *lat;
    int nbx1, nby1;
    int Nx, Ny, sx, sy, nx, ny, off_x, off_y, a_max, b_max;
    double scale;
    double dx, dy;
    const double *zw;  // depth planes of the build's layers (relative to the stations)
    int magnetic;
    int far32;  // far-field cubature in FP32 (FP32 operators)
    MagCoef mc;
    template <typename F> __device__ double far(double uc, double vc, double wc, double hw, double dist,
                                                double size) const {
        return dist < 3.0 * kFar * size ? far_cubature<5, F>(uc, 0.5 * dx, vc, 0.5 * dy, wc, hw, magnetic, mc)
             : dist < 8.0 * kFar * size ? far_cubature<4, F>(uc, 0.5 * dx, vc, 0.5 * dy, wc, hw, magnetic, mc)
                                        : far_cubature<3, F>(uc, 0.5 * dx, vc, 0.5 * dy, wc, hw, magnetic, mc);
    }
    __device__ void init() {}
    __device__ double value(int line, int j) const {
        const int r = line / Ny, iy = line % Ny;
        int cy, cx;
        if (iy <= sy - 1) cy = iy; else if (iy >= Ny - (ny - 1)) cy = iy - Ny; else return 0.0;
        if (j <= sx - 1) cx = j; else if (j >= Nx - (nx - 1)) cx = j - Nx; else return 0.0;
        {
            // the prism spans u in [-(cx + off_x) -+ 1/2] dx, v likewise, w in [zw[r], zw[r + 1]]
            const double uc = -(double)(cx + off_x) * dx, vc = -(double)(cy + off_y) * dy;
            const double w1 = zw[r], w2 = zw[r + 1];
            const double wc = 0.5 * (w1 + w2), hw = 0.5 * (w2 - w1);
            const double size = fmax(fmax(dx, dy), w2 - w1);
            const double dist = sqrt(uc * uc + vc * vc + wc * wc);
            if (dist >= kFar * size) {
                const double v = far32 ? far<float>(uc, vc, wc, hw, dist, size) : far<double>(uc, vc, wc, hw, dist, size);
                return v * scale;
            }
        }
        const int e = b_max - (cx + off_x);
        const int f = a_max - (cy + off_y);
        if (e < 0 || e + 1 >= nbx1 || f < 0 || f + 1 >= nby1) {
            // outside the lattice window (it covers every offset nearer than kFar prism
            // sizes, so this is never taken): the cubature, in FP64
            const double uc = -(double)(cx + off_x) * dx, vc = -(double)(cy + off_y) * dy;
            const double w1 = zw[r], w2 = zw[r + 1];
            const double size = fmax(fmax(dx, dy), w2 - w1);
            const double dist = sqrt(uc * uc + vc * vc + 0.25 * (w1 + w2) * (w1 + w2));
            return far<double>(uc, vc, 0.5 * (w1 + w2), 0.5 * (w2 - w1), dist, size) * scale;
        }
        double s = 0.0;
#pragma unroll
        for (int dk = 0; dk < 2; ++dk)
#pragma unroll
            for (int df = 0; df < 2; ++df)
#pragma unroll
                for (int de = 0; de < 2; ++de) {
                    const double t = lat[((size_t)(r + dk) * nby1 + (f + df)) * nbx1 + (e + de)];
                    s += ((de + df + dk) & 1) ? t : -t;
                }
        return s * scale;
    }
    __device__ __forceinline__ void fetch(int la, int lb, bool hb, int j, double &a, double &b) const {
        a = value(la, j);
        b = hb ? value(lb, j) : 0.0;
    }
    __device__ __forceinline__ void flush(double *) const {}
};

// Column pass of the setup: spec[r] = FFT_y of the row-pass output of layer r.
template <typename Rout>
__global__ void __launch_bounds__(256) k_col_spec(OpView<double> op, const double2 *Zs, cpx<Rout> *spec, int C,
                                                  int transposed, int real_only) {
    using Cx = double2;
    const int c0 = blockIdx.x * C;
    const int r = blockIdx.y;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ny = op.Ny, ncol = op.ncol;
    Cx *buf0 = reinterpret_cast<Cx *>(smem_raw);
    Cx *buf1 = buf0 + Ny * C;
    Cx *tw = buf1 + Ny * C;
    for (int i = threadIdx.x; i < Ny; i += blockDim.x) tw[i] = op.twy[i];
    const Cx *Zr = Zs + (size_t)r * Ny * ncol;
    for (int it = threadIdx.x; it < Ny * C; it += blockDim.x) {
        const int c = it % C, iy = it / C;
        buf0[it] = (c0 + c < ncol) ? Zr[(size_t)iy * ncol + c0 + c] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const Cx *X = fft_lines<double, false>(buf0, buf1, op.py, C, tw, Ny);
    cpx<Rout> *Sr = spec + (size_t)r * Ny * ncol;
    const int ke = even_spec_len(Ny);
    for (int it = threadIdx.x; it < Ny * C; it += blockDim.x) {
        const int c = it % C, ky = it / C;
        if (c0 + c < ncol) {
            if (real_only) {
                // the table is even in both offsets: the spectrum is real (its imaginary part
                // is zero in exact arithmetic) and even in ky, so only ky <= Ny/2 is kept,
                // as R[r][kx][ke] (fast path)
                if (ky <= Ny / 2)
                    reinterpret_cast<Rout *>(spec)[((size_t)r * ncol + c0 + c) * ke + ky] = (Rout)X[it].x;
            } else {
                const size_t at = transposed ? (size_t)(c0 + c) * Ny + ky : (size_t)ky * ncol + c0 + c;
                Sr[at] = mk<cpx<Rout>>((Rout)X[it].x, (Rout)X[it].y);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Host helpers

// Radix plan of an N-point transform.  order 0: the power-of-two part in radix 8
// (one or two radix-4 stages for the rest), then the odd primes ascending; order 1:
// the same stages in reverse; order 2: the power-of-two part in radix 4 (and one
// radix 2), then the odd primes.
bool plan_size(int N, FftPlanDev &plan, int order) {
    if (N < 1 || N > 2048 || order < 0 || order > 2) return false;
    int n = N, e = 0;
    while (n % 2 == 0) { n /= 2; ++e; }
    std::vector<int> rs;
    if (order == 2) {
        rs.assign(e / 2, 4);
        if (e % 2) rs.push_back(2);
    } else {
        rs.assign(e / 3, 8);
        if (e % 3 == 1) {
            if (!rs.empty()) { rs.back() = 4; rs.push_back(4); } else rs.push_back(2);
        } else if (e % 3 == 2) {
            rs.push_back(4);
        }
    }
    const int primes[] = {3, 5, 7, 11, 13, 17};
    for (int p : primes)
        while (n % p == 0) { n /= p; rs.push_back(p); }
    if (n != 1) return false;
    if (order == 1) std::reverse(rs.begin(), rs.end());
    if ((int)rs.size() > kMaxStages) return false;
    plan.N = N;
    plan.nst = (int)rs.size();
    for (int i = 0; i < kMaxStages; ++i) plan.radix[i] = i < plan.nst ? rs[i] : 1;
    return true;
}

int autotune_size(int minN) {
    for (int N = std::max(1, minN);; ++N) {
        int n = N;
        for (int p : {2, 3, 5, 7})
            while (n % p == 0) n /= p;
        if (n == 1) return N;
    }
}

void make_twiddles(int N, std::vector<double> &re, std::vector<double> &im) {
    re.resize(N);
    im.resize(N);
    const double two_pi = 6.283185307179586476925286766559;
    for (int k = 0; k < N; ++k) {
        // exact values at the quarter points keep the small radices exact
        if (4 * k % N == 0) {
            const int q = 4 * k / N;
            const double c[4] = {1, 0, -1, 0}, s[4] = {0, -1, 0, 1};
            re[k] = c[q];
            im[k] = s[q];
        } else {
            const double a = two_pi * (double)k / (double)N;
            re[k] = std::cos(a);
            im[k] = -std::sin(a);
        }
    }
}

size_t elem_bytes(gj_precision p) { return p == GJ_FP64 ? sizeof(double) : sizeof(float); }

// FP32, N_x = 512 with at most 256 prisms and stations along x, and N_y = 512 (or
// 256) with at most 256 (128) along y.
bool fast_eligible(const gj_op *op) {
    const int hy = op->Ny / 2;
    return op->prec == GJ_FP32_MIXED && op->Nx == 512 && (op->Ny == 512 || op->Ny == 256) && op->nx <= 256 &&
           op->sx <= 256 && op->ny <= hy && op->sy <= hy;
}

// Items per (field, kx) column of the fast column kernels: one per layer at N_y = 512,
// one per layer pair at N_y = 256.
int fast_col_items(int Ny, int nz) { return Ny == 256 ? (nz + 1) / 2 : nz; }

// Largest number of warps that share one (field, kx) column when persistent column
// kernels of `warps` warps split the (kx, field, item) sequence into balanced segments.
int fast_slots(int nfield, int ncol, int nz, long long warps) {
    const long long T = (long long)nfield * ncol * nz;
    const long long Wt = std::min(warps, T);
    auto owner = [&](long long t) { return ((t + 1) * Wt + T - 1) / T - 1; };
    long long mx = 1;
    for (long long c = 0; c < (long long)nfield * ncol; ++c)
        mx = std::max(mx, owner(c * nz + nz - 1) - owner(c * nz) + 1);
    return (int)mx;
}

bool fast1024_eligible(const gj_op *op) {
    return op->prec == GJ_FP32_MIXED && !op->fast && op->Ny == 1024 && op->ny <= 512 && op->sy <= 512;
}

int pick_row_pairs(int Nx, size_t cs) {
    int P = 16;
    while (P > 1 && row_smem(Nx, P, cs) > 96 * 1024) P >>= 1;
    return P;
}

int pick_col_tile(int Ny, size_t cs, int nbuf) {
    int C = 16;
    while (C > 1 && col_smem(Ny, C, nbuf, cs) > 100 * 1024) C >>= 1;
    return C;
}

static gj_status upload_twiddles(int N, gj_precision prec, void **out) {
    std::vector<double> re, im;
    make_twiddles(N, re, im);
    if (prec == GJ_FP64) {
        std::vector<double2> h(N);
        for (int k = 0; k < N; ++k) h[k] = make_double2(re[k], im[k]);
        GJ_CUDA(cudaMalloc(out, N * sizeof(double2)));
        GJ_CUDA(cudaMemcpy(*out, h.data(), N * sizeof(double2), cudaMemcpyHostToDevice));
    } else {
        std::vector<float2> h(N);
        for (int k = 0; k < N; ++k) h[k] = make_float2((float)re[k], (float)im[k]);
        GJ_CUDA(cudaMalloc(out, N * sizeof(float2)));
        GJ_CUDA(cudaMemcpy(*out, h.data(), N * sizeof(float2), cudaMemcpyHostToDevice));
    }
    return GJ_OK;
}

struct gj_setup_scratch_impl;
static void scratch_free(gj_setup_scratch_impl *sc);

static void free_op_memory(gj_op *op) {
    if (!op) return;
    scratch_free(op->scratch);
    op->scratch = nullptr;
    cudaFree(op->twx); cudaFree(op->twy); cudaFree(op->spec);
    cudaFree(op->Z); cudaFree(op->Y); cudaFree(op->W); cudaFree(op->V); cudaFree(op->twtab);
    op->twx = op->twy = op->spec = op->Z = op->Y = op->W = op->V = op->twtab = nullptr;
}

// Work buffers of the spectrum build for `layers` consecutive layers: the FP64
// corner lattice (layers + 1 depth planes), the FP64 row-pass output, the depths
// and FP64 twiddles.  Kept by operators that rebuild their spectra per layer.
struct gj_setup_scratch_impl {
    double *lat = nullptr;
    double2 *Zs = nullptr;
    double *zw = nullptr;
    void *twx64 = nullptr, *twy64 = nullptr;
    bool own_tw = false;
    int layers = 0;
};

static void scratch_free(gj_setup_scratch_impl *sc) {
    if (!sc) return;
    cudaFree(sc->lat); cudaFree(sc->Zs); cudaFree(sc->zw);
    if (sc->own_tw) { cudaFree(sc->twx64); cudaFree(sc->twy64); }
    delete sc;
}

// The corner lattice serves only the prisms nearer than kFar sizes (the rest take
// the cubature), so it spans the offsets c + off in [-W, W] of each direction that the
// table uses, W = ceil(kFar * largest side / cell) + 1: 2W + 2 points per direction
// at most, whatever the grid.  b_max is the largest offset in the window, nb1 the
// lattice points (offsets b_max down to the smallest, plus one).
struct LatticeWindow { int b_max, nbx1, a_max, nby1; };
static LatticeWindow lattice_window(const gj_op *op) {
    double size = std::max(op->dx, op->dy);
    for (int k = 0; k < op->nz; ++k) size = std::max(size, op->z_edges[k + 1] - op->z_edges[k]);
    auto one = [&](int off, int s, int n, double cell, int &hi, int &nb) {
        const int W = (int)std::ceil(kFar * size / cell) + 1;
        hi = std::min(off + s - 1, W);
        const int lo = std::max(off - n + 1, -W);
        nb = std::max(2, hi - lo + 2);
    };
    LatticeWindow w;
    one(op->off_x, op->sx, op->nx, op->dx, w.b_max, w.nbx1);
    one(op->off_y, op->sy, op->ny, op->dy, w.a_max, w.nby1);
    return w;
}

static gj_status scratch_alloc(const gj_op *op, int layers, gj_setup_scratch_impl **out) {
    gj_setup_scratch_impl *sc = new (std::nothrow) gj_setup_scratch_impl();
    if (!sc) { set_error("setup scratch: host allocation failed"); return GJ_ERR_OOM; }
    sc->layers = layers;
    gj_status rc = GJ_OK;
    cudaError_t e;
    if (op->prec == GJ_FP64) {
        sc->twx64 = op->twx;
        sc->twy64 = op->twy;
    } else {
        sc->own_tw = true;
        if ((rc = upload_twiddles(op->Nx, GJ_FP64, &sc->twx64)) != GJ_OK) { scratch_free(sc); return rc; }
        if ((rc = upload_twiddles(op->Ny, GJ_FP64, &sc->twy64)) != GJ_OK) { scratch_free(sc); return rc; }
    }
    const LatticeWindow lw = lattice_window(op);
    const size_t plane = (size_t)lw.nbx1 * lw.nby1;
    std::vector<double> zw(op->nz + 1);
    for (int k = 0; k <= op->nz; ++k) zw[k] = op->z_edges[k] - op->station_z;
    if ((e = cudaMalloc(&sc->lat, plane * (layers + 1) * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&sc->Zs, (size_t)layers * op->Ny * op->ncol * sizeof(double2))) != cudaSuccess ||
        (e = cudaMalloc(&sc->zw, zw.size() * sizeof(double))) != cudaSuccess ||
        (e = cudaMemcpy(sc->zw, zw.data(), zw.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) {
        scratch_free(sc);
        return cuda_fail(e, "setup scratch");
    }
    *out = sc;
    return GJ_OK;
}

// Spectra of layers r0 .. r0 + count - 1 (count <= the scratch's layers) into
// spec[0 .. count): corner lattice of the count + 1 depth planes, the circulant
// embedding of each layer's table differenced from it while loading the FP64 row
// transforms, FP64 column transforms, rounding to the operator's precision.
// Enqueues only (no synchronisation).
template <typename Rout>
static void build_layers(const gj_op *op, const gj_setup_scratch_impl &sc, int r0, int count, cpx<Rout> *spec,
                         cudaStream_t st) {
    Lattice L;
    const LatticeWindow lw = lattice_window(op);
    L.b_max = lw.b_max;
    L.a_max = lw.a_max;
    L.nbx1 = lw.nbx1;
    L.nby1 = lw.nby1;
    L.nz1 = count + 1;
    L.dx = op->dx;
    L.dy = op->dy;
    L.zw = sc.zw + r0;
    MagCoef mc{};
    double scale = 1.0 / ((double)op->Nx * (double)op->Ny);
    const int magnetic = op->field == GJ_MAGNETIC;
    if (magnetic) {
        const double d2r = 3.14159265358979323846 / 180.0;
        const double I = op->mag.incl_deg * d2r, D = op->mag.decl_deg * d2r;
        const double t[3] = {std::cos(I) * std::sin(D), std::cos(I) * std::cos(D), std::sin(I)};
        mc.c[0] = t[0] * t[0]; mc.c[1] = t[1] * t[1]; mc.c[2] = t[2] * t[2];
        mc.c[3] = 2 * t[0] * t[1]; mc.c[4] = 2 * t[0] * t[2]; mc.c[5] = 2 * t[1] * t[2];
        scale *= op->mag.F_nT / (4.0 * 3.14159265358979323846);
    } else {
        // G = 6.6743e-11 m^3 kg^-1 s^-2; g/cc -> kg/m^3 (1e3); m/s^2 -> mGal (1e5)
        scale *= 6.6743e-11 * 1.0e3 * 1.0e5;
    }
    const size_t lat_pts = (size_t)L.nbx1 * L.nby1 * L.nz1;
    k_corner_lattice<<<(int)std::min<size_t>(1216, (lat_pts + 255) / 256), 256, 0, st>>>(L, magnetic, mc, sc.lat);

    OpView<double> v{};
    v.sx = op->sx; v.sy = op->sy; v.nx = op->nx; v.ny = op->ny; v.nz = count;
    v.Nx = op->Nx; v.Ny = op->Ny; v.ncol = op->ncol; v.px = op->px; v.py = op->py;
    v.twx = static_cast<const double2 *>(sc.twx64);
    v.twy = static_cast<const double2 *>(sc.twy64);

    LoadTable lt;
    lt.lat = sc.lat; lt.nbx1 = L.nbx1; lt.nby1 = L.nby1;
    lt.Nx = op->Nx; lt.Ny = op->Ny; lt.sx = op->sx; lt.sy = op->sy; lt.nx = op->nx; lt.ny = op->ny;
    lt.off_x = op->off_x; lt.off_y = op->off_y; lt.a_max = L.a_max; lt.b_max = L.b_max;
    lt.scale = scale;
    lt.dx = op->dx; lt.dy = op->dy;
    lt.zw = sc.zw + r0;
    lt.magnetic = magnetic;
    lt.far32 = op->prec == GJ_FP32_MIXED ? 1 : 0;
    lt.mc = mc;
    PairMap pm{count * op->Ny, 0};
    const int P = pick_row_pairs(op->Nx, sizeof(double2));
    const int npairs = (pm.nlines + 1) / 2;
    const size_t rsm = row_smem(op->Nx, P, sizeof(double2));
    k_row_fwd<double, LoadTable><<<(npairs + P - 1) / P, 256, rsm, st>>>(v, pm, op->Nx, P, sc.Zs, sc.Zs, lt, nullptr);
    const int C = pick_col_tile(op->Ny, sizeof(double2), 2);
    const size_t csm = col_smem(op->Ny, C, 2, sizeof(double2));
    dim3 g((op->ncol + C - 1) / C, count);
    k_col_spec<Rout><<<g, 256, csm, st>>>(v, sc.Zs, spec, C, (op->fast || op->fast1024) ? 1 : 0, op->real_spec ? 1 : 0);
}

static void set_build_attributes() {
    allow_max_smem(k_row_fwd<double, LoadTable>);
    allow_max_smem(k_col_spec<float>);
    allow_max_smem(k_col_spec<double>);
}

template <typename Rout>
static gj_status build_spectra(gj_op *op, cudaStream_t st) {
    gj_setup_scratch_impl *sc = nullptr;
    gj_status rc = scratch_alloc(op, op->nz, &sc);
    if (rc != GJ_OK) return rc;
    set_build_attributes();
    build_layers<Rout>(op, *sc, 0, op->nz, static_cast<cpx<Rout> *>(op->spec), st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    scratch_free(sc);
    if (e != cudaSuccess) return cuda_fail(e, "spectra setup");
    return GJ_OK;
}

void recompute_layer(const gj_op *op, int r, cudaStream_t st) {
    if (op->prec == GJ_FP64)
        build_layers<double>(op, *op->scratch, r, 1, static_cast<cpx<double> *>(op->spec), st);
    else
        build_layers<float>(op, *op->scratch, r, 1, static_cast<cpx<float> *>(op->spec), st);
}

}  // namespace gj

using namespace gj;

extern "C" gj_status gj_bttb_setup_ex(const gj_grid *grid, gj_field field, const gj_mag *mag, gj_precision prec,
                                      int Npad_y, int Npad_x, int flags, gj_stream_t stream, gj_op **out) {
    if (!out) { set_error("gj_bttb_setup: out is NULL"); return GJ_ERR_ARG; }
    if (flags & ~GJ_SETUP_RECOMPUTE_SPECTRA) { set_error("gj_bttb_setup_ex: unknown flags"); return GJ_ERR_ARG; }
    *out = nullptr;
    if (!grid) { set_error("gj_bttb_setup: grid is NULL"); return GJ_ERR_ARG; }
    const gj_grid &G = *grid;
    if (G.sx < 1 || G.sy < 1 || G.nx < 1 || G.ny < 1 || G.nz < 1) {
        set_error("gj_bttb_setup: sizes must be >= 1"); return GJ_ERR_ARG;
    }
    if (!(G.dx > 0) || !(G.dy > 0) || !G.z_edges) {
        set_error("gj_bttb_setup: dx, dy must be > 0 and z_edges set"); return GJ_ERR_ARG;
    }
    for (int k = 0; k < G.nz; ++k)
        if (!(G.z_edges[k + 1] > G.z_edges[k])) { set_error("gj_bttb_setup: z_edges must increase"); return GJ_ERR_ARG; }
    if (!(G.station_z <= G.z_edges[0])) {
        set_error("gj_bttb_setup: stations must lie at or above the top of the mesh"); return GJ_ERR_ARG;
    }
    if (field != GJ_GRAVITY && field != GJ_MAGNETIC) { set_error("gj_bttb_setup: bad field"); return GJ_ERR_ARG; }
    if (field == GJ_MAGNETIC && !mag) { set_error("gj_bttb_setup: magnetic field needs gj_mag"); return GJ_ERR_ARG; }
    if (prec != GJ_FP64 && prec != GJ_FP32_MIXED) { set_error("gj_bttb_setup: bad precision"); return GJ_ERR_ARG; }
    const int minx = G.sx + G.nx - 1, miny = G.sy + G.ny - 1;
    int Nx = Npad_x > 0 ? Npad_x : autotune_size(minx);
    int Ny = Npad_y > 0 ? Npad_y : autotune_size(miny);
    if (Nx < minx || Ny < miny) {
        set_error("gj_bttb_setup: padded size must be >= stations + prisms - 1 in each direction");
        return GJ_ERR_ARG;
    }
    gj_op *op = new (std::nothrow) gj_op();
    if (!op) { set_error("gj_bttb_setup: host allocation failed"); return GJ_ERR_OOM; }
    if (!plan_size(Nx, op->px) || !plan_size(Ny, op->py)) {
        delete op;
        set_error("gj_bttb_setup: padded size unsupported (must be <= 2048 with prime factors <= 17)");
        return GJ_ERR_UNSUPPORTED;
    }
    op->sx = G.sx; op->sy = G.sy; op->nx = G.nx; op->ny = G.ny; op->nz = G.nz;
    op->off_x = G.off_x; op->off_y = G.off_y; op->dx = G.dx; op->dy = G.dy; op->station_z = G.station_z;
    op->z_edges.assign(G.z_edges, G.z_edges + G.nz + 1);
    op->field = field;
    op->mag = mag ? *mag : gj_mag{0, 0, 0};
    op->prec = prec;
    op->Nx = Nx; op->Ny = Ny; op->ncol = Nx / 2 + 1;
    const size_t cs = 2 * elem_bytes(prec);
    op->P_row = pick_row_pairs(Nx, cs);
    op->C_col = pick_col_tile(Ny, cs, 3);
    op->L_grp = 4;
    op->recompute = (flags & GJ_SETUP_RECOMPUTE_SPECTRA) != 0;
    op->fast = !op->recompute && fast_eligible(op);
    if (op->fast) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        op->col_grid = std::max(1, sms);
        const int ci = fast_col_items(Ny, G.nz);
        const long long warps = (long long)op->col_grid * f512::CWARPS;
        op->slots = std::max(fast_slots(1, 257, ci, warps), fast_slots(2, 257, ci, warps));
        // gravity over a station grid that covers the prisms with no offset: the table
        // is even in both offsets, so its spectrum is real
        op->real_spec = field == GJ_GRAVITY && G.sx == G.nx && G.sy == G.ny && G.off_x == 0 && G.off_y == 0;
    }
    op->fast1024 = !op->recompute && fast1024_eligible(op);
    if (op->fast1024) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        op->col_grid = std::max(1, sms);
        const long long warps = (long long)op->col_grid * f1024::CWF;
        op->slots = std::max(fast_slots(1, op->ncol, G.nz, warps), fast_slots(2, op->ncol, G.nz, warps));
        op->real_spec = field == GJ_GRAVITY && G.sx == G.nx && G.sy == G.ny && G.off_x == 0 && G.off_y == 0;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    gj_status rc;
    cudaError_t e;
    if ((rc = upload_twiddles(Nx, prec, &op->twx)) != GJ_OK) goto fail;
    if ((rc = upload_twiddles(Ny, prec, &op->twy)) != GJ_OK) goto fail;
    op->spec_bytes = op->real_spec ? (size_t)G.nz * op->ncol * even_spec_len(Ny) * (cs / 2)
                                   : (size_t)(op->recompute ? 1 : G.nz) * Ny * op->ncol * cs;
    if ((e = cudaMalloc(&op->spec, op->spec_bytes)) != cudaSuccess) { rc = cuda_fail(e, "spectra"); goto fail; }
    // the even spectra's padding entries stay zero
    if (op->real_spec && (e = cudaMemset(op->spec, 0, op->spec_bytes)) != cudaSuccess) {
        rc = cuda_fail(e, "spectra");
        goto fail;
    }
    if (op->recompute) {
        // one layer's spectrum plus the build's work buffers for one layer, kept
        if ((rc = scratch_alloc(op, 1, &op->scratch)) != GJ_OK) goto fail;
        set_build_attributes();
    } else {
        rc = (prec == GJ_FP64) ? build_spectra<double>(op, st) : build_spectra<float>(op, st);
        if (rc != GJ_OK) goto fail;
    }
    if (!op->fast && !op->fast1024) {
        const size_t zb = (size_t)G.nz * G.ny * op->ncol * cs;
        const size_t yb = (size_t)Ny * op->ncol * cs;
        const size_t wb = (size_t)std::max(G.sy, 1) * op->ncol * cs;
        op->ws_bytes = zb + yb + wb;
        if ((e = cudaMalloc(&op->Z, zb)) != cudaSuccess) { rc = cuda_fail(e, "workspace"); goto fail; }
        if ((e = cudaMalloc(&op->Y, yb)) != cudaSuccess) { rc = cuda_fail(e, "workspace"); goto fail; }
        if ((e = cudaMalloc(&op->W, wb)) != cudaSuccess) { rc = cuda_fail(e, "workspace"); goto fail; }
    } else {
        // transposed intermediates [r][kx][Ny/2], partials [kx][slots][Ny], counters
        const size_t zb = (size_t)G.nz * op->ncol * (Ny / 2) * cs;
        const size_t wb = (size_t)op->ncol * (Ny / 2) * cs;
        const size_t pb = (size_t)op->ncol * op->slots * Ny * cs;
        const size_t yb = pb + op->ncol * sizeof(int) + 64;
        op->ws_bytes = zb + wb + yb;
        if ((e = cudaMalloc(&op->Z, zb)) != cudaSuccess) { rc = cuda_fail(e, "workspace"); goto fail; }
        if ((e = cudaMalloc(&op->W, wb)) != cudaSuccess) { rc = cuda_fail(e, "workspace"); goto fail; }
        if ((e = cudaMalloc(&op->V, wb)) != cudaSuccess) { rc = cuda_fail(e, "workspace"); goto fail; }
        if ((e = cudaMalloc(&op->Y, yb)) != cudaSuccess) { rc = cuda_fail(e, "workspace"); goto fail; }
        op->ws_bytes += wb;
        // rows beyond the prisms / stations must read as zero; counters start at zero
        if ((e = cudaMemset(op->Z, 0, zb)) != cudaSuccess) { rc = cuda_fail(e, "workspace"); goto fail; }
        if ((e = cudaMemset(op->W, 0, wb)) != cudaSuccess) { rc = cuda_fail(e, "workspace"); goto fail; }
        if ((e = cudaMemset(op->V, 0, wb)) != cudaSuccess) { rc = cuda_fail(e, "workspace"); goto fail; }
        if ((e = cudaMemset(op->Y, 0, yb)) != cudaSuccess) { rc = cuda_fail(e, "workspace"); goto fail; }
        op->P = op->Y;
        op->cnt = reinterpret_cast<int *>(static_cast<char *>(op->Y) + pb);
        op->err = op->cnt + op->ncol + 8;
        const size_t tb = (size_t)(op->fast ? f512::TabTw<float>::WORDS : f1024::Tab1024<float>::WORDS) * sizeof(float2);
        if ((e = cudaMalloc(&op->twtab, tb)) != cudaSuccess) { rc = cuda_fail(e, "twiddle table"); goto fail; }
        if (op->fast)  // from the W512 table of the rows (N_x = 512 on this path, whatever N_y)
            f512::k_build_twtab<float><<<1, 256, 0, st>>>(static_cast<float2 *>(op->twtab),
                                                        static_cast<const float2 *>(op->twx));
        else  // from the W1024 table of the columns
            f1024::k_build_tab1024<float><<<1, 256, 0, st>>>(static_cast<float2 *>(op->twtab),
                                                           static_cast<const float2 *>(op->twy));
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { rc = cuda_fail(e, "twiddle table"); goto fail; }
    }
    *out = op;
    return GJ_OK;
fail:
    free_op_memory(op);
    delete op;
    return rc;
}

extern "C" gj_status gj_bttb_setup(const gj_grid *grid, gj_field field, const gj_mag *mag, gj_precision prec,
                                   int Npad_y, int Npad_x, gj_stream_t stream, gj_op **out) {
    return gj_bttb_setup_ex(grid, field, mag, prec, Npad_y, Npad_x, 0, stream, out);
}

extern "C" gj_status gj_op_tune(gj_op *op, int P_row, int C_col, int L_grp, int radix_order) {
    if (!op) { set_error("gj_op_tune: NULL operator"); return GJ_ERR_ARG; }
    int dev = 0, optin = 48 * 1024;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t cs = 2 * elem_bytes(op->prec);
    const size_t room = (size_t)optin - 1024;  // the kernels' static reduction scratch
    if (P_row > 0 && (P_row > 64 || row_smem(op->Nx, P_row, cs) > room)) {
        set_error("gj_op_tune: P_row too large for shared memory"); return GJ_ERR_ARG;
    }
    if (C_col > 0 && (C_col > 64 || col_smem(op->Ny, C_col, 3, cs) > room)) {
        set_error("gj_op_tune: C_col too large for shared memory"); return GJ_ERR_ARG;
    }
    if (L_grp > 0 && L_grp > op->nz) { set_error("gj_op_tune: L_grp above nz"); return GJ_ERR_ARG; }
    FftPlanDev px = op->px, py = op->py;
    if (radix_order >= 0 && (!plan_size(op->Nx, px, radix_order) || !plan_size(op->Ny, py, radix_order))) {
        set_error("gj_op_tune: radix_order must be 0, 1 or 2"); return GJ_ERR_ARG;
    }
    if (P_row > 0) op->P_row = P_row;
    if (C_col > 0) op->C_col = C_col;
    if (L_grp > 0) op->L_grp = L_grp;
    if (radix_order >= 0) op->radix_order = radix_order;
    op->px = px;
    op->py = py;
    return GJ_OK;
}

extern "C" gj_status gj_op_info(const gj_op *op, gj_op_info_t *info) {
    if (!op || !info) { set_error("gj_op_info: NULL argument"); return GJ_ERR_ARG; }
    info->sx = op->sx; info->sy = op->sy; info->nx = op->nx; info->ny = op->ny; info->nz = op->nz;
    info->Nx = op->Nx; info->Ny = op->Ny; info->ncol = op->ncol;
    info->field = op->field; info->precision = op->prec;
    info->spectrum_bytes = (int64_t)op->spec_bytes;
    info->workspace_bytes = (int64_t)op->ws_bytes;
    info->fast_path = op->fast ? 1 : (op->fast1024 ? 2 : 0);
    info->P_row = op->P_row; info->C_col = op->C_col; info->L_grp = op->L_grp;
    info->radix_order = op->radix_order;
    info->recompute = op->recompute ? 1 : 0;
    return GJ_OK;
}

extern "C" void gj_op_destroy(gj_op *op) {
    if (!op) return;
    cudaDeviceSynchronize();
    free_op_memory(op);
    delete op;
}
