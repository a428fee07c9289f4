// Regularised reweighted CG joint solve (Eq. RRCG:1-8) with Lp reweighting
// (Eq. W, Eq. WL), the Gramian coupling in the original space (RRCG:2-3),
// bounds (Sec. 2.5), the chi^2 stop (Eq. chi2) and the alpha schedule
// (Eq. regpara).  All vector work is fused into the prologues and epilogues of
// the FFT row passes; the scalars stay on the device.
//
// One loop body (iteration k -> k+1), both fields in every launch:
//   adjoint:  rows of v = W_d r~ -> columns -> conj-spectrum columns -> rows with
//             l = W^-1 A^T v + alpha (W m - W m_apr) + lambda l_G      (RRCG:4)
//   forward:  rows of p = l + beta p_prev, x = W^-1 p -> columns -> rows with
//             ||A~ p||^2                                              (RRCG:5-6)
//   scalars:  s = (p, l) / (||A~p||^2 + (alpha + lambda)||p||^2)
//   forward:  rows with m <- clip(m - s W^-1 p) and the Gramian sums -> columns
//             -> rows with r~ = W_d (A m - d), Phi = ||r~||^2          (RRCG:7-8, 1)
//   scalars:  chi^2 flags, alpha freeze/decay, stop flag
// The first forward of m_0 and its scalars run once when the solver is created.
#include <math.h>
#include <stddef.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include "fast_launch.cuh"
#include "view.cuh"

namespace gj {

struct SolverDev {
    int k, done, status, pending_update;
    int sat[2];
    int kmax, stop_on_chi2, per_field;
    int anchor;           // GJ_ANCHOR_*
    int gspace;           // GJ_GRAMIAN_*
    int p[2];
    double eps2;
    double alpha[2], q[2], alpha_min[2], lam[2], lo[2], hi[2];
    double chi2_target[2];
    double s[2], beta[2];
    double ll_prev[2];
    double phi_last[2], SG_last;
    // accumulators, zeroed after use
    double G[3];          // (m1,m1), (m2,m2), (m1,m2) of the current models
    double phi[2];        // ||r~||^2
    double ll[2];         // ||l||^2
    double pl[2], pp[2];  // (p,l), ||p||^2
    double qq[2];         // ||A~ p||^2
    gj_rrcg_hist *hist;
};

template <typename R>
struct FieldVecs {
    R *m[2];
    R *p[2];
    R *l[2];
    R *v[2];               // W_d r~ (s values)
    const R *wd[2];        // 1 / sigma
    const R *dobs[2];
    const R *mapr[2];      // may be null
    const R *wdep[2];      // nz values
    const R *iwdep[2];     // 1 / wdep, nz values
    const R *whard[2];     // may be null
    R *mtp[2];             // W_{k-1} m_{k-1} (previous-model anchor only), else null
};

template <typename R> __device__ __forceinline__ R rsqrt_t(R x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

// Diagonal of W = W_depth W_hard W_L at cell c of layer r (Eq. W, Eq. WL).
template <typename R>
__device__ __forceinline__ R weight(const FieldVecs<R> &F, int i, int p, R eps2, int r, size_t c, R m) {
    R w = F.wdep[i][r];
    if (F.whard[i]) w *= F.whard[i][c];
    if (p == 1) {
        const R d = m - (F.mapr[i] ? F.mapr[i][c] : R(0));
        w *= rsqrt_t<R>(sqrt(d * d + eps2));
    }
    return w;
}

// The L1 reweighting factor of Eq. WL and its reciprocal for p = 1 (1 for p = 2):
// ((m - m_apr)^2 + eps^2)^(-1/4) and ((m - m_apr)^2 + eps^2)^(1/4).
template <typename R>
__device__ __forceinline__ void lp_factors(int p, R d, R eps2, R &wl, R &inv_wl) {
    if (p == 1) {
        const R q = sqrt(d * d + eps2);
        wl = rsqrt_t<R>(q);
        inv_wl = sqrt(q);
    } else {
        wl = R(1);
        inv_wl = R(1);
    }
}
// One hardware reciprocal square root (relative error about 1e-7; arguments below
// FLT_MIN flush to zero).  Its arguments here are d^2 + eps^2 and (d^2 + eps^2)^-1/2.
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// FP32: two reciprocal square roots, u = q^-1/2, q^1/4 = u^-1/2, q^-1/4 = u q^1/4
template <>
__device__ __forceinline__ void lp_factors<float>(int p, float d, float eps2, float &wl, float &inv_wl) {
    if (p == 1) {
        const float u = rsqrt_approx(d * d + eps2);
        inv_wl = rsqrt_approx(u);
        wl = u * inv_wl;
    } else {
        wl = 1.0f;
        inv_wl = 1.0f;
    }
}

// Forward of m with the pending model update (RRCG:7-8 and the bounds) and the
// Gramian sums of the updated models.
template <typename R, bool OPT = true>
struct ProModel {
    FieldVecs<R> F;
    SolverDev *S;
    int nx, ny;
    // per-thread
    int upd, pw[2], gsp;
    R s[2], lo[2], hi[2], eps2;
    R acc[3];
    __device__ void init() {
        upd = S->pending_update;
        gsp = S->gspace;
        eps2 = (R)S->eps2;
        for (int i = 0; i < 2; ++i) {
            s[i] = (R)S->s[i]; lo[i] = (R)S->lo[i]; hi[i] = (R)S->hi[i]; pw[i] = S->p[i];
        }
        acc[0] = acc[1] = acc[2] = 0;
    }
    __device__ __forceinline__ void fetch(int la, int lb, bool, int j, R &a, R &b) {
        const size_t c = (size_t)la * nx + j;
        const int r = la / ny;
        R mv[2], gv[2];
        for (int i = 0; i < 2; ++i) {
            R mi = F.m[i][c];
            if (upd) {
                const R w = weight(F, i, pw[i], eps2, r, c, mi);
                if (OPT && F.mtp[i]) F.mtp[i][c] = w * mi;  // W_k m_k, the next anchor
                mi = mi - s[i] * F.p[i][c] / w;
                mi = fmin(fmax(mi, lo[i]), hi[i]);
                F.m[i][c] = mi;
            }
            mv[i] = mi;
            gv[i] = gsp ? weight(F, i, pw[i], eps2, r, c, mi) * mi : mi;  // Gramian space
        }
        acc[0] += gv[0] * gv[0];
        acc[1] += gv[1] * gv[1];
        acc[2] += gv[0] * gv[1];
        a = mv[0];
        b = mv[1];
    }
    // rows a line needs in every launch (m, p), staged ahead by the persistent row
    // pass as pre[a][field][j]; the optional rows are read in place
    static constexpr int NPRE = 2;
    __device__ const R *pre_src(int a, int i) const { return a == 0 ? F.m[i] : (upd ? F.p[i] : nullptr); }
    // batched form: every load of the K elements is issued before any store
    template <int K, bool PRE = false>
    __device__ __forceinline__ void fetch_batch(int la, int, bool, int j0, int stride, int n, R (&a)[K], R (&b)[K],
                                                const R *pre = nullptr) {
        const size_t c0 = (size_t)la * nx;
        const int r = la / ny;
        R mv[2][K], pv[2][K], wh[2][K], ma[2][K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + k * stride;
            const bool ok = j < n;
            const size_t c = c0 + j;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                mv[i][k] = ok ? (PRE ? pre[i * f512::H + j] : F.m[i][c]) : R(0);
                pv[i][k] = (ok && upd) ? (PRE ? pre[(2 + i) * f512::H + j] : F.p[i][c]) : R(0);
                wh[i][k] = (ok && OPT && F.whard[i]) ? F.whard[i][c] : R(1);
                ma[i][k] = (ok && OPT && F.mapr[i]) ? F.mapr[i][c] : R(0);
            }
        }
        R wd[2], iwd[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) { wd[i] = F.wdep[i][r]; iwd[i] = F.iwdep[i][r]; }
        if (upd) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int j = j0 + k * stride;
                if (j >= n) continue;
                const size_t c = c0 + j;
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    R wl, iwl;
                    lp_factors<R>(pw[i], mv[i][k] - ma[i][k], eps2, wl, iwl);
                    R inv_w = iwl * iwd[i];
                    if (OPT && F.whard[i]) inv_w /= wh[i][k];
                    if (OPT && F.mtp[i]) F.mtp[i][c] = wd[i] * wh[i][k] * wl * mv[i][k];  // W_k m_k, the next anchor
                    R mi = mv[i][k] - s[i] * pv[i][k] * inv_w;
                    mi = fmin(fmax(mi, lo[i]), hi[i]);
                    F.m[i][c] = mi;
                    mv[i][k] = mi;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            R gv[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                gv[i] = mv[i][k];
                if (gsp) {  // the Gramian of the weighted models W(m) m
                    R wl, iwl;
                    lp_factors<R>(pw[i], mv[i][k] - ma[i][k], eps2, wl, iwl);
                    gv[i] = wd[i] * wh[i][k] * wl * mv[i][k];
                }
            }
            acc[0] += gv[0] * gv[0];
            acc[1] += gv[1] * gv[1];
            acc[2] += gv[0] * gv[1];
            a[k] = mv[0][k];
            b[k] = mv[1][k];
        }
    }
    __device__ void flush(double *red) { block_accumulate<3>(acc, S->G, red); }
};

// Residual epilogue: r~ = W_d (A m - d), v = W_d r~, Phi partials (RRCG:1).
template <typename R>
struct EpiResidual {
    FieldVecs<R> F;
    SolverDev *S;
    int sx;
    R acc[2];
    __device__ void init() { acc[0] = acc[1] = 0; }
    __device__ __forceinline__ void store(int la, int, bool, int j, R a, R b) {
        const size_t t = (size_t)la * sx + j;
        const R y[2] = {a, b};
        for (int i = 0; i < 2; ++i) {
            const R w = F.wd[i][t];
            const R rt = w * (y[i] - F.dobs[i][t]);
            acc[i] += rt * rt;
            F.v[i][t] = w * rt;
        }
    }
    // fused form, in two steps so that the loads can be issued before the transform:
    // resid_load fetches W_d and d; resid_apply takes y in a, b and returns v = W_d r~
    template <int K>
    __device__ __forceinline__ void resid_load(int la, int j0, int stride, int n, R (&w)[2][K], R (&d)[2][K]) const {
        const size_t t0 = (size_t)la * sx;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + k * stride;
            const bool ok = j < n;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                w[i][k] = ok ? F.wd[i][t0 + j] : R(0);
                d[i][k] = ok ? F.dobs[i][t0 + j] : R(0);
            }
        }
    }
    template <int K>
    __device__ __forceinline__ void resid_apply(int j0, int stride, int n, const R (&w)[2][K], const R (&d)[2][K],
                                                R (&a)[K], R (&b)[K]) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + k * stride;
            const bool ok = j < n;
            const R r0 = w[0][k] * (a[k] - d[0][k]);
            const R r1 = w[1][k] * (b[k] - d[1][k]);
            if (ok) {
                acc[0] += r0 * r0;
                acc[1] += r1 * r1;
            }
            a[k] = ok ? w[0][k] * r0 : R(0);
            b[k] = ok ? w[1][k] * r1 : R(0);
        }
    }
    template <int K>
    __device__ __forceinline__ void store_batch(int la, int, bool, int j0, int stride, int n, const R (&a)[K],
                                                const R (&b)[K]) {
        const size_t t0 = (size_t)la * sx;
        R w[2][K], d[2][K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + k * stride;
            const bool ok = j < n;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                w[i][k] = ok ? F.wd[i][t0 + j] : R(0);
                d[i][k] = ok ? F.dobs[i][t0 + j] : R(0);
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + k * stride;
            if (j >= n) continue;
            const R y[2] = {a[k], b[k]};
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const R rt = w[i][k] * (y[i] - d[i][k]);
                acc[i] += rt * rt;
                F.v[i][t0 + j] = w[i][k] * rt;
            }
        }
    }
    __device__ void flush(double *red) { block_accumulate<2>(acc, S->phi, red); }
};

template <typename R>
struct LoadPair {
    const R *x0;
    const R *x1;
    int pitch;
    __device__ void init() {}
    __device__ __forceinline__ void fetch(int la, int lb, bool, int j, R &a, R &b) const {
        a = x0[(size_t)la * pitch + j];
        b = x1[(size_t)lb * pitch + j];
    }
    template <int K>
    __device__ __forceinline__ void fetch_batch(int la, int lb, bool, int j0, int stride, int n, R (&a)[K],
                                                R (&b)[K]) const {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + k * stride;
            a[k] = j < n ? x0[(size_t)la * pitch + j] : R(0);
            b[k] = j < n ? x1[(size_t)lb * pitch + j] : R(0);
        }
    }
    __device__ void flush(double *) {}
};

// Gradient epilogue (RRCG:2-4): l = W^-1 A^T v + alpha (W m - W m_apr) + lambda l_G.
template <typename R, bool OPT = true>
struct EpiGradient {
    FieldVecs<R> F;
    SolverDev *S;
    int nx, ny;
    R alpha[2], lam[2], eps2, g11, g22, g12;
    int pw[2], gsp, prev;
    R acc[2];
    __device__ void init() {
        for (int i = 0; i < 2; ++i) { alpha[i] = (R)S->alpha[i]; lam[i] = (R)S->lam[i]; pw[i] = S->p[i]; }
        eps2 = (R)S->eps2;
        g11 = (R)S->G[0]; g22 = (R)S->G[1]; g12 = (R)S->G[2];
        gsp = S->gspace;
        prev = S->anchor == GJ_ANCHOR_PREVIOUS && S->k > 0;  // W_{k-1} m_{k-1} exists from k = 1
        acc[0] = acc[1] = 0;
    }
    __device__ __forceinline__ void store(int la, int, bool, int j, R a, R b) {
        const size_t c = (size_t)la * nx + j;
        const int r = la / ny;
        const R mm[2] = {F.m[0][c], F.m[1][c]};
        const R w[2] = {weight(F, 0, pw[0], eps2, r, c, mm[0]), weight(F, 1, pw[1], eps2, r, c, mm[1])};
        // ascent directions in the chosen space (RRCG:2-3 or Eq. steepestascenta/b)
        const R u0 = gsp ? w[0] * mm[0] : mm[0], u1 = gsp ? w[1] * mm[1] : mm[1];
        const R lG[2] = {g22 * u0 - g12 * u1, g11 * u1 - g12 * u0};
        const R g[2] = {a, b};
        for (int i = 0; i < 2; ++i) {
            const R ma = (OPT && F.mapr[i]) ? F.mapr[i][c] : R(0);
            const R anchor = (OPT && prev) ? F.mtp[i][c] : w[i] * ma;
            const R li = g[i] / w[i] + alpha[i] * (w[i] * mm[i] - anchor) + lam[i] * lG[i];
            F.l[i][c] = li;
            acc[i] += li * li;
        }
    }
    static constexpr int NPRE = 1;  // m, staged ahead by the persistent row pass
    __device__ const R *pre_src(int, int i) const { return F.m[i]; }
    template <int K, bool PRE = false>
    __device__ __forceinline__ void store_batch(int la, int, bool, int j0, int stride, int n, const R (&a)[K],
                                                const R (&b)[K], const R *pre = nullptr) {
        const size_t c0 = (size_t)la * nx;
        const int r = la / ny;
        R mv[2][K], wh[2][K], ma[2][K], an[2][K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + k * stride;
            const bool ok = j < n;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                mv[i][k] = ok ? (PRE ? pre[i * f512::H + j] : F.m[i][c0 + j]) : R(0);
                wh[i][k] = (ok && OPT && F.whard[i]) ? F.whard[i][c0 + j] : R(1);
                ma[i][k] = (ok && OPT && F.mapr[i]) ? F.mapr[i][c0 + j] : R(0);
                an[i][k] = (ok && OPT && prev) ? F.mtp[i][c0 + j] : R(0);
            }
        }
        R wd[2], iwd[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) { wd[i] = F.wdep[i][r]; iwd[i] = F.iwdep[i][r]; }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + k * stride;
            if (j >= n) continue;
            R w[2], inv_w[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                R wl, iwl;
                lp_factors<R>(pw[i], mv[i][k] - ma[i][k], eps2, wl, iwl);
                w[i] = wd[i] * wl;
                inv_w[i] = iwl * iwd[i];
                if (OPT && F.whard[i]) { w[i] *= wh[i][k]; inv_w[i] /= wh[i][k]; }
            }
            const R u0 = gsp ? w[0] * mv[0][k] : mv[0][k], u1 = gsp ? w[1] * mv[1][k] : mv[1][k];
            const R lG[2] = {g22 * u0 - g12 * u1, g11 * u1 - g12 * u0};
            const R g[2] = {a[k], b[k]};
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const R anchor = (OPT && prev) ? an[i][k] : w[i] * ma[i][k];
                const R li = g[i] * inv_w[i] + alpha[i] * (w[i] * mv[i][k] - anchor) + lam[i] * lG[i];
                F.l[i][c0 + j] = li;
                acc[i] += li * li;
            }
        }
    }
    __device__ void flush(double *red) { block_accumulate<2>(acc, S->ll, red); }
};

// Search direction (RRCG:5) and the forward input W^-1 p.
template <typename R, bool OPT = true>
struct ProDirection {
    FieldVecs<R> F;
    SolverDev *S;
    int nx, ny;
    R beta[2], eps2;
    int first, pw[2];
    R acc[4];  // (p,l)_0, (p,l)_1, ||p||^2_0, ||p||^2_1
    __device__ void init() {
        first = S->k == 0;
        eps2 = (R)S->eps2;
        for (int i = 0; i < 2; ++i) pw[i] = S->p[i];
        if (S->per_field) {
            for (int i = 0; i < 2; ++i) beta[i] = S->ll_prev[i] > 0 ? (R)(S->ll[i] / S->ll_prev[i]) : R(0);
        } else {
            const double den = S->ll_prev[0] + S->ll_prev[1];
            const R b = den > 0 ? (R)((S->ll[0] + S->ll[1]) / den) : R(0);
            beta[0] = beta[1] = b;
        }
        acc[0] = acc[1] = acc[2] = acc[3] = 0;
    }
    __device__ __forceinline__ void fetch(int la, int, bool, int j, R &a, R &b) {
        const size_t c = (size_t)la * nx + j;
        const int r = la / ny;
        R x[2];
        for (int i = 0; i < 2; ++i) {
            const R li = F.l[i][c];
            const R pi = first ? li : li + beta[i] * F.p[i][c];
            F.p[i][c] = pi;
            acc[i] += pi * li;
            acc[2 + i] += pi * pi;
            x[i] = pi / weight(F, i, pw[i], eps2, r, c, F.m[i][c]);
        }
        a = x[0];
        b = x[1];
    }
    static constexpr int NPRE = 3;  // l, p, m, staged ahead by the persistent row pass
    __device__ const R *pre_src(int a, int i) const {
        return a == 0 ? F.l[i] : (a == 1 ? (first ? nullptr : F.p[i]) : F.m[i]);
    }
    template <int K, bool PRE = false>
    __device__ __forceinline__ void fetch_batch(int la, int, bool, int j0, int stride, int n, R (&a)[K], R (&b)[K],
                                                const R *pre = nullptr) {
        const size_t c0 = (size_t)la * nx;
        const int r = la / ny;
        R lv[2][K], pv[2][K], mv[2][K], wh[2][K], ma[2][K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + k * stride;
            const bool ok = j < n;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                lv[i][k] = ok ? (PRE ? pre[i * f512::H + j] : F.l[i][c0 + j]) : R(0);
                pv[i][k] = (ok && !first) ? (PRE ? pre[(2 + i) * f512::H + j] : F.p[i][c0 + j]) : R(0);
                mv[i][k] = ok ? (PRE ? pre[(4 + i) * f512::H + j] : F.m[i][c0 + j]) : R(0);
                wh[i][k] = (ok && OPT && F.whard[i]) ? F.whard[i][c0 + j] : R(1);
                ma[i][k] = (ok && OPT && F.mapr[i]) ? F.mapr[i][c0 + j] : R(0);
            }
        }
        R iwd[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) iwd[i] = F.iwdep[i][r];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + k * stride;
            const bool ok = j < n;
            R x[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const R pi = first ? lv[i][k] : lv[i][k] + beta[i] * pv[i][k];
                R wl, iwl;
                lp_factors<R>(pw[i], mv[i][k] - ma[i][k], eps2, wl, iwl);
                R inv_w = iwl * iwd[i];
                if (OPT && F.whard[i]) inv_w /= wh[i][k];
                if (ok) {
                    F.p[i][c0 + j] = pi;
                    acc[i] += pi * lv[i][k];
                    acc[2 + i] += pi * pi;
                }
                x[i] = ok ? pi * inv_w : R(0);
            }
            a[k] = x[0];
            b[k] = x[1];
        }
    }
    __device__ void flush(double *red) {
        // pl and pp are adjacent in SolverDev: one pass adds all four sums
        static_assert(offsetof(SolverDev, pp) == offsetof(SolverDev, pl) + 2 * sizeof(double), "layout");
        block_accumulate<4>(acc, S->pl, red);
    }
};

// ||A~ p||^2 = ||W_d A (W^-1 p)||^2 partials (RRCG:6).
template <typename R>
struct EpiQNorm {
    FieldVecs<R> F;
    SolverDev *S;
    int sx;
    R acc[2];
    __device__ void init() { acc[0] = acc[1] = 0; }
    __device__ __forceinline__ void store(int la, int, bool, int j, R a, R b) {
        const size_t t = (size_t)la * sx + j;
        const R q0 = F.wd[0][t] * a, q1 = F.wd[1][t] * b;
        acc[0] += q0 * q0;
        acc[1] += q1 * q1;
    }
    // batched form (the 512 kernels): prefetch loads W_d of line la, elements
    // lane + 32 k, before the transform; store_batch(j0 = lane or lane + 128) uses them
    R wq[2][8];
    __device__ __forceinline__ void prefetch(int la, int, bool, int lane, int n) {
        const size_t t0 = (size_t)la * sx;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int j = lane + 32 * k;
            wq[0][k] = j < n ? F.wd[0][t0 + j] : R(0);
            wq[1][k] = j < n ? F.wd[1][t0 + j] : R(0);
        }
    }
    template <int K>
    __device__ __forceinline__ void store_batch(int, int, bool, int j0, int stride, int n, const R (&a)[K],
                                                const R (&b)[K]) {
        const int o = (j0 - (int)(threadIdx.x & 31)) / 32;  // 0 or 4
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + k * stride;
            if (j >= n) continue;
            const R q0 = wq[0][o + k] * a[k], q1 = wq[1][o + k] * b[k];
            acc[0] += q0 * q0;
            acc[1] += q1 * q1;
        }
    }
    __device__ void flush(double *red) { block_accumulate<2>(acc, S->qq, red); }
};

// The one-thread scalar steps run on a shared-memory copy of the solver state: a
// warp copies it in with one coalesced read (instead of a chain of dependent global
// loads), thread 0 takes the step, and the warp copies the state back.
static_assert(sizeof(SolverDev) % sizeof(unsigned long long) == 0 && alignof(SolverDev) == 8,
              "the state copies as 8-byte words");
constexpr int kStateWords = (int)(sizeof(SolverDev) / sizeof(unsigned long long));
__device__ __forceinline__ void state_copy(void *dst, const void *src) {
    for (int i = threadIdx.x; i < kStateWords; i += 32)
        static_cast<unsigned long long *>(dst)[i] = static_cast<const unsigned long long *>(src)[i];
}
template <void (*STEP)(SolverDev *)>
__device__ __forceinline__ void scalar_step_on_copy(SolverDev *S) {
    __shared__ SolverDev sh;
    state_copy(&sh, S);
    __syncwarp();
    if (threadIdx.x == 0) STEP(&sh);
    __syncwarp();
    state_copy(S, &sh);
}

// chi^2 test, alpha schedule and stop (Eq. chi2, Eq. regpara); one thread.
__device__ void scalars_after_residual(SolverDev *S) {
    if (S->done) return;
    const int k = S->k;
    for (int i = 0; i < 2; ++i)
        if (S->phi[i] <= S->chi2_target[i]) S->sat[i] = 1;
    if (k > 0)
        for (int i = 0; i < 2; ++i)
            if (!S->sat[i]) S->alpha[i] = fmax(S->q[i] * S->alpha[i], S->alpha_min[i]);
    const double SG = S->G[0] * S->G[1] - S->G[2] * S->G[2];
    S->phi_last[0] = S->phi[0];
    S->phi_last[1] = S->phi[1];
    S->SG_last = SG;
    if (S->hist) {
        gj_rrcg_hist &h = S->hist[k];
        h.phi[0] = S->phi[0]; h.phi[1] = S->phi[1];
        h.alpha[0] = S->alpha[0]; h.alpha[1] = S->alpha[1];
        h.S_G = SG;
        h.s[0] = h.s[1] = h.beta[0] = h.beta[1] = 0.0;
    }
    S->pending_update = 0;
    if (!isfinite(S->phi[0]) || !isfinite(S->phi[1])) {
        S->status = GJ_ERR_NONFINITE;
        S->done = 1;
        return;
    }
    if ((S->stop_on_chi2 && S->sat[0] && S->sat[1]) || k >= S->kmax) S->done = 1;
    S->phi[0] = S->phi[1] = 0.0;
}

// Step length s_k (RRCG:6); one thread.
__device__ void scalars_after_direction(SolverDev *S) {
    if (S->done) return;
    const int k = S->k;
    double den[2], beta[2];
    for (int i = 0; i < 2; ++i) den[i] = S->qq[i] + (S->alpha[i] + S->lam[i]) * S->pp[i];
    if (S->per_field) {
        for (int i = 0; i < 2; ++i) {
            S->s[i] = den[i] > 0 ? S->pl[i] / den[i] : 0.0;
            beta[i] = (k > 0 && S->ll_prev[i] > 0) ? S->ll[i] / S->ll_prev[i] : 0.0;
        }
    } else {
        const double d = den[0] + den[1];
        const double s = d > 0 ? (S->pl[0] + S->pl[1]) / d : 0.0;
        S->s[0] = S->s[1] = s;
        const double lp = S->ll_prev[0] + S->ll_prev[1];
        beta[0] = beta[1] = (k > 0 && lp > 0) ? (S->ll[0] + S->ll[1]) / lp : 0.0;
    }
    if (S->hist) {
        gj_rrcg_hist &h = S->hist[k];
        h.s[0] = S->s[0]; h.s[1] = S->s[1];
        h.beta[0] = beta[0]; h.beta[1] = beta[1];
    }
    if (!isfinite(S->s[0]) || !isfinite(S->s[1])) {
        S->status = GJ_ERR_NONFINITE;
        S->done = 1;
        return;
    }
    S->ll_prev[0] = S->ll[0];
    S->ll_prev[1] = S->ll[1];
    S->ll[0] = S->ll[1] = 0.0;
    S->pl[0] = S->pl[1] = S->pp[0] = S->pp[1] = 0.0;
    S->qq[0] = S->qq[1] = 0.0;
    S->G[0] = S->G[1] = S->G[2] = 0.0;
    S->pending_update = 1;
    S->k = k + 1;
}

// one warp each (launched as <<<1, 32>>>)
__global__ void k_scalars_after_residual(SolverDev *S) { scalar_step_on_copy<scalars_after_residual>(S); }
__global__ void k_scalars_after_direction(SolverDev *S) { scalar_step_on_copy<scalars_after_direction>(S); }

// The report of the solver state into device memory (one thread): the same fields
// as gj_rrcg_report_get, without a host round trip.
__global__ void k_report(const SolverDev *S, const int *err, gj_rrcg_report *rep) {
    rep->status = S->status;
    if (err && *err != 0 && rep->status == GJ_OK) rep->status = *err;
    rep->iterations = S->k;
    rep->converged = S->sat[0] && S->sat[1];
    rep->satisfied[0] = S->sat[0];
    rep->satisfied[1] = S->sat[1];
    rep->phi[0] = S->phi_last[0];
    rep->phi[1] = S->phi_last[1];
    rep->alpha[0] = S->alpha[0];
    rep->alpha[1] = S->alpha[1];
    rep->S_G = S->SG_last;
}

template <typename R>
__global__ void k_reciprocal(int n, const R *sigma, R *wd) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) wd[i] = R(1) / sigma[i];
}

}  // namespace gj

using namespace gj;

struct ProfilePair { cudaEvent_t a, b; };

struct gj_rrcg {
    const gj_op *op[2];
    gj_precision prec;
    SolverDev *S = nullptr;   // device
    void *buf = nullptr;      // p, l (2 fields each, n), v (2 x s), wd (2 x s)
    const void *dobs[2], *mapr[2], *wdep[2], *whard[2];
    bool prev_anchor = false;
    void *m[2];
    gj_rrcg_hist *hist = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    int profile = 0;
    std::vector<ProfilePair> eager_pairs;   // recorded since the last read
    std::vector<ProfilePair> graph_pairs;   // unused: events inside a graph cannot be timed
    std::vector<ProfilePair> free_pairs;
    bool capturing = false;
    // profiled graph form: the body captured as segments cut around each timed launch
    std::vector<cudaGraph_t> seg_graph;
    std::vector<cudaGraphExec_t> seg_exec;
    cudaStream_t cap_stream = nullptr;   // stream being captured while segmenting
    cudaError_t cap_err = cudaSuccess;
    int grid = 0;  // CTAs of the persistent fast-path launches (0: the operator's, one per SM)
};

namespace gj {

static ProfilePair take_pair(gj_rrcg *sv) {
    ProfilePair p;
    if (!sv->free_pairs.empty()) { p = sv->free_pairs.back(); sv->free_pairs.pop_back(); }
    else { cudaEventCreate(&p.a); cudaEventCreate(&p.b); }
    return p;
}

// Ends the capture in progress, keeps the captured segment, and begins the next.
static void cut_segment(gj_rrcg *sv, cudaStream_t st) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (e == cudaSuccess) sv->seg_graph.push_back(g);
    else if (sv->cap_err == cudaSuccess) sv->cap_err = e;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess && sv->cap_err == cudaSuccess) sv->cap_err = e;
}

template <typename R>
struct SolverLaunch {
    gj_rrcg *sv;
    OpView<R> v0, v1;
    f512::View2<R> V2;
    bool fast = false;
    bool fast1024 = false;  // general row kernels (transposed intermediates) + N_y = 1024 column kernels
    bool rows1024 = false;  // fast1024 with N_x = 1024: the warp-FFT row kernels of fast1024.cuh
    FieldVecs<R> F;
    int P, C, L;
    int grid;  // CTAs of the persistent fast-path launches
    size_t rsm, msm, csm;
    int n_rows_cells, n_rows_st;  // pairs in the cell / station row passes

    void setup() {  // views and launch shapes only (no CUDA calls: safe during capture)
        const gj_op *o = sv->op[0];
        grid = sv->grid > 0 ? sv->grid : o->col_grid;
        v0 = view_of<R>(sv->op[0]);
        v1 = view_of<R>(sv->op[1]);
        if constexpr (std::is_same_v<R, float>) {
            fast = o->fast && sv->op[1]->fast;
            fast1024 = o->fast1024 && sv->op[1]->fast1024;
            rows1024 = fast1024 && o->Nx == 1024;
            if (fast || fast1024) V2 = f512::make_view2<R>(sv->op[0], sv->op[1]);
        }
        const size_t cs = sizeof(cpx<R>);
        P = o->P_row; C = o->C_col; L = o->L_grp;
        rsm = row_smem(o->Nx, P, cs);
        msm = col_smem(o->Ny, C, 3, cs);
        csm = col_smem(o->Ny, C, 2, cs);
        const int n = o->nx * o->ny * o->nz, s = o->sx * o->sy;
        R *b = static_cast<R *>(sv->buf);
        for (int i = 0; i < 2; ++i) {
            F.m[i] = static_cast<R *>(sv->m[i]);
            F.p[i] = b + (size_t)i * n;
            F.l[i] = b + (size_t)(2 + i) * n;
            F.v[i] = b + (size_t)4 * n + (size_t)i * s;
            F.wd[i] = b + (size_t)4 * n + (size_t)(2 + i) * s;
            F.dobs[i] = static_cast<const R *>(sv->dobs[i]);
            F.mapr[i] = static_cast<const R *>(sv->mapr[i]);
            F.wdep[i] = static_cast<const R *>(sv->wdep[i]);
            F.iwdep[i] = b + (size_t)4 * n + (size_t)4 * s + (size_t)i * o->nz;
            F.mtp[i] = sv->prev_anchor ? b + (size_t)4 * n + (size_t)4 * s + (size_t)2 * o->nz + (size_t)i * n : nullptr;
            F.whard[i] = static_cast<const R *>(sv->whard[i]);
        }
    }

    // any optional row (hard weights, a-priori model, previous-model anchor) present:
    // the functors' variants without them skip those loads and factors entirely
    bool opt_rows() const {
        for (int i = 0; i < 2; ++i)
            if (F.whard[i] || F.mapr[i] || F.mtp[i]) return true;
        return false;
    }

    void set_attributes() {
        // Load every kernel of an iteration now: with lazy module loading, the first
        // launch of a kernel inside a stream capture would invalidate the capture.
        cudaFuncAttributes fa;
        cudaFuncGetAttributes(&fa, k_scalars_after_direction);
        cudaFuncGetAttributes(&fa, k_scalars_after_residual);
        if constexpr (std::is_same_v<R, float>) if (fast) {
            using namespace f512;
            set_row_fwd_t_attr<R, ProModel<R, true>>();
            set_row_fwd_t_attr<R, ProDirection<R, true>>();
            set_row_fwd_t_attr<R, ProModel<R, false>>();
            set_row_fwd_t_attr<R, ProDirection<R, false>>();
            set_row_resid_attr<R, EpiResidual<R>, kDataNW>();
            set_row_inv_t_attr<R, EpiGradient<R, true>>();
            set_row_inv_t_attr<R, EpiGradient<R, false>>();
            set_row_inv_attr<R, EpiQNorm<R>, kDataNW, kDataFPW>();
            set_col_attr<R>();
            return;
        }
        if constexpr (std::is_same_v<R, float>) if (fast1024) {
            f1024::set_col_attr<R>();
            f1024::set_row_fwd_attr<R, ProModel<R>>();
            f1024::set_row_fwd_attr<R, ProDirection<R>>();
            f1024::set_row_fwd_attr<R, LoadPair<R>>();
            f1024::set_row_inv_attr<R, EpiResidual<R>>();
            f1024::set_row_inv_attr<R, EpiGradient<R>>();
            f1024::set_row_inv_attr<R, EpiQNorm<R>>();
        }
        allow_max_smem(k_row_fwd<R, ProModel<R>>);
        allow_max_smem(k_row_fwd<R, ProDirection<R>>);
        allow_max_smem(k_row_fwd<R, LoadPair<R>>);
        allow_max_smem(k_row_inv<R, EpiResidual<R>>);
        allow_max_smem(k_row_inv<R, EpiGradient<R>>);
        allow_max_smem(k_row_inv<R, EpiQNorm<R>>);
        allow_max_smem(k_col_fwd_mac<R>);
        allow_max_smem(k_col_inv<R>);
        allow_max_smem(k_col_fft<R>);
        allow_max_smem(k_col_adj<R>);
    }

    // Row passes of the general path over both fields (joint pair maps): the block FFT
    // kernels, or at N_x = 1024 with the N_y = 1024 columns the warp-FFT row kernels.
    template <class Pro>
    void rows_fwd(const PairMap &pm, int n_in, cpx<R> *o0, cpx<R> *o1, const Pro &pro, const int *done,
                  cudaStream_t st) {
        if constexpr (std::is_same_v<R, float>) if (rows1024) {
            f1024::row_fwd<R>(v0, pm, n_in, o0, o1, sv->op[0]->twtab, pro, done, st);
            return;
        }
        k_row_fwd<R, Pro><<<(pm.nlines + P - 1) / P, 256, rsm, st>>>(v0, pm, n_in, P, o0, o1, pro, done);
    }
    template <class Epi>
    void rows_inv(const PairMap &pm, int n_out, const cpx<R> *i0, const cpx<R> *i1, const Epi &epi, const int *done,
                  cudaStream_t st) {
        if constexpr (std::is_same_v<R, float>) if (rows1024) {
            f1024::row_inv<R>(v0, pm, n_out, i0, i1, sv->op[0]->twtab, epi, done, st);
            return;
        }
        k_row_inv<R, Epi><<<(pm.nlines + P - 1) / P, 256, rsm, st>>>(v0, pm, n_out, P, i0, i1, epi, done);
    }

    // Forward columns (Y = sum_r T^_r FFT_y(Z_r)) and inverse columns, both fields.
    void forward_columns(cudaStream_t st) {
        const gj_op *o = sv->op[0];
        if constexpr (std::is_same_v<R, float>) if (fast) {
            ProfilePair pp{};
            if (sv->profile && sv->capturing) {
                cut_segment(sv, st);  // the timed launch gets a segment of its own
            } else if (sv->profile) {
                pp = take_pair(sv);
                cudaEventRecord(pp.a, st);
            }
            f512::col_fwd<R>(V2, grid, &sv->S->done, st);
            if (sv->profile && sv->capturing) {
                cut_segment(sv, st);
            } else if (sv->profile) {
                cudaEventRecord(pp.b, st);
                sv->eager_pairs.push_back(pp);
            }
            return;
        }
        if constexpr (std::is_same_v<R, float>) if (fast1024) {
            ProfilePair pp{};
            if (sv->profile && !sv->capturing) {
                pp = take_pair(sv);
                cudaEventRecord(pp.a, st);
            }
            f1024::col_fwd<R>(V2, grid, &sv->S->done, st);
            if (sv->profile && !sv->capturing) {
                cudaEventRecord(pp.b, st);
                sv->eager_pairs.push_back(pp);
            }
            return;
        }
        const size_t cs = sizeof(cpx<R>);
        cudaMemsetAsync(v0.Y, 0, (size_t)o->Ny * o->ncol * cs, st);
        cudaMemsetAsync(v1.Y, 0, (size_t)o->Ny * o->ncol * cs, st);
        const int nt = (o->ncol + C - 1) / C;
        ProfilePair pp{};
        if (sv->profile && !sv->capturing) {
            pp = take_pair(sv);
            cudaEventRecord(pp.a, st);
        }
        k_col_fwd_mac<R><<<dim3(nt, (o->nz + L - 1) / L, 2), 256, msm, st>>>(v0, v1, C, L, &sv->S->done);
        if (sv->profile && !sv->capturing) {
            cudaEventRecord(pp.b, st);
            sv->eager_pairs.push_back(pp);
        }
        k_col_inv<R><<<dim3(nt, 2), 256, csm, st>>>(v0, v1, C, &sv->S->done);
    }

    void head(cudaStream_t st) {  // forward of (updated) m, residual, chi^2 scalars
        const gj_op *o = sv->op[0];
        const int *done = &sv->S->done;
        if constexpr (std::is_same_v<R, float>) if (fast) {
            using namespace f512;
            if (opt_rows()) {
                ProModel<R, true> pm{F, sv->S, o->nx, o->ny};
                row_fwd_t<R>(V2, grid, o->nz, o->ny, o->nx, 0, pm, done, st);
            } else {
                ProModel<R, false> pm{F, sv->S, o->nx, o->ny};
                row_fwd_t<R>(V2, grid, o->nz, o->ny, o->nx, 0, pm, done, st);
            }
            forward_columns(st);
            // residual, Phi and the residual rows' spectra for the adjoint, in one pass
            EpiResidual<R> er{F, sv->S, o->sx};
            row_resid<R, kDataNW>(V2, o->sy, o->sx, er, done, st);
            k_scalars_after_residual<<<1, 32, 0, st>>>(sv->S);
            return;
        }
        PairMap pc{o->nz * o->ny, 1, o->ny};
        ProModel<R> pm{F, sv->S, o->nx, o->ny};
        rows_fwd(pc, o->nx, v0.Z, v1.Z, pm, done, st);
        forward_columns(st);
        PairMap ps{o->sy, 1, o->sy};
        EpiResidual<R> er{F, sv->S, o->sx};
        rows_inv(ps, o->sx, v0.W, v1.W, er, done, st);
        k_scalars_after_residual<<<1, 32, 0, st>>>(sv->S);
    }

    void body(cudaStream_t st) {
        const gj_op *o = sv->op[0];
        const int *done = &sv->S->done;
        if constexpr (std::is_same_v<R, float>) if (fast) {
            using namespace f512;
            col_adj<R>(V2, grid, done, st);
            if (opt_rows()) {
                EpiGradient<R, true> eg{F, sv->S, o->nx, o->ny};
                row_inv_t<R>(V2, grid, o->nz, o->ny, o->nx, 0, eg, done, st);
                ProDirection<R, true> pd{F, sv->S, o->nx, o->ny};
                row_fwd_t<R>(V2, grid, o->nz, o->ny, o->nx, 0, pd, done, st);
            } else {
                EpiGradient<R, false> eg{F, sv->S, o->nx, o->ny};
                row_inv_t<R>(V2, grid, o->nz, o->ny, o->nx, 0, eg, done, st);
                ProDirection<R, false> pd{F, sv->S, o->nx, o->ny};
                row_fwd_t<R>(V2, grid, o->nz, o->ny, o->nx, 0, pd, done, st);
            }
            forward_columns(st);
            EpiQNorm<R> eq{F, sv->S, o->sx};
            row_inv<R, kDataNW, kDataFPW>(V2, 1, o->sy, o->sy, o->sx, 1, eq, done, st);
            k_scalars_after_direction<<<1, 32, 0, st>>>(sv->S);
            head(st);
            return;
        }
        const int nt = (o->ncol + C - 1) / C;
        PairMap ps{o->sy, 1, o->sy};
        PairMap pc{o->nz * o->ny, 1, o->ny};
        // adjoint: rows of v -> W, columns -> Y, per-layer conj-spectrum columns -> Z
        // (N_y = 1024 column kernels: rows of v -> V, then one persistent column pass)
        LoadPair<R> lv{F.v[0], F.v[1], o->sx};
        bool cols1024 = false;
        if constexpr (std::is_same_v<R, float>) cols1024 = fast1024;
        if (cols1024) {
            rows_fwd(ps, o->sx, v0.V, v1.V, lv, done, st);
            if constexpr (std::is_same_v<R, float>) f1024::col_adj<R>(V2, grid, done, st);
        } else {
            k_row_fwd<R, LoadPair<R>><<<(ps.nlines + P - 1) / P, 256, rsm, st>>>(v0, ps, o->sx, P, v0.W, v1.W, lv,
                                                                                done);
            k_col_fft<R><<<dim3(nt, 2), 256, csm, st>>>(v0, v1, C, done);
            k_col_adj<R><<<dim3(nt, o->nz, 2), 256, csm, st>>>(v0, v1, C, done);
        }
        EpiGradient<R> eg{F, sv->S, o->nx, o->ny};
        rows_inv(pc, o->nx, v0.Z, v1.Z, eg, done, st);
        // direction and its forward product
        ProDirection<R> pd{F, sv->S, o->nx, o->ny};
        rows_fwd(pc, o->nx, v0.Z, v1.Z, pd, done, st);
        forward_columns(st);
        EpiQNorm<R> eq{F, sv->S, o->sx};
        rows_inv(ps, o->sx, v0.W, v1.W, eq, done, st);
        k_scalars_after_direction<<<1, 32, 0, st>>>(sv->S);
        // model update, its forward product and the chi^2 scalars
        head(st);
    }
};

template <typename R>
static void run_head(gj_rrcg *sv, cudaStream_t st) {
    SolverLaunch<R> L{sv};
    L.setup();
    L.set_attributes();
    L.head(st);
}

template <typename R>
static void run_body(gj_rrcg *sv, cudaStream_t st) {
    SolverLaunch<R> L{sv};
    L.setup();
    L.body(st);
}

static gj_status check_ops(const gj_op *const ops[2]) {
    if (!ops || !ops[0] || !ops[1]) { set_error("rrcg: ops must be non-NULL"); return GJ_ERR_ARG; }
    const gj_op *a = ops[0], *b = ops[1];
    if (a->field != GJ_GRAVITY || b->field != GJ_MAGNETIC) {
        set_error("rrcg: ops[0] must be gravity and ops[1] magnetic"); return GJ_ERR_ARG;
    }
    if (a->sx != b->sx || a->sy != b->sy || a->nx != b->nx || a->ny != b->ny || a->nz != b->nz ||
        a->Nx != b->Nx || a->Ny != b->Ny || a->prec != b->prec) {
        set_error("rrcg: both operators must share grid sizes, padded sizes and precision"); return GJ_ERR_ARG;
    }
    if (a->recompute || b->recompute) {
        set_error("rrcg: operators that recompute their spectra per layer serve products only");
        return GJ_ERR_UNSUPPORTED;
    }
    return GJ_OK;
}

}  // namespace gj

extern "C" gj_status gj_rrcg_create(const gj_op *const ops[2], const gj_rrcg_params *P,
                                    const void *const dobs[2], const void *const sigma[2],
                                    const void *const m_apr[2], const void *const w_depth[2],
                                    const void *const w_hard[2], void *const m[2], gj_rrcg_hist *hist,
                                    gj_stream_t stream, gj_rrcg **out) {
    if (!out) { set_error("gj_rrcg_create: out is NULL"); return GJ_ERR_ARG; }
    *out = nullptr;
    gj_status rc = check_ops(ops);
    if (rc != GJ_OK) return rc;
    if (!P || !dobs || !sigma || !w_depth || !m) { set_error("gj_rrcg_create: NULL argument"); return GJ_ERR_ARG; }
    for (int i = 0; i < 2; ++i) {
        if (!dobs[i] || !sigma[i] || !w_depth[i] || !m[i]) { set_error("gj_rrcg_create: NULL vector"); return GJ_ERR_ARG; }
        if (P->p[i] != 1 && P->p[i] != 2) { set_error("gj_rrcg_create: p must be 1 or 2"); return GJ_ERR_ARG; }
        if (!(P->lo[i] <= P->hi[i])) { set_error("gj_rrcg_create: lo must not exceed hi"); return GJ_ERR_ARG; }
        if (!(P->alpha1[i] >= 0) || !(P->lambda[i] >= 0) || !(P->q[i] > 0)) {
            set_error("gj_rrcg_create: alpha1, lambda must be >= 0 and q > 0"); return GJ_ERR_ARG;
        }
    }
    if (P->kmax < 0) { set_error("gj_rrcg_create: kmax must be >= 0"); return GJ_ERR_ARG; }
    if (!(P->eps2 > 0)) { set_error("gj_rrcg_create: eps2 must be > 0"); return GJ_ERR_ARG; }
    if (P->scalars < 0 || P->scalars > 2) { set_error("gj_rrcg_create: bad scalars mode"); return GJ_ERR_ARG; }
    if (P->anchor != GJ_ANCHOR_APRIORI && P->anchor != GJ_ANCHOR_PREVIOUS) {
        set_error("gj_rrcg_create: bad anchor"); return GJ_ERR_ARG;
    }
    if (P->gramian_space != GJ_GRAMIAN_ORIGINAL && P->gramian_space != GJ_GRAMIAN_WEIGHTED) {
        set_error("gj_rrcg_create: bad gramian_space"); return GJ_ERR_ARG;
    }
    gj_rrcg *sv = new (std::nothrow) gj_rrcg();
    if (!sv) { set_error("gj_rrcg_create: host allocation failed"); return GJ_ERR_OOM; }
    const gj_op *o = ops[0];
    sv->op[0] = ops[0]; sv->op[1] = ops[1];
    sv->prec = o->prec;
    for (int i = 0; i < 2; ++i) {
        sv->dobs[i] = dobs[i];
        sv->mapr[i] = m_apr ? m_apr[i] : nullptr;
        sv->wdep[i] = w_depth[i];
        sv->whard[i] = w_hard ? w_hard[i] : nullptr;
        sv->m[i] = m[i];
    }
    sv->hist = hist;
    sv->prev_anchor = P->anchor == GJ_ANCHOR_PREVIOUS;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t es = elem_bytes(o->prec);
    const size_t n = (size_t)o->nx * o->ny * o->nz, s = (size_t)o->sx * o->sy;
    cudaError_t e;
    if ((e = cudaMalloc(&sv->S, sizeof(SolverDev))) != cudaSuccess) { delete sv; return cuda_fail(e, "solver state"); }
    const size_t nbuf = 4 * n + 4 * s + 2 * (size_t)o->nz + (sv->prev_anchor ? 2 * n : 0);
    if ((e = cudaMalloc(&sv->buf, nbuf * es)) != cudaSuccess) {
        cudaFree(sv->S); delete sv; return cuda_fail(e, "solver vectors");
    }
    SolverDev h{};
    h.kmax = P->kmax;
    h.stop_on_chi2 = P->stop_on_chi2;
    const bool lam0 = P->lambda[0] == 0 && P->lambda[1] == 0;
    h.per_field = P->scalars == GJ_SCALARS_PER_FIELD || (P->scalars == GJ_SCALARS_AUTO && lam0);
    h.anchor = P->anchor;
    h.gspace = P->gramian_space;
    h.eps2 = P->eps2;
    for (int i = 0; i < 2; ++i) {
        h.p[i] = P->p[i];
        h.alpha[i] = P->alpha1[i]; h.q[i] = P->q[i]; h.alpha_min[i] = P->alpha_min[i];
        h.lam[i] = P->lambda[i]; h.lo[i] = P->lo[i]; h.hi[i] = P->hi[i];
        h.chi2_target[i] = (double)s + sqrt(2.0 * (double)s);
    }
    h.hist = hist;
    cudaMemcpyAsync(sv->S, &h, sizeof(h), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(sv->buf, 0, 4 * n * es, st);
    // W_d = 1 / sigma
    for (int i = 0; i < 2; ++i) {
        void *wd = static_cast<char *>(sv->buf) + (4 * n + (2 + i) * s) * es;
        if (o->prec == GJ_FP64)
            k_reciprocal<double><<<64, 256, 0, st>>>((int)s, (const double *)sigma[i], (double *)wd);
        else
            k_reciprocal<float><<<64, 256, 0, st>>>((int)s, (const float *)sigma[i], (float *)wd);
    }
    // 1 / W_depth
    for (int i = 0; i < 2; ++i) {
        void *iw = static_cast<char *>(sv->buf) + (4 * n + 4 * s + (size_t)i * o->nz) * es;
        if (o->prec == GJ_FP64)
            k_reciprocal<double><<<1, 256, 0, st>>>(o->nz, (const double *)w_depth[i], (double *)iw);
        else
            k_reciprocal<float><<<1, 256, 0, st>>>(o->nz, (const float *)w_depth[i], (float *)iw);
    }
    if (o->prec == GJ_FP64) run_head<double>(sv, st); else run_head<float>(sv, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(sv->S); cudaFree(sv->buf); delete sv;
        return cuda_fail(e, "gj_rrcg_create");
    }
    *out = sv;
    return GJ_OK;
}

extern "C" gj_status gj_rrcg_iterate(gj_rrcg *sv, int iters, int use_graph, gj_stream_t stream) {
    if (!sv || iters < 0) { set_error("gj_rrcg_iterate: bad argument"); return GJ_ERR_ARG; }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (use_graph && sv->profile && sv->prec == GJ_FP32_MIXED && sv->op[0]->fast) {
        // segments [.. | col | .. | col | ..] with stream events around the column launches
        if (sv->seg_exec.empty()) {
            cudaStream_t cap;
            GJ_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            sv->capturing = true;
            sv->cap_err = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (sv->cap_err == cudaSuccess) {
                run_body<float>(sv, cap);
                cudaGraph_t g = nullptr;
                cudaError_t e = cudaStreamEndCapture(cap, &g);
                if (e == cudaSuccess) sv->seg_graph.push_back(g);
                else if (sv->cap_err == cudaSuccess) sv->cap_err = e;
            }
            sv->capturing = false;
            cudaStreamDestroy(cap);
            if (sv->cap_err != cudaSuccess || sv->seg_graph.size() != 5) {
                for (auto g : sv->seg_graph) cudaGraphDestroy(g);
                sv->seg_graph.clear();
                return cuda_fail(sv->cap_err != cudaSuccess ? sv->cap_err : cudaErrorUnknown, "rrcg segment capture");
            }
            for (auto g : sv->seg_graph) {
                cudaGraphExec_t x;
                GJ_CUDA(cudaGraphInstantiate(&x, g, 0));
                sv->seg_exec.push_back(x);
            }
        }
        for (int it = 0; it < iters; ++it) {
            for (int sgi = 0; sgi < 5; ++sgi) {
                ProfilePair pp{};
                if (sgi == 1 || sgi == 3) {
                    pp = take_pair(sv);
                    GJ_CUDA(cudaEventRecord(pp.a, st));
                }
                GJ_CUDA(cudaGraphLaunch(sv->seg_exec[sgi], st));
                if (sgi == 1 || sgi == 3) {
                    GJ_CUDA(cudaEventRecord(pp.b, st));
                    sv->eager_pairs.push_back(pp);
                }
            }
        }
        return GJ_OK;
    }
    if (use_graph) {
        if (!sv->exec) {
            cudaStream_t cap;
            GJ_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            sv->capturing = true;
            cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                if (sv->prec == GJ_FP64) run_body<double>(sv, cap); else run_body<float>(sv, cap);
                e = cudaStreamEndCapture(cap, &sv->graph);
            }
            sv->capturing = false;
            cudaStreamDestroy(cap);
            if (e != cudaSuccess) return cuda_fail(e, "rrcg graph capture");
            GJ_CUDA(cudaGraphInstantiate(&sv->exec, sv->graph, 0));
        }
        for (int it = 0; it < iters; ++it) GJ_CUDA(cudaGraphLaunch(sv->exec, st));
    } else {
        for (int it = 0; it < iters; ++it) {
            if (sv->prec == GJ_FP64) run_body<double>(sv, st); else run_body<float>(sv, st);
        }
        GJ_CUDA(cudaGetLastError());
    }
    return GJ_OK;
}

extern "C" gj_status gj_rrcg_report_get(gj_rrcg *sv, gj_rrcg_report *rep, gj_stream_t stream) {
    if (!sv || !rep) { set_error("gj_rrcg_report_get: NULL argument"); return GJ_ERR_ARG; }
    SolverDev h;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    GJ_CUDA(cudaMemcpyAsync(&h, sv->S, sizeof(h), cudaMemcpyDeviceToHost, st));
    GJ_CUDA(cudaStreamSynchronize(st));
    rep->status = h.status;
    rep->iterations = h.k;
    rep->converged = h.sat[0] && h.sat[1];
    rep->satisfied[0] = h.sat[0];
    rep->satisfied[1] = h.sat[1];
    rep->phi[0] = h.phi_last[0];
    rep->phi[1] = h.phi_last[1];
    rep->alpha[0] = h.alpha[0];
    rep->alpha[1] = h.alpha[1];
    rep->S_G = h.SG_last;
    if (sv->op[0]->err) {
        int e = 0;
        GJ_CUDA(cudaMemcpy(&e, sv->op[0]->err, sizeof(int), cudaMemcpyDeviceToHost));
        if (e != 0 && rep->status == GJ_OK) rep->status = e;
    }
    return GJ_OK;
}

extern "C" gj_status gj_rrcg_report_device(gj_rrcg *sv, gj_rrcg_report *rep, gj_stream_t stream) {
    if (!sv || !rep) { set_error("gj_rrcg_report_device: NULL argument"); return GJ_ERR_ARG; }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    k_report<<<1, 1, 0, st>>>(sv->S, sv->op[0]->err, rep);
    GJ_CUDA(cudaGetLastError());
    return GJ_OK;
}

extern "C" int gj_rrcg_done(gj_rrcg *sv, gj_stream_t stream) {
    if (!sv) return -1;
    int d = 0;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&d, &sv->S->done, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
    return d;
}

extern "C" gj_status gj_rrcg_profile(gj_rrcg *sv, int enable) {
    if (!sv) { set_error("gj_rrcg_profile: NULL solver"); return GJ_ERR_ARG; }
    sv->profile = enable ? 1 : 0;
    return GJ_OK;
}

extern "C" gj_status gj_rrcg_profile_read(gj_rrcg *sv, int *launches, double *total_ms) {
    if (!sv || !launches || !total_ms) { set_error("gj_rrcg_profile_read: NULL argument"); return GJ_ERR_ARG; }
    GJ_CUDA(cudaDeviceSynchronize());
    double tot = 0.0;
    int cnt = 0;
    auto acc = [&](const std::vector<ProfilePair> &v) -> gj_status {
        for (const auto &p : v) {
            float ms = 0.f;
            cudaError_t e = cudaEventElapsedTime(&ms, p.a, p.b);
            if (e != cudaSuccess) return cuda_fail(e, "gj_rrcg_profile_read");
            tot += ms;
            ++cnt;
        }
        return GJ_OK;
    };
    gj_status rc = acc(sv->eager_pairs);
    if (rc != GJ_OK) return rc;
    for (auto &p : sv->eager_pairs) sv->free_pairs.push_back(p);
    sv->eager_pairs.clear();
    *launches = cnt;
    *total_ms = tot;
    return GJ_OK;
}

extern "C" void gj_rrcg_destroy(gj_rrcg *sv) {
    if (!sv) return;
    cudaDeviceSynchronize();
    if (sv->exec) cudaGraphExecDestroy(sv->exec);
    if (sv->graph) cudaGraphDestroy(sv->graph);
    for (auto x : sv->seg_exec) cudaGraphExecDestroy(x);
    for (auto g : sv->seg_graph) cudaGraphDestroy(g);
    for (auto *v : {&sv->eager_pairs, &sv->graph_pairs, &sv->free_pairs})
        for (auto &p : *v) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    cudaFree(sv->S);
    cudaFree(sv->buf);
    delete sv;
}

// Two page-locked ints per host thread for the one-shot solve's stop flags,
// allocated on first use and kept for the life of the process (portable: any
// device may write them).  NULL if page-locked memory is not available.
static int *pinned_flags() {
    thread_local int *p = nullptr;
    thread_local bool tried = false;
    if (!tried) {
        tried = true;
        if (cudaHostAlloc(reinterpret_cast<void **>(&p), 2 * sizeof(int), cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    return p;
}

extern "C" gj_status gj_rrcg_joint_solve(const gj_op *const ops[2], const gj_rrcg_params *P,
                                         const void *const dobs[2], const void *const sigma[2],
                                         const void *const m_apr[2], const void *const w_depth[2],
                                         const void *const w_hard[2], void *const m[2], gj_rrcg_hist *hist,
                                         gj_rrcg_report *rep, gj_stream_t stream) {
    if (!rep) { set_error("gj_rrcg_joint_solve: rep is NULL"); return GJ_ERR_ARG; }
    gj_rrcg *sv = nullptr;
    gj_status rc = gj_rrcg_create(ops, P, dobs, sigma, m_apr, w_depth, w_hard, m, hist, stream, &sv);
    if (rc != GJ_OK) return rc;
    // Iterations go in chunks of eight graph replays.  The stop flag of chunk c - 1 is
    // copied into page-locked memory behind it and read while chunk c runs, so the
    // device never waits for the host; a chunk queued after the stop does no work
    // (every kernel returns at the flag).
    int left = P->kmax;
    const int chunk = 8;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int *flags = pinned_flags();
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (flags && (cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) != cudaSuccess ||
                  cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess))
        flags = nullptr;
    for (int c = 0; left > 0; ++c) {
        const int it = std::min(chunk, left);
        rc = gj_rrcg_iterate(sv, it, 1, stream);
        if (rc != GJ_OK) break;
        left -= it;
        if (!flags) {  // no page-locked flag: a synchronous check after each chunk
            const int d = gj_rrcg_done(sv, stream);
            if (d < 0) { rc = cuda_fail(cudaGetLastError(), "gj_rrcg_joint_solve"); break; }
            if (d) break;
            continue;
        }
        cudaError_t e = cudaMemcpyAsync(flags + (c & 1), &sv->S->done, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev[c & 1], st);
        if (e == cudaSuccess && c > 0) e = cudaEventSynchronize(ev[(c - 1) & 1]);
        if (e != cudaSuccess) { rc = cuda_fail(e, "gj_rrcg_joint_solve: stop flag"); break; }
        if (c > 0 && flags[(c - 1) & 1]) break;
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (rc == GJ_OK) rc = gj_rrcg_report_get(sv, rep, stream);
    gj_rrcg_destroy(sv);
    if (rc == GJ_OK && rep->status != GJ_OK) {
        set_error("gj_rrcg_joint_solve: non-finite scalar");
        return (gj_status)rep->status;
    }
    return rc;
}

// ---------------------------------------------------------------------------
// Batched form: several independent joint inversions (any sizes and precisions)
// advanced by one CUDA graph whose branches are the solvers' iterations.

struct gj_rrcg_batch {
    std::vector<gj_rrcg *> sv;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" gj_status gj_rrcg_batch_create(gj_rrcg *const *solvers, int count, gj_stream_t stream,
                                          gj_rrcg_batch **out) {
    (void)stream;
    if (!out || !solvers || count < 1) { set_error("gj_rrcg_batch_create: bad argument"); return GJ_ERR_ARG; }
    *out = nullptr;
    for (int i = 0; i < count; ++i)
        if (!solvers[i]) { set_error("gj_rrcg_batch_create: NULL solver"); return GJ_ERR_ARG; }
    // the graph runs the solvers concurrently: an operator's workspace cannot be shared
    for (int i = 0; i < count; ++i)
        for (int j = 0; j < i; ++j)
            for (int a = 0; a < 2; ++a)
                for (int b2 = 0; b2 < 2; ++b2)
                    if (solvers[i]->op[a] == solvers[j]->op[b2]) {
                        set_error("gj_rrcg_batch_create: two solvers share an operator (give each its own)");
                        return GJ_ERR_ARG;
                    }
    gj_rrcg_batch *b = new (std::nothrow) gj_rrcg_batch();
    if (!b) { set_error("gj_rrcg_batch_create: host allocation failed"); return GJ_ERR_OOM; }
    b->sv.assign(solvers, solvers + count);
    // The branches run concurrently: the fast-path solvers get grids in proportion to
    // their work (column items, scaled by N_y, plus row lines per layer), so that their
    // persistent kernels (one CTA per SM each) can be resident at the same time.  Each
    // gets twice its proportional share: the branches finish at different times, and
    // grids that add up to one CTA per SM leave SMs idle once the smaller problems are
    // done.  A smaller grid never needs more layer-sum slots than the operator holds
    // (each warp's segment only grows); the check below keeps the full grid otherwise.
    {
        auto work = [](const gj_op *o) { return (double)o->nz * (2.0 * 257 * o->Ny / 512 + o->ny); };
        double tot = 0.0;
        int sms = 0;
        for (gj_rrcg *sv : b->sv)
            if (sv->op[0]->fast && sv->prec == GJ_FP32_MIXED) {
                tot += work(sv->op[0]);
                sms = sv->op[0]->col_grid;
            }
        for (gj_rrcg *sv : b->sv) {
            sv->grid = 0;
            const gj_op *o = sv->op[0];
            if (!(o->fast && sv->prec == GJ_FP32_MIXED) || tot <= 0.0) continue;
            const double share = work(o) / tot;
            const int g = std::max(1, std::min(o->col_grid, (int)(2.0 * sms * share)));
            const int ci = fast_col_items(o->Ny, o->nz);
            const long long warps = (long long)g * f512::CWARPS;
            if (g < o->col_grid && fast_slots(2, 257, ci, warps) <= o->slots && fast_slots(1, 257, ci, warps) <= o->slots)
                sv->grid = g;
        }
    }
    // streams and events exist before the capture begins
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> br(count, nullptr);
    std::vector<cudaEvent_t> join(count, nullptr);
    cudaEvent_t fork = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t ce = cudaEventRecord(fork, cap);
        for (int i = 0; i < count && ce == cudaSuccess; ++i) {
            ce = cudaStreamWaitEvent(br[i], fork, 0);
            if (ce != cudaSuccess) break;
            gj_rrcg *sv = b->sv[i];
            sv->capturing = true;
            if (sv->prec == GJ_FP64) run_body<double>(sv, br[i]); else run_body<float>(sv, br[i]);
            sv->capturing = false;
            ce = cudaEventRecord(join[i], br[i]);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cap, join[i], 0);
        }
        cudaError_t ee = cudaStreamEndCapture(cap, &b->graph);
        e = ce != cudaSuccess ? ce : ee;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    for (gj_rrcg *sv : b->sv) sv->grid = 0;  // stepwise calls outside the batch use the full grid
    for (int i = 0; i < count; ++i) {
        if (br[i]) cudaStreamDestroy(br[i]);
        if (join[i]) cudaEventDestroy(join[i]);
    }
    if (fork) cudaEventDestroy(fork);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        if (b->graph) cudaGraphDestroy(b->graph);
        delete b;
        return cuda_fail(e, "gj_rrcg_batch_create");
    }
    *out = b;
    return GJ_OK;
}

extern "C" gj_status gj_rrcg_batch_step(gj_rrcg_batch *b, int iters, gj_stream_t stream) {
    if (!b || iters < 0) { set_error("gj_rrcg_batch_step: bad argument"); return GJ_ERR_ARG; }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (int it = 0; it < iters; ++it) GJ_CUDA(cudaGraphLaunch(b->exec, st));
    return GJ_OK;
}

extern "C" void gj_rrcg_batch_destroy(gj_rrcg_batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
}

// ---------------------------------------------------------------------------
// Host-buffer form of the one-shot solve: the inputs are copied to the device,
// the solve runs as in gj_rrcg_joint_solve, and the models are copied back.

extern "C" gj_status gj_rrcg_joint_solve_host(const gj_op *const ops[2], const gj_rrcg_params *P,
                                              const void *const dobs[2], const void *const sigma[2],
                                              const void *const m_apr[2], const void *const w_depth[2],
                                              const void *const w_hard[2], void *const m[2], gj_rrcg_report *rep,
                                              gj_stream_t stream) {
    gj_status rc = check_ops(ops);
    if (rc != GJ_OK) return rc;
    if (!P || !dobs || !sigma || !w_depth || !m || !rep) {
        set_error("gj_rrcg_joint_solve_host: NULL argument");
        return GJ_ERR_ARG;
    }
    for (int i = 0; i < 2; ++i)
        if (!dobs[i] || !sigma[i] || !w_depth[i] || !m[i]) {
            set_error("gj_rrcg_joint_solve_host: NULL vector");
            return GJ_ERR_ARG;
        }
    const gj_op *o = ops[0];
    const size_t es = elem_bytes(o->prec);
    const size_t n = (size_t)o->nx * o->ny * o->nz, s = (size_t)o->sx * o->sy, nz = (size_t)o->nz;
    // one device block: dobs, sigma (s each), w_depth (nz), m, m_apr, w_hard (n each), per field
    size_t per = 2 * s + nz + n;
    if (m_apr && (m_apr[0] || m_apr[1])) per += n;
    if (w_hard && (w_hard[0] || w_hard[1])) per += n;
    char *blk = nullptr;
    cudaError_t e = cudaMalloc(&blk, 2 * per * es);
    if (e != cudaSuccess) return cuda_fail(e, "gj_rrcg_joint_solve_host: device buffers");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const void *d_dobs[2], *d_sig[2], *d_wdep[2], *d_mapr[2] = {nullptr, nullptr}, *d_wh[2] = {nullptr, nullptr};
    void *d_m[2];
    char *at = blk;
    auto put = [&](const void *src, size_t count) -> const void * {
        void *dst = at;
        at += count * es;
        if (src && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, count * es, cudaMemcpyHostToDevice, st);
        return dst;
    };
    for (int i = 0; i < 2; ++i) {
        d_dobs[i] = put(dobs[i], s);
        d_sig[i] = put(sigma[i], s);
        d_wdep[i] = put(w_depth[i], nz);
        d_m[i] = const_cast<void *>(put(m[i], n));
        if (m_apr && (m_apr[0] || m_apr[1])) {
            const void *p = put(m_apr[i], n);
            d_mapr[i] = m_apr[i] ? p : nullptr;
        }
        if (w_hard && (w_hard[0] || w_hard[1])) {
            const void *p = put(w_hard[i], n);
            d_wh[i] = w_hard[i] ? p : nullptr;
        }
    }
    if (e != cudaSuccess) {
        cudaFree(blk);
        return cuda_fail(e, "gj_rrcg_joint_solve_host: copies in");
    }
    rc = gj_rrcg_joint_solve(ops, P, d_dobs, d_sig, d_mapr, d_wdep, d_wh, d_m, nullptr, rep, stream);
    if (rc == GJ_OK || rc == GJ_ERR_NONFINITE) {
        for (int i = 0; i < 2 && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(m[i], d_m[i], n * es, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "gj_rrcg_joint_solve_host: copies out");
    }
    cudaFree(blk);
    return rc;
}
