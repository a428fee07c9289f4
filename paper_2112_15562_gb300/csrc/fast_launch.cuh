// Host-side launch helpers of the fast path (N_x = 512; N_y = 512 or 256).
#pragma once
#include "fast1024.cuh"
#include "fast512_rows.cuh"
#include "view.cuh"

namespace gj {
namespace f512 {

template <typename R>
inline View2<R> make_view2(const gj_op *a, const gj_op *b) {
    View2<R> V;
    V.op[0] = view_of<R>(a);
    V.op[1] = view_of<R>(b ? b : a);
    V.P[0] = static_cast<cpx<R> *>(a->P);
    V.P[1] = static_cast<cpx<R> *>((b ? b : a)->P);
    V.cnt[0] = a->cnt;
    V.cnt[1] = (b ? b : a)->cnt;
    V.slots = a->slots;
    V.nfield = b ? 2 : 1;
    V.err = a->err;
    V.twtab = static_cast<const cpx<R> *>(a->twtab);
    V.hy = a->Ny / 2;
    return V;
}

// row-pass shapes: cell lines use 8 warps x 2 transforms, data lines 4 warps x 1
constexpr int kCellNW = 8, kCellFPW = 2, kDataNW = 4, kDataFPW = 1;
// persistent joint row passes: warps per CTA (one CTA per SM, teams of four)
constexpr int kRowNW = 12;

template <typename R, class Pro, int NW, int FPW>
inline void set_row_fwd_attr() {
    allow_max_smem(k_row_fwd512<R, Pro, NW, FPW>);
}
template <typename R, class Epi, int NW, int FPW>
inline void set_row_inv_attr() {
    allow_max_smem(k_row_inv512<R, Epi, NW, FPW>);
}
template <typename R, class Epi, int NW>
inline void set_row_resid_attr() {
    allow_max_smem(k_row_resid512<R, Epi, NW>);
}
template <typename R, class Pro, bool PAIR = false>
inline void set_row_fwd_t_attr() {
    allow_max_smem(k_row_fwd512t<R, Pro, kRowNW, PAIR>);
}
template <typename R, class Epi, bool PAIR = false>
inline void set_row_inv_t_attr() {
    allow_max_smem(k_row_inv512t<R, Epi, kRowNW, PAIR>);
}
template <typename R>
inline void set_col_attr() {
    allow_max_smem(k_col_fwd512<R>);
    allow_max_smem(k_col_adj512<R>);
    allow_max_smem(k_col_fwd256<R>);
    allow_max_smem(k_col_adj256<R>);
}

// out_sel / in_sel: 0 = Z, 1 = W, 2 = V
// nfield = 2 (single mode, with LoadPlain2 / StorePlain2): the lines of both fields,
// grid y = field
template <typename R, int NW, int FPW, class Pro>
inline void row_fwd(const View2<R> &V, int joint, int nlines, int lpl, int n_in, int out_sel, const Pro &pro,
                    const int *done, cudaStream_t st, int nfield = 1) {
    const int per = (joint ? 1 : 2) * NW * FPW;
    k_row_fwd512<R, Pro, NW, FPW><<<dim3((nlines + per - 1) / per, nfield), NW * 32, smem_row_fwd<R, NW, FPW>(), st>>>(
        V, joint, nlines, lpl, n_in, out_sel, pro, done);
}

template <typename R, int NW, int FPW, class Epi>
inline void row_inv(const View2<R> &V, int joint, int nlines, int lpl, int n_out, int in_sel, const Epi &epi,
                    const int *done, cudaStream_t st, int nfield = 1) {
    const int per = (joint ? 1 : 2) * NW * FPW;
    k_row_inv512<R, Epi, NW, FPW><<<dim3((nlines + per - 1) / per, nfield), NW * 32, smem_row_inv<R, NW, FPW>(), st>>>(
        V, joint, nlines, lpl, n_out, in_sel, epi, done);
}

template <typename R, int NW, class Epi>
inline void row_resid(const View2<R> &V, int nlines, int n_out, const Epi &epi, const int *done, cudaStream_t st) {
    k_row_resid512<R, Epi, NW><<<(nlines + NW - 1) / NW, NW * 32, smem_row_resid<R, NW>(), st>>>(V, nlines, n_out, epi,
                                                                                                 done);
}

// persistent team row passes over nz layers of lpl lines (grid: one CTA per SM);
// PAIR: one field, two of its lines per transform; else both fields, one line each
template <typename R, bool PAIR = false, class Pro>
inline void row_fwd_t(const View2<R> &V, int grid, int nz, int lpl, int n_in, int out_sel, const Pro &pro,
                      const int *done, cudaStream_t st) {
    k_row_fwd512t<R, Pro, kRowNW, PAIR><<<grid, kRowNW * 32, smem_row_t<R, kRowNW, Pro::NPRE>(), st>>>(
        V, nz, lpl, n_in, out_sel, pro, done);
}
template <typename R, bool PAIR = false, class Epi>
inline void row_inv_t(const View2<R> &V, int grid, int nz, int lpl, int n_out, int in_sel, const Epi &epi,
                      const int *done, cudaStream_t st) {
    k_row_inv512t<R, Epi, kRowNW, PAIR><<<grid, kRowNW * 32, smem_row_t<R, kRowNW, Epi::NPRE>(), st>>>(
        V, nz, lpl, n_out, in_sel, epi, done);
}

// the column passes of the operator's N_y (512 or 256)
template <typename R>
inline void col_fwd(const View2<R> &V, int grid, const int *done, cudaStream_t st) {
    if (V.op[0].Ny == N2)
        k_col_fwd256<R><<<grid, CWARPS * 32, smem_col_fwd256<R>(), st>>>(V, done);
    else
        k_col_fwd512<R><<<grid, CWARPS * 32, smem_col_fwd<R>(), st>>>(V, done);
}

template <typename R>
inline void col_adj(const View2<R> &V, int grid, const int *done, cudaStream_t st) {
    if (V.op[0].Ny == N2)
        k_col_adj256<R><<<grid, CWARPS * 32, smem_col_adj256<R>(), st>>>(V, done);
    else
        k_col_adj512<R><<<grid, CWARPS * 32, smem_col_adj<R>(), st>>>(V, done);
}

}  // namespace f512

namespace f1024 {

template <typename R>
inline void set_col_attr() {
    allow_max_smem(k_col_fwd1024<R>);
    allow_max_smem(k_col_adj1024<R>);
}

template <typename R>
inline void col_fwd(const f512::View2<R> &V, int grid, const int *done, cudaStream_t st) {
    k_col_fwd1024<R><<<grid, CWF * 32, smem_col_fwd<R>(), st>>>(V, done);
}

template <typename R>
inline void col_adj(const f512::View2<R> &V, int grid, const int *done, cudaStream_t st) {
    k_col_adj1024<R><<<grid, CWA * 32, smem_col_adj<R>(), st>>>(V, done);
}

// the N_x = 1024 row passes (the operator's Tab1024 serves the rows too when N_x = N_y)
template <typename R, class Pro>
inline void set_row_fwd_attr() { allow_max_smem(k_row_fwd1024<R, Pro>); }
template <typename R, class Epi>
inline void set_row_inv_attr() { allow_max_smem(k_row_inv1024<R, Epi>); }
inline int row_grid(const PairMap &pm) {
    const int np = pm.joint ? pm.nlines : (pm.nlines + 1) / 2;
    return (np + RW - 1) / RW;
}
// nfield = 2 (pairs of one field's lines, LoadPlain2 / StorePlain2): both fields in one
// launch, grid y = field, field 1's buffers in o1 / i1
template <typename R, class Pro>
inline void row_fwd(const OpView<R> &v, const PairMap &pm, int n_in, cpx<R> *o0, cpx<R> *o1, const void *tab,
                    const Pro &pro, const int *done, cudaStream_t st, int nfield = 1) {
    k_row_fwd1024<R, Pro><<<dim3(row_grid(pm), nfield), RW * 32, smem_row<R>(), st>>>(
        v, pm, n_in, o0, o1, static_cast<const cpx<R> *>(tab), pro, done);
}
template <typename R, class Epi>
inline void row_inv(const OpView<R> &v, const PairMap &pm, int n_out, const cpx<R> *i0, const cpx<R> *i1,
                    const void *tab, const Epi &epi, const int *done, cudaStream_t st, int nfield = 1) {
    k_row_inv1024<R, Epi><<<dim3(row_grid(pm), nfield), RW * 32, smem_row<R>(), st>>>(
        v, pm, n_out, i0, i1, static_cast<const cpx<R> *>(tab), epi, done);
}

}  // namespace f1024
}  // namespace gj
