// Host-side launch helpers of the 512 x 512 fast path.
#pragma once
#include "fast512.cuh"
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
    return V;
}

template <typename R, class Pro>
inline void set_row_fwd_attr() {
    cudaFuncSetAttribute(k_row_fwd512<R, Pro>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row_fwd<R>());
}
template <typename R, class Epi>
inline void set_row_inv_attr() {
    cudaFuncSetAttribute(k_row_inv512<R, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row_inv<R>());
}
template <typename R>
inline void set_col_attr() {
    cudaFuncSetAttribute(k_col_fwd512<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_col_fwd<R>());
    cudaFuncSetAttribute(k_col_adj512<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_col_adj<R>());
}

template <typename R, class Pro>
inline void row_fwd(const View2<R> &V, int joint, int nlines, int lpl, int n_in, int out_is_W, const Pro &pro,
                    const int *done, cudaStream_t st) {
    const int per = joint ? 16 : 32;
    k_row_fwd512<R, Pro><<<(nlines + per - 1) / per, WARPS * 32, smem_row_fwd<R>(), st>>>(V, joint, nlines, lpl, n_in,
                                                                                         out_is_W, pro, done);
}

template <typename R, class Epi>
inline void row_inv(const View2<R> &V, int joint, int nlines, int lpl, int n_out, int in_is_W, const Epi &epi,
                    const int *done, cudaStream_t st) {
    const int per = joint ? 16 : 32;
    k_row_inv512<R, Epi><<<(nlines + per - 1) / per, WARPS * 32, smem_row_inv<R>(), st>>>(V, joint, nlines, lpl, n_out,
                                                                                         in_is_W, epi, done);
}

template <typename R>
inline void col_fwd(const View2<R> &V, int grid, const int *done, cudaStream_t st) {
    k_col_fwd512<R><<<grid, WARPS * 32, smem_col_fwd<R>(), st>>>(V, done);
}

template <typename R>
inline void col_adj(const View2<R> &V, int grid, const int *done, cudaStream_t st) {
    k_col_adj512<R><<<grid, WARPS * 32, smem_col_adj<R>(), st>>>(V, done);
}

}  // namespace f512
}  // namespace gj
