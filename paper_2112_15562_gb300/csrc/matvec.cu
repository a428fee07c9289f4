// G m and G^T r of one field (Sec. 2.7.1): the C-ABI entry points and the launch
// sequences shared with the solver.
#include "fast_launch.cuh"
#include "view.cuh"

namespace gj {

template <typename R>
static void launch_forward(const gj_op *o, const R *m, R *d, cudaStream_t st) {
    OpView<R> v = view_of<R>(o);
    const size_t cs = sizeof(cpx<R>);
    // rows: m -> Z (pairs of consecutive (layer, row) lines)
    PairMap pm{o->nz * o->ny, 0};
    const int P = o->P_row;
    const size_t rsm = row_smem(o->Nx, P, cs);
    allow_max_smem(k_row_fwd<R, LoadPlain<R>>);
    const int npr = (pm.nlines + 1) / 2;
    k_row_fwd<R, LoadPlain<R>><<<(npr + P - 1) / P, 256, rsm, st>>>(v, pm, o->nx, P, v.Z, v.Z,
                                                                    LoadPlain<R>{m, m, o->nx}, nullptr);
    // columns with the layer spectra, summed over layers
    cudaMemsetAsync(v.Y, 0, (size_t)o->Ny * o->ncol * cs, st);
    const int C = o->C_col;
    const int nt = (o->ncol + C - 1) / C;
    const size_t msm = col_smem(o->Ny, C, 3, cs);
    allow_max_smem(k_col_fwd_mac<R>);
    if (o->recompute) {
        // one layer at a time: rebuild its spectrum, then add its column products
        for (int r = 0; r < o->nz; ++r) {
            recompute_layer(o, r, st);
            OpView<R> vr = v;
            vr.rbase = r;
            vr.spec_r0 = r;
            k_col_fwd_mac<R><<<dim3(nt, 1, 1), 256, msm, st>>>(vr, vr, C, 1, nullptr);
        }
    } else {
        k_col_fwd_mac<R><<<dim3(nt, (o->nz + o->L_grp - 1) / o->L_grp, 1), 256, msm, st>>>(v, v, C, o->L_grp, nullptr);
    }
    // inverse columns
    const size_t ism = col_smem(o->Ny, C, 2, cs);
    allow_max_smem(k_col_inv<R>);
    k_col_inv<R><<<dim3(nt, 1), 256, ism, st>>>(v, v, C, nullptr);
    // inverse rows, cropped to the stations
    PairMap ps{o->sy, 0};
    const int nps = (ps.nlines + 1) / 2;
    allow_max_smem(k_row_inv<R, StorePlain<R>>);
    k_row_inv<R, StorePlain<R>><<<(nps + P - 1) / P, 256, rsm, st>>>(v, ps, o->sx, P, v.W, v.W,
                                                                     StorePlain<R>{d, d, o->sx}, nullptr);
}

// N_y = 1024 column kernels: the general row kernels write and read the transposed
// intermediates (PairMap.lpl gives the lines per layer); a pair call shares the column
// launch of both fields.
static void fast1024_forward(const gj_op *a, const gj_op *b, const float *m0, const float *m1, float *d0, float *d1,
                             cudaStream_t st) {
    using R = float;
    const size_t cs = sizeof(cpx<R>);
    const int P = a->P_row;
    const size_t rsm = row_smem(a->Nx, P, cs);
    allow_max_smem(k_row_fwd<R, LoadPlain<R>>);
    allow_max_smem(k_row_inv<R, StorePlain<R>>);
    f1024::set_col_attr<R>();
    const bool rows1024 = a->Nx == 1024;  // warp-FFT rows as well
    if (rows1024) {
        f1024::set_row_fwd_attr<R, LoadPlain<R>>();
        f1024::set_row_inv_attr<R, StorePlain<R>>();
    }
    const gj_op *ops[2] = {a, b};
    const float *ms[2] = {m0, m1};
    float *ds[2] = {d0, d1};
    const int nf = b ? 2 : 1;
    if (rows1024 && nf == 2) {
        // both fields' row passes in one launch each (grid y = field)
        f1024::set_row_fwd_attr<R, LoadPlain2<R>>();
        f1024::set_row_inv_attr<R, StorePlain2<R>>();
        OpView<R> va = view_of<R>(a), vb = view_of<R>(b);
        PairMap pm{a->nz * a->ny, 0, a->ny};
        f1024::row_fwd<R>(va, pm, a->nx, va.Z, vb.Z, a->twtab, LoadPlain2<R>{{m0, m1}, a->nx}, nullptr, st, 2);
        f1024::col_fwd<R>(f512::make_view2<R>(a, b), a->col_grid, nullptr, st);
        PairMap ps{a->sy, 0, a->sy};
        f1024::row_inv<R>(va, ps, a->sx, va.W, vb.W, a->twtab, StorePlain2<R>{{d0, d1}, a->sx}, nullptr, st, 2);
        return;
    }
    for (int i = 0; i < nf; ++i) {
        const gj_op *o = ops[i];
        OpView<R> v = view_of<R>(o);
        PairMap pm{o->nz * o->ny, 0, o->ny};
        const int npr = (pm.nlines + 1) / 2;
        const LoadPlain<R> lp{ms[i], ms[i], o->nx};
        if (rows1024)
            f1024::row_fwd<R>(v, pm, o->nx, v.Z, v.Z, o->twtab, lp, nullptr, st);
        else
            k_row_fwd<R, LoadPlain<R>><<<(npr + P - 1) / P, 256, rsm, st>>>(v, pm, o->nx, P, v.Z, v.Z, lp, nullptr);
    }
    f1024::col_fwd<R>(f512::make_view2<R>(a, b), a->col_grid, nullptr, st);
    for (int i = 0; i < nf; ++i) {
        const gj_op *o = ops[i];
        OpView<R> v = view_of<R>(o);
        PairMap ps{o->sy, 0, o->sy};
        const int nps = (ps.nlines + 1) / 2;
        const StorePlain<R> sp{ds[i], ds[i], o->sx};
        if (rows1024)
            f1024::row_inv<R>(v, ps, o->sx, v.W, v.W, o->twtab, sp, nullptr, st);
        else
            k_row_inv<R, StorePlain<R>><<<(nps + P - 1) / P, 256, rsm, st>>>(v, ps, o->sx, P, v.W, v.W, sp, nullptr);
    }
}

static void fast1024_adjoint(const gj_op *a, const gj_op *b, const float *r0, const float *r1, float *g0, float *g1,
                             cudaStream_t st) {
    using R = float;
    const size_t cs = sizeof(cpx<R>);
    const int P = a->P_row;
    const size_t rsm = row_smem(a->Nx, P, cs);
    allow_max_smem(k_row_fwd<R, LoadPlain<R>>);
    allow_max_smem(k_row_inv<R, StorePlain<R>>);
    f1024::set_col_attr<R>();
    const bool rows1024 = a->Nx == 1024;
    if (rows1024) {
        f1024::set_row_fwd_attr<R, LoadPlain<R>>();
        f1024::set_row_inv_attr<R, StorePlain<R>>();
    }
    const gj_op *ops[2] = {a, b};
    const float *rs[2] = {r0, r1};
    float *gs[2] = {g0, g1};
    const int nf = b ? 2 : 1;
    if (rows1024 && nf == 2) {
        // both fields' row passes in one launch each (grid y = field)
        f1024::set_row_fwd_attr<R, LoadPlain2<R>>();
        f1024::set_row_inv_attr<R, StorePlain2<R>>();
        OpView<R> va = view_of<R>(a), vb = view_of<R>(b);
        PairMap ps{a->sy, 0, a->sy};
        f1024::row_fwd<R>(va, ps, a->sx, va.V, vb.V, a->twtab, LoadPlain2<R>{{r0, r1}, a->sx}, nullptr, st, 2);
        f1024::col_adj<R>(f512::make_view2<R>(a, b), a->col_grid, nullptr, st);
        PairMap pm{a->nz * a->ny, 0, a->ny};
        f1024::row_inv<R>(va, pm, a->nx, va.Z, vb.Z, a->twtab, StorePlain2<R>{{g0, g1}, a->nx}, nullptr, st, 2);
        return;
    }
    for (int i = 0; i < nf; ++i) {
        const gj_op *o = ops[i];
        OpView<R> v = view_of<R>(o);
        PairMap ps{o->sy, 0, o->sy};
        const int nps = (ps.nlines + 1) / 2;
        const LoadPlain<R> lp{rs[i], rs[i], o->sx};
        if (rows1024)
            f1024::row_fwd<R>(v, ps, o->sx, v.V, v.V, o->twtab, lp, nullptr, st);
        else
            k_row_fwd<R, LoadPlain<R>><<<(nps + P - 1) / P, 256, rsm, st>>>(v, ps, o->sx, P, v.V, v.V, lp, nullptr);
    }
    f1024::col_adj<R>(f512::make_view2<R>(a, b), a->col_grid, nullptr, st);
    for (int i = 0; i < nf; ++i) {
        const gj_op *o = ops[i];
        OpView<R> v = view_of<R>(o);
        PairMap pm{o->nz * o->ny, 0, o->ny};
        const int npr = (pm.nlines + 1) / 2;
        const StorePlain<R> sp{gs[i], gs[i], o->nx};
        if (rows1024)
            f1024::row_inv<R>(v, pm, o->nx, v.Z, v.Z, o->twtab, sp, nullptr, st);
        else
            k_row_inv<R, StorePlain<R>><<<(npr + P - 1) / P, 256, rsm, st>>>(v, pm, o->nx, P, v.Z, v.Z, sp, nullptr);
    }
}

template <typename R>
static void launch_adjoint(const gj_op *o, const R *r, R *g, cudaStream_t st) {
    OpView<R> v = view_of<R>(o);
    const size_t cs = sizeof(cpx<R>);
    const int P = o->P_row;
    const size_t rsm = row_smem(o->Nx, P, cs);
    // rows of the residual -> W
    PairMap ps{o->sy, 0};
    const int nps = (ps.nlines + 1) / 2;
    allow_max_smem(k_row_fwd<R, LoadPlain<R>>);
    k_row_fwd<R, LoadPlain<R>><<<(nps + P - 1) / P, 256, rsm, st>>>(v, ps, o->sx, P, v.W, v.W,
                                                                    LoadPlain<R>{r, r, o->sx}, nullptr);
    const int C = o->C_col;
    const int nt = (o->ncol + C - 1) / C;
    const size_t sm2 = col_smem(o->Ny, C, 2, cs);
    allow_max_smem(k_col_fft<R>);
    k_col_fft<R><<<dim3(nt, 1), 256, sm2, st>>>(v, v, C, nullptr);
    allow_max_smem(k_col_adj<R>);
    if (o->recompute) {
        for (int r = 0; r < o->nz; ++r) {
            recompute_layer(o, r, st);
            OpView<R> vr = v;
            vr.rbase = r;
            vr.spec_r0 = r;
            k_col_adj<R><<<dim3(nt, 1, 1), 256, sm2, st>>>(vr, vr, C, nullptr);
        }
    } else {
        k_col_adj<R><<<dim3(nt, o->nz, 1), 256, sm2, st>>>(v, v, C, nullptr);
    }
    PairMap pm{o->nz * o->ny, 0};
    const int npr = (pm.nlines + 1) / 2;
    allow_max_smem(k_row_inv<R, StorePlain<R>>);
    k_row_inv<R, StorePlain<R>><<<(npr + P - 1) / P, 256, rsm, st>>>(v, pm, o->nx, P, v.Z, v.Z,
                                                                     StorePlain<R>{g, g, o->nx}, nullptr);
}

// 512 x 512 fast path: rows -> persistent layer-summed columns -> inverse rows
static void fast_forward(const gj_op *o, const float *m, float *d, cudaStream_t st) {
    using namespace f512;
    View2<float> V = make_view2<float>(o, nullptr);
    set_row_fwd_t_attr<float, LoadPlain<float>, true>();
    set_row_inv_attr<float, StorePlain<float>, kDataNW, kDataFPW>();
    set_col_attr<float>();
    row_fwd_t<float, true>(V, o->col_grid, o->nz, o->ny, o->nx, 0, LoadPlain<float>{m, m, o->nx}, nullptr, st);
    col_fwd<float>(V, o->col_grid, nullptr, st);
    row_inv<float, kDataNW, kDataFPW>(V, 0, o->sy, o->sy, o->sx, 1, StorePlain<float>{d, d, o->sx}, nullptr, st);
}

static void fast_adjoint(const gj_op *o, const float *r, float *g, cudaStream_t st) {
    using namespace f512;
    View2<float> V = make_view2<float>(o, nullptr);
    set_row_fwd_attr<float, LoadPlain<float>, kDataNW, kDataFPW>();
    set_row_inv_t_attr<float, StorePlain<float>, true>();
    set_col_attr<float>();
    row_fwd<float, kDataNW, kDataFPW>(V, 0, o->sy, o->sy, o->sx, 2, LoadPlain<float>{r, r, o->sx}, nullptr, st);
    col_adj<float>(V, o->col_grid, nullptr, st);
    row_inv_t<float, true>(V, o->col_grid, o->nz, o->ny, o->nx, 0, StorePlain<float>{g, g, o->nx}, nullptr, st);
}

// Both fields of a joint problem with shared column passes: the row and data-line
// passes run per field (two lines of one field per complex transform, as in the
// single-field products), because a complex transform that carried a line of each
// field would mix their rounding errors (the magnetic data are typically some 100
// times the gravity data); the persistent column passes take both fields' columns in
// one launch, where the fields never mix, which fills the GPU better than two
// single-field column launches.
static void fast_forward_pair(const gj_op *a, const gj_op *b, const float *m0, const float *m1, float *d0, float *d1,
                              cudaStream_t st) {
    using namespace f512;
    View2<float> V = make_view2<float>(a, b);
    set_row_fwd_t_attr<float, LoadPlain2<float>, true>();
    set_row_inv_attr<float, StorePlain2<float>, kDataNW, kDataFPW>();
    set_col_attr<float>();
    // one launch per pass: the row passes take both fields' lines (pair mode, each
    // field's functor), the column pass both fields' columns
    row_fwd_t<float, true>(V, a->col_grid, a->nz, a->ny, a->nx, 0, LoadPlain2<float>{{m0, m1}, a->nx}, nullptr, st);
    col_fwd<float>(V, a->col_grid, nullptr, st);
    row_inv<float, kDataNW, kDataFPW>(V, 0, a->sy, a->sy, a->sx, 1, StorePlain2<float>{{d0, d1}, a->sx}, nullptr, st,
                                      2);
}

static void fast_adjoint_pair(const gj_op *a, const gj_op *b, const float *r0, const float *r1, float *g0, float *g1,
                              cudaStream_t st) {
    using namespace f512;
    View2<float> V = make_view2<float>(a, b);
    set_row_fwd_attr<float, LoadPlain2<float>, kDataNW, kDataFPW>();
    set_row_inv_t_attr<float, StorePlain2<float>, true>();
    set_col_attr<float>();
    row_fwd<float, kDataNW, kDataFPW>(V, 0, a->sy, a->sy, a->sx, 2, LoadPlain2<float>{{r0, r1}, a->sx}, nullptr, st,
                                      2);
    col_adj<float>(V, a->col_grid, nullptr, st);
    row_inv_t<float, true>(V, a->col_grid, a->nz, a->ny, a->nx, 0, StorePlain2<float>{{g0, g1}, a->nx}, nullptr, st);
}

// Two operators serve one joint launch when both are on the fast path with the same
// grid (their workspaces stay separate; the launch uses the first one's error word).
static bool pair_eligible(const gj_op *a, const gj_op *b) {
    return a != b && ((a->fast && b->fast) || (a->fast1024 && b->fast1024)) && a->sx == b->sx && a->sy == b->sy &&
           a->nx == b->nx && a->ny == b->ny && a->nz == b->nz && a->Ny == b->Ny && a->Nx == b->Nx &&
           a->P_row == b->P_row && a->col_grid == b->col_grid;
}

gj_status forward_enqueue(const gj_op *o, const void *m, void *d, cudaStream_t st) {
    if (o->fast) fast_forward(o, (const float *)m, (float *)d, st);
    else if (o->fast1024) fast1024_forward(o, nullptr, (const float *)m, nullptr, (float *)d, nullptr, st);
    else if (o->prec == GJ_FP64) launch_forward<double>(o, (const double *)m, (double *)d, st);
    else launch_forward<float>(o, (const float *)m, (float *)d, st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GJ_OK : cuda_fail(e, "g_forward launch");
}

gj_status adjoint_enqueue(const gj_op *o, const void *r, void *g, cudaStream_t st) {
    if (o->fast) fast_adjoint(o, (const float *)r, (float *)g, st);
    else if (o->fast1024) fast1024_adjoint(o, nullptr, (const float *)r, nullptr, (float *)g, nullptr, st);
    else if (o->prec == GJ_FP64) launch_adjoint<double>(o, (const double *)r, (double *)g, st);
    else launch_adjoint<float>(o, (const float *)r, (float *)g, st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GJ_OK : cuda_fail(e, "g_adjoint launch");
}

}  // namespace gj

extern "C" gj_status gj_g_forward(const gj_op *op, const void *m, void *d, gj_stream_t stream) {
    if (!op || !m || !d) { gj::set_error("gj_g_forward: NULL argument"); return GJ_ERR_ARG; }
    return gj::forward_enqueue(op, m, d, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" gj_status gj_g_adjoint(const gj_op *op, const void *r, void *g, gj_stream_t stream) {
    if (!op || !r || !g) { gj::set_error("gj_g_adjoint: NULL argument"); return GJ_ERR_ARG; }
    return gj::adjoint_enqueue(op, r, g, reinterpret_cast<cudaStream_t>(stream));
}

namespace gj {
// The bounded wait on a barrier that nothing completes (no copy is issued, so
// nothing can land after the wait gives up): records its status in *err.
static __global__ void k_wait_selftest(unsigned long long limit_ns, int *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) f512::mbar_init(&bar);
    f512::mbar_fence_init();
    __syncthreads();
    if (threadIdx.x == 0 && f512::mbar_wait(&bar, 0, err, limit_ns)) *err = GJ_OK;
}
}  // namespace gj

extern "C" gj_status gj_op_status(gj_op *op, int reset, gj_stream_t stream) {
    if (!op) { gj::set_error("gj_op_status: NULL operator"); return GJ_ERR_ARG; }
    if (!op->err) return GJ_OK;  // only the fast path's column kernels wait on copies
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int e = 0;
    GJ_CUDA(cudaMemcpyAsync(&e, op->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GJ_CUDA(cudaStreamSynchronize(st));
    if (e == 0) return GJ_OK;
    if (reset) {
        // the counters of a column whose warps gave up may be nonzero: restart them
        GJ_CUDA(cudaMemsetAsync(op->cnt, 0, op->ncol * sizeof(int), st));
        GJ_CUDA(cudaMemsetAsync(op->err, 0, sizeof(int), st));
        GJ_CUDA(cudaStreamSynchronize(st));
    }
    gj::set_error("gj_op_status: a bounded device wait of this operator gave up (GJ_ERR_TIMEOUT)");
    return (gj_status)e;
}

extern "C" gj_status gj_selftest_bounded_wait(int64_t limit_ns, gj_stream_t stream) {
    if (limit_ns < 0 || limit_ns > 10LL * 1000 * 1000 * 1000) {
        gj::set_error("gj_selftest_bounded_wait: limit_ns must be in [0, 1e10]");
        return GJ_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int *err = nullptr;
    GJ_CUDA(cudaMalloc(&err, sizeof(int)));
    cudaError_t e = cudaMemsetAsync(err, 0xff, sizeof(int), st);  // -1 until the kernel writes
    if (e == cudaSuccess) {
        gj::k_wait_selftest<<<1, 32, 0, st>>>((unsigned long long)limit_ns, err);
        e = cudaGetLastError();
    }
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(err);
    if (e != cudaSuccess) return gj::cuda_fail(e, "gj_selftest_bounded_wait");
    return (gj_status)h;
}

extern "C" gj_status gj_g_forward_pair(const gj_op *const ops[2], const void *const m[2], void *const d[2],
                                       gj_stream_t stream) {
    if (!ops || !m || !d || !ops[0] || !ops[1] || !m[0] || !m[1] || !d[0] || !d[1]) {
        gj::set_error("gj_g_forward_pair: NULL argument");
        return GJ_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (gj::pair_eligible(ops[0], ops[1])) {
        if (ops[0]->fast1024)
            gj::fast1024_forward(ops[0], ops[1], (const float *)m[0], (const float *)m[1], (float *)d[0], (float *)d[1], st);
        else
            gj::fast_forward_pair(ops[0], ops[1], (const float *)m[0], (const float *)m[1], (float *)d[0], (float *)d[1], st);
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? GJ_OK : gj::cuda_fail(e, "gj_g_forward_pair launch");
    }
    gj_status rc = gj::forward_enqueue(ops[0], m[0], d[0], st);
    return rc == GJ_OK ? gj::forward_enqueue(ops[1], m[1], d[1], st) : rc;
}

extern "C" gj_status gj_g_adjoint_pair(const gj_op *const ops[2], const void *const r[2], void *const g[2],
                                       gj_stream_t stream) {
    if (!ops || !r || !g || !ops[0] || !ops[1] || !r[0] || !r[1] || !g[0] || !g[1]) {
        gj::set_error("gj_g_adjoint_pair: NULL argument");
        return GJ_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (gj::pair_eligible(ops[0], ops[1])) {
        if (ops[0]->fast1024)
            gj::fast1024_adjoint(ops[0], ops[1], (const float *)r[0], (const float *)r[1], (float *)g[0], (float *)g[1], st);
        else
            gj::fast_adjoint_pair(ops[0], ops[1], (const float *)r[0], (const float *)r[1], (float *)g[0], (float *)g[1], st);
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? GJ_OK : gj::cuda_fail(e, "gj_g_adjoint_pair launch");
    }
    gj_status rc = gj::adjoint_enqueue(ops[0], r[0], g[0], st);
    return rc == GJ_OK ? gj::adjoint_enqueue(ops[1], r[1], g[1], st) : rc;
}
