/*
 * gj.h - C ABI of the GB300 joint gravity-magnetic inversion library.
 *
 * Implements the hot path of Vatankhah, Renaut, Huang, Mickus & Gharloghi,
 * "Large-scale focusing joint inversion of gravity and magnetic data with
 * Gramian constraint" (arXiv 2112.15562): the per-depth-layer BTTB sensitivity
 * products A m and A^T r of the gravity and magnetic problems evaluated with 2-D
 * FFTs of the BCCB embedding (Sec. 2.7.1), and the regularised reweighted CG
 * joint solve with Lp stabilisers and the Gramian coupling (Eq. RRCG:1-8,
 * Secs. 2.2-2.8).
 *
 * Conventions (all calls):
 *  - Pointers are DEVICE pointers unless the comment says "host".  The caller
 *    owns every buffer it passes; the library never frees caller memory.
 *  - Vectors use the precision of the operator: double for GJ_FP64, float for
 *    GJ_FP32_MIXED.  Scalars reported by the library are always double.
 *  - Model vectors are layer-major m[r][iy][ix] (ix fastest, r = depth layer,
 *    n = nx*ny*nz); data vectors are d[jy][jx] (s = sx*sy).  x = East,
 *    y = North, z = Down.
 *  - Calls are asynchronous on `stream` unless stated.  A gj_op owns a device
 *    workspace, so calls that use the same gj_op must be ordered (one stream,
 *    or explicit events); different gj_op objects are independent.
 *  - Errors: argument checks run synchronously and return a negative
 *    gj_status without enqueuing work; gj_last_error() then returns a message
 *    (per thread).  CUDA launch failures return GJ_ERR_CUDA.
 *  - Kernel attributes (shared-memory limits) are set once per kernel and device
 *    and kept for the life of the process; a caller that resets a device
 *    (cudaDeviceReset) must not use the library on it afterwards.
 */
#ifndef GJ_H
#define GJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *gj_stream_t;

typedef enum {
    GJ_OK = 0,
    GJ_ERR_ARG = -1,         /* invalid argument (message in gj_last_error) */
    GJ_ERR_OOM = -2,         /* device allocation failed */
    GJ_ERR_CUDA = -3,        /* a CUDA runtime call or launch failed */
    GJ_ERR_NONFINITE = -4,   /* the solver met a non-finite scalar */
    GJ_ERR_TIMEOUT = -5,     /* a bounded device wait gave up */
    GJ_ERR_UNSUPPORTED = -6  /* e.g. a padded size with a prime factor > 17 */
} gj_status;

typedef enum { GJ_GRAVITY = 1, GJ_MAGNETIC = 2 } gj_field;
typedef enum { GJ_FP64 = 0, GJ_FP32_MIXED = 1 } gj_precision;

/* Station grid and prism mesh (Sec. 2.7.1).  Prism (r, iy, ix) spans
 * [ix*dx, (ix+1)*dx] x [iy*dy, (iy+1)*dy] x [z_edges[r], z_edges[r+1]];
 * station (jy, jx) sits at the horizontal centre of prism column
 * (jy + off_y, jx + off_x) at depth station_z, which must not lie below
 * z_edges[0] (stations at or above the top of the mesh). */
typedef struct {
    int sx, sy;              /* stations in x and y */
    int nx, ny, nz;          /* prisms in x, y and depth layers */
    double dx, dy;           /* cell sizes, metres */
    const double *z_edges;   /* host, nz + 1 increasing depths, metres */
    double station_z;        /* station depth, metres (0 = top of the mesh) */
    int off_x, off_y;        /* prism columns left of / below the first station */
} gj_grid;

/* Inducing field for the total-field anomaly with induced magnetisation only
 * (Sec. 2.1: no remanence, no self-demagnetisation). */
typedef struct {
    double F_nT;             /* intensity, nT */
    double incl_deg;         /* inclination, degrees, positive down */
    double decl_deg;         /* declination, degrees east of north */
} gj_mag;

typedef struct gj_op gj_op;  /* opaque: one field's operator, its spectra and workspace */

typedef struct {
    int sx, sy, nx, ny, nz;
    int Nx, Ny;              /* padded BCCB sizes in use */
    int ncol;                /* stored spectrum columns, Nx/2 + 1 */
    gj_field field;
    gj_precision precision;
    int64_t spectrum_bytes;  /* device bytes of the stored layer spectra (one layer when
                                recomputed per layer) */
    int64_t workspace_bytes; /* device bytes of the per-op workspace */
    int fast_path;           /* 1: the specialised warp-FFT kernels serve this op (FP32,
                                Nx = 512 and Ny = 512 or 256, at most Nx/2 prisms and
                                stations along x and Ny/2 along y); 2: warp-FFT column
                                kernels (FP32, Ny = 1024, at most 512 prisms and stations
                                along y, any Nx) behind warp-FFT row kernels when
                                Nx = 1024 and the general row kernels otherwise; 0: the
                                general kernels */
    int P_row, C_col, L_grp; /* launch shapes of the general kernels (gj_op_tune) */
    int radix_order;         /* radix plan of the general kernels' transforms (gj_op_tune) */
    int recompute;           /* 1: spectra rebuilt per layer (GJ_SETUP_RECOMPUTE_SPECTRA) */
} gj_op_info_t;

/*
 * gj_bttb_setup - build one field's operator (Sec. 2.7.1, Eq. d=gm).
 *
 * Evaluates, in FP64 on the device, the closed-form prism field (vertical
 * gravity in mGal per g/cc, or total-field anomaly in nT per SI unit) for
 * every station-minus-prism offset of each depth layer, embeds each layer's
 * table T_r in an Ny x Nx circulant array (T[c mod N] = K(c + off) for
 * c in [-(n-1), s-1]), and keeps its 2-D FFT (scaled by 1/(Nx Ny)) in the
 * operator's precision.  Npad_y/Npad_x = 0 selects the smallest size
 * >= s + n - 1 whose prime factors are all <= 7; otherwise each must be
 * >= s + n - 1 with prime factors <= 17 (any such size gives the same
 * product).  In FP32, Npad = (512, 512) with at most 256 prisms and stations
 * per direction, or (256, 512) with at most 128 along y, selects the specialised
 * warp-FFT kernels; Npad_y = 1024 with at most 512 along y selects warp-FFT column
 * kernels, behind warp-FFT row kernels when Npad_x = 1024 and the general row
 * kernels otherwise (gj_op_info_t.fast_path); any other size runs the general
 * kernels.
 * `mag` is required for GJ_MAGNETIC and ignored for GJ_GRAVITY.
 * Synchronous with respect to the host on return (the op is ready).
 * Returns GJ_ERR_ARG for invalid sizes, GJ_ERR_UNSUPPORTED for a padded size
 * above 2048 or with a larger prime factor, GJ_ERR_OOM if device memory runs
 * out.  On success *out owns device memory until gj_op_destroy.
 */
gj_status gj_bttb_setup(const gj_grid *grid, gj_field field, const gj_mag *mag,
                        gj_precision precision, int Npad_y, int Npad_x,
                        gj_stream_t stream, gj_op **out);

/* Setup flags for gj_bttb_setup_ex. */
enum {
    /* Keep one layer's spectrum instead of all n_z: every product rebuilds each
     * layer's spectrum from the closed-form prism fields (FP64 corner lattice of
     * the layer's two depth planes, FP64 2-D FFT of its circulant table, rounded to
     * the operator's precision) just before using it (Sec. 2.7.1 applied per
     * layer).  The spectra are bit-identical to the stored ones; the cost is the
     * setup work of one layer per layer per product.  Served by the general
     * kernels (never the warp-FFT fast path); products only: the joint solver
     * rejects such operators with GJ_ERR_UNSUPPORTED. */
    GJ_SETUP_RECOMPUTE_SPECTRA = 1
};

/*
 * gj_bttb_setup_ex - gj_bttb_setup with setup flags (0 or
 * GJ_SETUP_RECOMPUTE_SPECTRA); gj_bttb_setup(...) equals gj_bttb_setup_ex(...,
 * 0, ...).  Unknown flags return GJ_ERR_ARG.
 */
gj_status gj_bttb_setup_ex(const gj_grid *grid, gj_field field, const gj_mag *mag,
                           gj_precision precision, int Npad_y, int Npad_x, int flags,
                           gj_stream_t stream, gj_op **out);

/* Sizes of an operator (host struct filled synchronously). */
gj_status gj_op_info(const gj_op *op, gj_op_info_t *info);

/*
 * gj_op_tune - launch shapes of the general (non-512) product kernels, the knobs
 * of the autotuner (the paper has no counterpart).  P_row: line pairs per CTA of
 * the row passes; C_col: columns per CTA of the column passes; L_grp: layers per
 * CTA of the layer-summed spectrum multiply; radix_order: the radix plan of the
 * transforms (0: radix 8 first, then the odd primes ascending; 1: the same stages
 * reversed; 2: radix 4 for the power-of-two part).  A value <= 0 (or < 0 for
 * radix_order) keeps the current choice.  Any choice gives the same products up
 * to rounding.  Synchronous, host-side only; GJ_ERR_ARG if a tile does not fit
 * in shared memory.  Not for operators in use on another stream.
 */
gj_status gj_op_tune(gj_op *op, int P_row, int C_col, int L_grp, int radix_order);

/* Frees an operator (waits for the device to finish using it).  NULL is a no-op. */
void gj_op_destroy(gj_op *op);

/*
 * gj_op_status - reads the operator's device error word (synchronises
 * `stream`).  Returns GJ_OK if no bounded wait of its kernels has given up,
 * else the recorded status (GJ_ERR_TIMEOUT).  With reset = 1 a recorded error
 * is also cleared together with the layer-sum arrival counters, which makes
 * the operator usable again; the products computed while it was set are not
 * repaired.  Operators off the fast path never wait and always return GJ_OK.
 * (A library safeguard; the paper has no counterpart.)
 */
gj_status gj_op_status(gj_op *op, int reset, gj_stream_t stream);

/*
 * gj_selftest_bounded_wait - runs the library's bounded mbarrier wait on a
 * barrier that nothing ever completes, giving up after limit_ns nanoseconds
 * (0 <= limit_ns <= 1e10), and returns the status the kernel recorded:
 * GJ_ERR_TIMEOUT when the bound works.  No copy is in flight, so nothing can
 * land after the wait gives up, and the context stays usable.  Synchronous;
 * allocates one int of device memory.  (A diagnostic of the failure path; the
 * paper has no counterpart.)
 */
gj_status gj_selftest_bounded_wait(int64_t limit_ns, gj_stream_t stream);

/*
 * gj_g_forward - d = A m for one field (Eq. d=gm): the sum over depth layers
 * of IFFT2(FFT2(T_r) . FFT2(X_r)) cropped to the station block, where X_r is
 * layer r of m in the upper-left corner of an Ny x Nx zero array
 * (Sec. 2.7.1).  m: n values, d: s values, both of the op's precision;
 * m and d must not overlap.
 *
 * Device-side failures (this and gj_g_adjoint): on the warp-FFT fast path the
 * column kernels wait on their bulk copies with a bound (200 ms per wait).  A
 * wait that gives up records GJ_ERR_TIMEOUT in the operator's error word and
 * leaves d (or g) incomplete; every later fast-path column launch of that
 * operator then returns at once (the operator is unusable) until
 * gj_op_status(op, 1, ...) reads and clears the word.  The call itself has
 * already returned GJ_OK by then, so check gj_op_status after products whose
 * results matter.
 *
 * Stream use (this, gj_g_adjoint and the pair forms): the call enqueues kernels
 * and asynchronous memsets on `stream` only, allocates nothing and does not
 * synchronise the host, so a sequence of products can be recorded by stream
 * capture into a CUDA graph once the operator has served one product outside
 * the capture (the first product sets the kernels' attributes); tested with
 * operators that store their spectra, on each kernel family.
 */
gj_status gj_g_forward(const gj_op *op, const void *m, void *d, gj_stream_t stream);

/*
 * gj_g_adjoint - g = A^T r for one field: per layer,
 * IFFT2(conj(FFT2(T_r)) . FFT2(V)) cropped to the prism block, V = r in the
 * upper-left corner (Sec. 2.7.1).  r: s values, g: n values.
 */
gj_status gj_g_adjoint(const gj_op *op, const void *r, void *g, gj_stream_t stream);

/*
 * gj_g_forward_pair / gj_g_adjoint_pair - the products of two operators in one
 * call: d[i] = A_i m[i] (or g[i] = A_i^T r[i]) for i = 0, 1, with the vectors as in
 * gj_g_forward / gj_g_adjoint.  When both operators are on the warp-FFT fast path
 * with the same grid and padded size (the gravity and magnetic operators of one joint problem), the
 * persistent column passes take both fields' columns in one launch, which fills the
 * GPU better than two single-field calls; the row passes stay per field, so that
 * the results round as the single-field products do.  Otherwise the call runs the
 * two products one after the other.  The two operators must differ
 * (each owns its workspace); failures as for the single products.
 */
gj_status gj_g_forward_pair(const gj_op *const ops[2], const void *const m[2], void *const d[2],
                            gj_stream_t stream);
gj_status gj_g_adjoint_pair(const gj_op *const ops[2], const void *const r[2], void *const g[2],
                            gj_stream_t stream);

/*
 * gj_gramian_value_grad - the Gramian coupling (Eq. Gramian, RRCG:2-3).
 * S = (m1,m1)(m2,m2) - (m1,m2)^2 written to the device double *S, and the
 * ascent directions l1 = (m2,m2) m1 - (m1,m2) m2, l2 = (m1,m1) m2 - (m1,m2) m1
 * (half the gradient of S).  l1 / l2 may be NULL to skip them.  Vectors of
 * length n in the given precision; inner products accumulate in FP64.
 */
gj_status gj_gramian_value_grad(int64_t n, gj_precision precision,
                                const void *m1, const void *m2, double *S,
                                void *l1, void *l2, gj_stream_t stream);

/*
 * gj_gramian_value_grad_noalloc - the same outputs as gj_gramian_value_grad,
 * for callers that must not allocate device memory: hosts whose device memory
 * is owned by another allocator (a framework's caching pool, a fixed arena), or
 * real-time loops that forbid allocation.  (The paper has no counterpart; this
 * is an interface for such callers.)
 *
 * The call allocates nothing: no cudaMalloc, cudaMallocAsync or cudaFree.  Its
 * reduction scratch is a fixed 131,096-byte device array inside the library,
 * which every GPU that loads the library holds until the process exits.  The
 * first call on each device looks up that array's device address
 * (cudaGetSymbolAddress, with the device current); make that first call before
 * any stream capture.  The address is kept per device index for the life of
 * the process: a caller that resets a device (cudaDeviceReset) must not call
 * this entry point on that device again.  Limit: n <= 16,777,216; larger n returns GJ_ERR_ARG
 * (use gj_gramian_value_grad).  All calls on a device share the array, which
 * keeps the last call's contents; every slot a call reads is written earlier
 * in the same call, so nothing needs clearing.  Calls that overlap on the GPU
 * (other streams, other host threads) race on the array: serialise them.
 * Arguments, outputs and precisions are those of gj_gramian_value_grad.
 */
gj_status gj_gramian_value_grad_noalloc(int64_t n, gj_precision precision,
                                        const void *m1, const void *m2, double *S,
                                        void *l1, void *l2, gj_stream_t stream);

/*
 * gj_pearson - Pearson correlation coefficient of the vectors a and b (n values
 * each, the given precision) into the device double *r: means first, then the
 * centred sums in FP64 (0 when either vector has no spread).  The measure of
 * "correlated models" in the lambda selection of Secs. 3.1.3 and 5, whose
 * figures judge it from density-susceptibility cross-plots.  Asynchronous on
 * `stream`; allocates its reduction scratch with cudaMallocAsync.
 */
gj_status gj_pearson(int64_t n, gj_precision precision, const void *a, const void *b, double *r,
                     gj_stream_t stream);

/* Solver options (Eq. RRCG:1-8; Secs. 2.5, 2.6, 2.8). Index 0 = gravity, 1 = magnetic. */
enum { GJ_SCALARS_AUTO = 0, GJ_SCALARS_JOINT = 1, GJ_SCALARS_PER_FIELD = 2 };
/* Regulariser anchor of RRCG:4: the a-priori model W_k m_apr (default; the first
 * variation, Eq. FirstVariation) or the previous weighted model W_{k-1} m_{k-1}
 * (the difference as printed in RRCG:4). */
enum { GJ_ANCHOR_APRIORI = 0, GJ_ANCHOR_PREVIOUS = 1 };
/* Space of the Gramian coupling: the original models (RRCG:2-3, the paper's
 * choice) or the weighted models W m (Eq. steepestascenta/b, Sec. 3.1.4). */
enum { GJ_GRAMIAN_ORIGINAL = 0, GJ_GRAMIAN_WEIGHTED = 1 };

typedef struct {
    int p[2];              /* Lp stabiliser, 1 (Eq. WL) or 2 (W_L = I, Sec. 3.1.5) */
    double eps2;           /* focusing parameter eps^2 of Eq. WL (paper: 1e-9) */
    double alpha1[2];      /* initial regularisation parameters */
    double q[2];           /* decay of Eq. regpara */
    double alpha_min[2];   /* lower bound on alpha (0 = none) */
    double lambda[2];      /* Lagrange parameters of the Gramian term */
    double lo[2], hi[2];   /* bounds of Sec. 2.5 */
    int kmax;              /* maximum number of model updates */
    int stop_on_chi2;      /* 1: stop once both fields pass Eq. chi2 */
    int scalars;           /* GJ_SCALARS_*: AUTO = per field iff both lambdas are 0 */
    int anchor;            /* GJ_ANCHOR_* */
    int gramian_space;     /* GJ_GRAMIAN_*; with WEIGHTED the history's S_G is the weighted Gramian */
} gj_rrcg_params;

typedef struct {
    int status;            /* GJ_OK, GJ_ERR_NONFINITE (a non-finite misfit or step length
                              stopped the solve) or GJ_ERR_TIMEOUT (a bounded wait of the
                              gravity operator's column kernels gave up; see gj_op_status) */
    int iterations;        /* model updates performed */
    int converged;         /* 1 if both fields passed Eq. chi2 */
    int satisfied[2];
    double phi[2];         /* chi^2 misfit of the returned models */
    double alpha[2];       /* regularisation parameters at the end */
    double S_G;            /* Gramian of the returned models */
} gj_rrcg_report;

/* Per-iteration history record (optional). */
typedef struct {
    double phi[2], alpha[2], S_G, s[2], beta[2];
} gj_rrcg_hist;

/*
 * gj_rrcg_joint_solve - joint RRCG solve of Eq. (GlobalFunction2) with the
 * Gramian in the original space (Eq. RRCG:1-8), bounds (Sec. 2.5), the chi^2
 * stop (Eq. chi2) and the alpha schedule (Eq. regpara).
 *
 * ops[0] is the gravity operator, ops[1] the magnetic one; both must have the
 * same grid sizes, padded sizes and precision.  dobs[i], sigma[i]: s values
 * (W_d = 1/sigma); w_depth[i]: nz per-layer depth weights; w_hard[i]: n values
 * or NULL (identity); m_apr[i]: n values or NULL (zero).  m[i]: n values, the
 * starting model on entry, the result on return.  hist: device array of
 * kmax + 1 records or NULL.  *rep (host) is filled on return; the call
 * synchronises `stream`.  Non-convergence by kmax is not an error
 * (rep->converged = 0).
 */
gj_status gj_rrcg_joint_solve(const gj_op *const ops[2], const gj_rrcg_params *params,
                              const void *const dobs[2], const void *const sigma[2],
                              const void *const m_apr[2], const void *const w_depth[2],
                              const void *const w_hard[2], void *const m[2],
                              gj_rrcg_hist *hist, gj_rrcg_report *rep, gj_stream_t stream);

/*
 * gj_rrcg_joint_solve_host - the same solve with HOST buffers: dobs, sigma,
 * w_depth, m_apr, w_hard and m are host pointers (m: the starting models on
 * entry, the result on return); everything else is as in gj_rrcg_joint_solve
 * (no history).  The call allocates one device block for the copies, copies
 * the inputs in with cudaMemcpyAsync on `stream` (page-locked host memory lets
 * the copies run asynchronously), solves, copies both models back, frees the
 * block and synchronises `stream`.  On GJ_ERR_NONFINITE the models are still
 * copied back.
 */
gj_status gj_rrcg_joint_solve_host(const gj_op *const ops[2], const gj_rrcg_params *params,
                                   const void *const dobs[2], const void *const sigma[2],
                                   const void *const m_apr[2], const void *const w_depth[2],
                                   const void *const w_hard[2], void *const m[2],
                                   gj_rrcg_report *rep, gj_stream_t stream);

/* Stepwise form of the same solve: a solver object holds the state (search
 * directions, scalars) and enqueues whole iterations without host round trips;
 * the stop test runs on the device and later iterations become no-ops. */
typedef struct gj_rrcg gj_rrcg;

gj_status gj_rrcg_create(const gj_op *const ops[2], const gj_rrcg_params *params,
                         const void *const dobs[2], const void *const sigma[2],
                         const void *const m_apr[2], const void *const w_depth[2],
                         const void *const w_hard[2], void *const m[2],
                         gj_rrcg_hist *hist, gj_stream_t stream, gj_rrcg **out);
/* Enqueue `iters` iterations (each: 2 forward and 1 adjoint product per field
 * plus the fused vector updates).  use_graph = 1 replays one captured CUDA
 * graph per iteration. */
gj_status gj_rrcg_iterate(gj_rrcg *solver, int iters, int use_graph, gj_stream_t stream);
/* Synchronises `stream` and fills *rep (host). */
gj_status gj_rrcg_report_get(gj_rrcg *solver, gj_rrcg_report *rep, gj_stream_t stream);
/* Writes the same report into DEVICE memory `rep` (one thread, asynchronous on
 * `stream`, no host round trip), e.g. from inside a captured loop. */
gj_status gj_rrcg_report_device(gj_rrcg *solver, gj_rrcg_report *rep, gj_stream_t stream);
/* Synchronises `stream`; returns 1 once the device-side stop flag is set, 0 if
 * not, -1 on error. */
int gj_rrcg_done(gj_rrcg *solver, gj_stream_t stream);
/* Kernel timing for roofline measurements: while enabled, a CUDA event pair is
 * recorded on the launching stream around every launch of the spectrum
 * multiply-and-sum column kernel (two per iteration).  Enabling it drops a graph
 * captured without the events.  gj_rrcg_profile_read synchronises the device and
 * returns the number of timed launches and their total milliseconds since the
 * previous read (for graph replays: the launches of the last replay). */
gj_status gj_rrcg_profile(gj_rrcg *solver, int enable);
gj_status gj_rrcg_profile_read(gj_rrcg *solver, int *launches, double *total_ms);
void gj_rrcg_destroy(gj_rrcg *solver);

/*
 * Batched form: several independent joint inversions, of any sizes and
 * precisions, advanced together.  gj_rrcg_batch_create captures one CUDA graph
 * whose parallel branches are one iteration of each solver (as in
 * gj_rrcg_iterate); gj_rrcg_batch_step replays it `iters` times on `stream`, so
 * one launch advances every problem by one RRCG iteration (solvers that have
 * stopped do no work).  The solvers stay owned by the caller and must outlive
 * the batch; while a batch exists, do not step its solvers on other streams.
 * The branches run concurrently, so no two solvers may share an operator (each
 * gj_op owns one workspace): GJ_ERR_ARG otherwise.
 */
typedef struct gj_rrcg_batch gj_rrcg_batch;
gj_status gj_rrcg_batch_create(gj_rrcg *const *solvers, int count, gj_stream_t stream, gj_rrcg_batch **out);
gj_status gj_rrcg_batch_step(gj_rrcg_batch *batch, int iters, gj_stream_t stream);
void gj_rrcg_batch_destroy(gj_rrcg_batch *batch);

/*
 * gj_probe_fma_rate - measures the device's fused multiply-add rate (a roofline
 * denominator for the FFT kernels; the paper has no counterpart).  kind 0: FP32
 * fma.rn.f32, 1: paired FP32 fma.rn.f32x2 (two FMAs per instruction), 2: FP64
 * fma.rn.f64.  A grid of 8 blocks of 256 threads per SM runs `iters` x 128
 * independent FMAs per thread (eight chains); the second of two launches is
 * timed with CUDA events on `stream`.  *gflops = 2 x FMAs / time, *ms = the
 * launch's time.  Synchronous; allocates 8 bytes of device memory.
 */
gj_status gj_probe_fma_rate(int kind, int iters, double *gflops, double *ms, gj_stream_t stream);

/* Last error message of the calling thread ("" if none). */
const char *gj_last_error(void);

/* Library version string. */
const char *gj_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GJ_H */
