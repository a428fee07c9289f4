// Host-side internals shared by the translation units of the library.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/gj.h"
#include "fft.cuh"

namespace gj { struct gj_setup_scratch_impl; }

struct gj_op {
    // geometry
    int sx, sy, nx, ny, nz, off_x, off_y;
    double dx, dy, station_z;
    std::vector<double> z_edges;
    gj_field field;
    gj_mag mag;
    gj_precision prec;
    // padded sizes and plans
    int Nx, Ny, ncol;
    gj::FftPlanDev px, py;
    // device memory (op precision unless noted)
    void *twx = nullptr, *twy = nullptr;  // twiddles W_N^k
    void *spec = nullptr;                 // [nz][Ny][ncol] complex
    void *Z = nullptr, *Y = nullptr, *W = nullptr, *V = nullptr;
    size_t spec_bytes = 0, ws_bytes = 0;
    // launch shapes
    int P_row = 8, C_col = 8, L_grp = 4;
    int radix_order = 0;
    // fast path (FP32, N_x = 512 and N_y = 512 or 256, at most N/2 prisms and stations
    // per direction): transposed spectra and intermediates, layer-sum partials and counters
    bool fast = false;
    bool real_spec = false;  // fast path: the table is even in both offsets, its spectrum is real
    void *P = nullptr;     // [ncol][slots][Ny] complex
    int *cnt = nullptr;    // [ncol] arrival counters
    int *err = nullptr;    // device error word (bounded waits)
    void *twtab = nullptr; // the column kernels' twiddle table (FP32, TabTw or Tab1024 layout)
    // N_y = 1024 (FP32, at most 512 prisms and stations per column): warp-FFT column
    // kernels with the general row kernels writing and reading transposed Z, W, V;
    // spectra, partials, counters and the error word as on the fast path
    bool fast1024 = false;
    // per-layer spectrum recomputation (GJ_SETUP_RECOMPUTE_SPECTRA): `spec` holds one
    // layer, rebuilt from the closed forms before each use
    bool recompute = false;
    gj::gj_setup_scratch_impl *scratch = nullptr;
    int slots = 0;
    int col_grid = 0;      // CTAs of the persistent column kernels
};

namespace gj {

void set_error(const std::string &msg);
gj_status cuda_fail(cudaError_t e, const char *what);
bool plan_size(int N, FftPlanDev &plan, int order = 0);  // false if N has an unsupported factor
int  autotune_size(int minN);               // smallest 7-smooth N >= minN
size_t elem_bytes(gj_precision p);           // bytes of one real value
void make_twiddles(int N, std::vector<double> &re, std::vector<double> &im);

// smem sizing helpers
int pick_row_pairs(int Nx, size_t csize);
int pick_col_tile(int Ny, size_t csize, int nbuf);

template <typename R> struct OpView;
template <typename R> OpView<R> view_of(const gj_op *op);

// fast-path helpers (setup.cu)
bool fast_eligible(const gj_op *op);
int fast_col_items(int Ny, int nz);  // items per column of the fast column kernels
// partial slots per column for persistent column kernels of `warps` warps in total
int fast_slots(int nfield, int ncol, int items_per_col, long long warps);
bool fast1024_eligible(const gj_op *op);

// rebuilds layer r's spectrum into spec (recompute mode; setup.cu)
void recompute_layer(const gj_op *op, int r, cudaStream_t st);

// enqueue products (matvec.cu)
gj_status forward_enqueue(const gj_op *op, const void *m, void *d, cudaStream_t s);
gj_status adjoint_enqueue(const gj_op *op, const void *r, void *g, cudaStream_t s);

}  // namespace gj

#define GJ_CUDA(call)                                                  \
    do {                                                               \
        cudaError_t _e = (call);                                       \
        if (_e != cudaSuccess) return gj::cuda_fail(_e, #call);        \
    } while (0)
