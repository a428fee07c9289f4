// Device view of a host-side operator.
#pragma once
#include "bttb_kernels.cuh"
#include "gj_internal.h"

namespace gj {

template <typename R>
inline OpView<R> view_of(const gj_op *op) {
    OpView<R> v;
    v.sx = op->sx; v.sy = op->sy; v.nx = op->nx; v.ny = op->ny; v.nz = op->nz;
    v.Nx = op->Nx; v.Ny = op->Ny; v.ncol = op->ncol;
    v.px = op->px; v.py = op->py;
    v.twx = static_cast<const cpx<R> *>(op->twx);
    v.twy = static_cast<const cpx<R> *>(op->twy);
    v.spec = static_cast<const cpx<R> *>(op->spec);
    v.Z = static_cast<cpx<R> *>(op->Z);
    v.Y = static_cast<cpx<R> *>(op->Y);
    v.W = static_cast<cpx<R> *>(op->W);
    v.V = static_cast<cpx<R> *>(op->V);
    v.real_spec = op->real_spec ? 1 : 0;
    v.rbase = 0;
    v.spec_r0 = 0;
    v.tcol = op->fast1024 ? op->Ny / 2 : 0;
    return v;
}

inline size_t row_smem(int Nx, int P, size_t cs) { return (size_t)(2 * Nx * P + Nx) * cs; }
inline size_t col_smem(int Ny, int C, int nbuf, size_t cs) { return (size_t)(nbuf * Ny * C + Ny) * cs; }

}  // namespace gj
