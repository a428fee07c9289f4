"""Python-facing wrappers with the C-ABI names (argument marshalling only)."""
from __future__ import annotations

import ctypes as ct
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L
from ._lib import check, load

_PREC = {"fp64": L.GJ_FP64, "fp32": L.GJ_FP32_MIXED, L.GJ_FP64: L.GJ_FP64, L.GJ_FP32_MIXED: L.GJ_FP32_MIXED}
_FIELD = {"gravity": L.GJ_GRAVITY, "magnetic": L.GJ_MAGNETIC, L.GJ_GRAVITY: L.GJ_GRAVITY,
          L.GJ_MAGNETIC: L.GJ_MAGNETIC}


def _stream(stream=None) -> ct.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ct.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[ct.c_void_p]:
    return None if t is None else ct.c_void_p(t.data_ptr())


def _vec(t: torch.Tensor, dtype, n: int, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of {n} values")
    return t


class Op:
    """One field's BTTB operator (owns device spectra and workspace)."""

    def __init__(self, handle: int, info: L.OpInfo):
        self._h = ct.c_void_p(handle)
        self.info = info
        self.precision = info.precision
        self.dtype = torch.float64 if info.precision == L.GJ_FP64 else torch.float32
        self.n = info.nx * info.ny * info.nz
        self.s = info.sx * info.sy

    @property
    def handle(self):
        return self._h

    def forward(self, m: torch.Tensor, d: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        return g_forward(self, m, d, stream)

    def adjoint(self, r: torch.Tensor, g: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        return g_adjoint(self, r, g, stream)

    def tune(self, P_row: int = 0, C_col: int = 0, L_grp: int = 0, radix_order: int = -1):
        """gj_op_tune: launch shapes and radix plan of the general product kernels."""
        check(load().gj_op_tune(self._h, int(P_row), int(C_col), int(L_grp), int(radix_order)))
        check(load().gj_op_info(self._h, ct.byref(self.info)))

    def tiles(self) -> dict:
        """The general kernels' current launch shapes and radix plan."""
        return {"P_row": self.info.P_row, "C_col": self.info.C_col, "L_grp": self.info.L_grp,
                "radix_order": self.info.radix_order}

    def close(self):
        if self._h is not None and self._h.value:
            load().gj_op_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bttb_setup(grid, field, mag=None, precision="fp32", npad=(0, 0), stream=None, recompute=False) -> Op:
    """gj_bttb_setup_ex: ``grid`` has sx, sy, nx, ny, nz, dx, dy, z_edges[, station_z, off_x, off_y];
    ``mag`` has F, incl, decl (magnetic only); ``recompute`` keeps one layer's spectrum and
    rebuilds each layer's spectrum in every product (GJ_SETUP_RECOMPUTE_SPECTRA)."""
    lib = load()
    z = np.ascontiguousarray(np.asarray(grid.z_edges, dtype=np.float64))
    g = L.Grid(int(grid.sx), int(grid.sy), int(grid.nx), int(grid.ny), int(grid.nz), float(grid.dx),
               float(grid.dy), z.ctypes.data_as(ct.POINTER(ct.c_double)), float(getattr(grid, "station_z", 0.0)),
               int(getattr(grid, "off_x", 0)), int(getattr(grid, "off_y", 0)))
    m = None
    if mag is not None:
        m = L.Mag(float(mag.F), float(mag.incl), float(mag.decl))
    out = ct.c_void_p()
    check(lib.gj_bttb_setup_ex(ct.byref(g), _FIELD[field], ct.byref(m) if m is not None else None,
                               _PREC[precision], int(npad[0]), int(npad[1]),
                               L.GJ_SETUP_RECOMPUTE_SPECTRA if recompute else 0, _stream(stream), ct.byref(out)))
    info = L.OpInfo()
    check(lib.gj_op_info(out, ct.byref(info)))
    return Op(out.value, info)


def g_forward(op: Op, m: torch.Tensor, d: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """gj_g_forward: d = A m."""
    _vec(m, op.dtype, op.n, "m")
    if d is None:
        d = torch.empty(op.s, dtype=op.dtype, device=m.device)
    _vec(d, op.dtype, op.s, "d")
    check(load().gj_g_forward(op.handle, _ptr(m), _ptr(d), _stream(stream)))
    return d


def g_adjoint(op: Op, r: torch.Tensor, g: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """gj_g_adjoint: g = A^T r."""
    _vec(r, op.dtype, op.s, "r")
    if g is None:
        g = torch.empty(op.n, dtype=op.dtype, device=r.device)
    _vec(g, op.dtype, op.n, "g")
    check(load().gj_g_adjoint(op.handle, _ptr(r), _ptr(g), _stream(stream)))
    return g


def g_forward_pair(ops: Sequence[Op], m, d=None, stream=None):
    """gj_g_forward_pair: d[i] = A_i m[i] for both operators in one call."""
    if ops[0] is ops[1]:
        raise ValueError("the two operators must differ")
    for i in range(2):
        _vec(m[i], ops[i].dtype, ops[i].n, f"m[{i}]")
    if d is None:
        d = [torch.empty(ops[i].s, dtype=ops[i].dtype, device=m[i].device) for i in range(2)]
    for i in range(2):
        _vec(d[i], ops[i].dtype, ops[i].s, f"d[{i}]")
    handles = (ct.c_void_p * 2)(ops[0].handle.value, ops[1].handle.value)
    check(load().gj_g_forward_pair(handles, (ct.c_void_p * 2)(m[0].data_ptr(), m[1].data_ptr()),
                                   (ct.c_void_p * 2)(d[0].data_ptr(), d[1].data_ptr()), _stream(stream)))
    return d


def g_adjoint_pair(ops: Sequence[Op], r, g=None, stream=None):
    """gj_g_adjoint_pair: g[i] = A_i^T r[i] for both operators in one call."""
    if ops[0] is ops[1]:
        raise ValueError("the two operators must differ")
    for i in range(2):
        _vec(r[i], ops[i].dtype, ops[i].s, f"r[{i}]")
    if g is None:
        g = [torch.empty(ops[i].n, dtype=ops[i].dtype, device=r[i].device) for i in range(2)]
    for i in range(2):
        _vec(g[i], ops[i].dtype, ops[i].n, f"g[{i}]")
    handles = (ct.c_void_p * 2)(ops[0].handle.value, ops[1].handle.value)
    check(load().gj_g_adjoint_pair(handles, (ct.c_void_p * 2)(r[0].data_ptr(), r[1].data_ptr()),
                                   (ct.c_void_p * 2)(g[0].data_ptr(), g[1].data_ptr()), _stream(stream)))
    return g


def gramian_value_grad(m1: torch.Tensor, m2: torch.Tensor, want_dirs: bool = True, stream=None):
    """gj_gramian_value_grad: returns (S as a 1-element float64 CUDA tensor, l1, l2)."""
    if m1.dtype not in (torch.float32, torch.float64) or m2.dtype != m1.dtype:
        raise ValueError("m1 and m2 must share float32 or float64")
    n = m1.numel()
    _vec(m1, m1.dtype, n, "m1")
    _vec(m2, m1.dtype, n, "m2")
    prec = L.GJ_FP64 if m1.dtype == torch.float64 else L.GJ_FP32_MIXED
    S = torch.empty(1, dtype=torch.float64, device=m1.device)
    l1 = torch.empty_like(m1) if want_dirs else None
    l2 = torch.empty_like(m2) if want_dirs else None
    check(load().gj_gramian_value_grad(n, prec, _ptr(m1), _ptr(m2), _ptr(S), _ptr(l1), _ptr(l2), _stream(stream)))
    return S, l1, l2


def solver_params(p=(1, 1), eps2=1e-9, alpha1=(2e4, 2e4), q=(0.95, 0.95), alpha_min=(0.0, 0.0),
                  lam=(0.0, 0.0), lo=(0.0, 0.0), hi=(1.0, 0.1), kmax=50, stop_on_chi2=True,
                  scalars="auto", anchor="apriori", gramian_space="original") -> L.RRCGParams:
    P = L.RRCGParams()
    P.p[:] = [int(v) for v in p]
    P.eps2 = float(eps2)
    P.alpha1[:] = [float(v) for v in alpha1]
    P.q[:] = [float(v) for v in q]
    P.alpha_min[:] = [float(v) for v in alpha_min]
    P.lambda_[:] = [float(v) for v in lam]
    P.lo[:] = [float(v) for v in lo]
    P.hi[:] = [float(v) for v in hi]
    P.kmax = int(kmax)
    P.stop_on_chi2 = 1 if stop_on_chi2 else 0
    P.scalars = {"auto": L.GJ_SCALARS_AUTO, "joint": L.GJ_SCALARS_JOINT, "per_field": L.GJ_SCALARS_PER_FIELD}[scalars]
    P.anchor = {"apriori": 0, "previous": 1}[anchor]
    P.gramian_space = {"original": 0, "weighted": 1}[gramian_space]
    return P


def _pair(vals, name, op, n, allow_none=False):
    arr = (ct.c_void_p * 2)()
    if vals is None:
        if not allow_none:
            raise ValueError(f"{name} is required")
        return None
    for i in range(2):
        v = vals[i]
        if v is None:
            if not allow_none:
                raise ValueError(f"{name}[{i}] is required")
            arr[i] = None
        else:
            _vec(v, op.dtype, n, f"{name}[{i}]")
            arr[i] = v.data_ptr()
    return arr


def _report(rep: L.RRCGReport) -> dict:
    return {"status": rep.status, "iterations": rep.iterations, "converged": bool(rep.converged),
            "satisfied": [bool(rep.satisfied[0]), bool(rep.satisfied[1])], "phi": list(rep.phi),
            "alpha": list(rep.alpha), "S_G": rep.S_G}


def _hist_rows(h: torch.Tensor, count: int):
    a = h[:count].cpu().numpy()
    return [{"phi": list(r[0:2]), "alpha": list(r[2:4]), "S_G": float(r[4]), "s": list(r[5:7]),
             "beta": list(r[7:9])} for r in a]


class Solver:
    """Stepwise joint RRCG (gj_rrcg_create / iterate / report_get)."""

    def __init__(self, ops: Sequence[Op], params: L.RRCGParams, dobs, sigma, w_depth, m, m_apr=None,
                 w_hard=None, history=False, stream=None):
        lib = load()
        self.ops = list(ops)
        o = ops[0]
        self._keep = [dobs, sigma, w_depth, m, m_apr, w_hard]
        self.hist = None
        if history:
            self.hist = torch.zeros((params.kmax + 1, 9), dtype=torch.float64, device=m[0].device)
        handles = (ct.c_void_p * 2)(ops[0].handle.value, ops[1].handle.value)
        out = ct.c_void_p()
        nz = o.info.nz
        check(lib.gj_rrcg_create(handles, ct.byref(params), _pair(dobs, "dobs", o, o.s), _pair(sigma, "sigma", o, o.s),
                                 _pair(m_apr, "m_apr", o, o.n, True), _pair(w_depth, "w_depth", o, nz),
                                 _pair(w_hard, "w_hard", o, o.n, True), _pair(m, "m", o, o.n),
                                 _ptr(self.hist), _stream(stream), ct.byref(out)))
        self._h = out
        self.kmax = params.kmax

    def iterate(self, iters: int, use_graph: bool = True, stream=None):
        check(load().gj_rrcg_iterate(self._h, int(iters), 1 if use_graph else 0, _stream(stream)))

    def done(self, stream=None) -> bool:
        d = load().gj_rrcg_done(self._h, _stream(stream))
        if d < 0:
            check(-3)
        return bool(d)

    def report(self, stream=None) -> dict:
        rep = L.RRCGReport()
        check(load().gj_rrcg_report_get(self._h, ct.byref(rep), _stream(stream)))
        out = _report(rep)
        if self.hist is not None:
            out["history"] = _hist_rows(self.hist, out["iterations"] + 1)
        return out

    def profile(self, enable: bool = True):
        check(load().gj_rrcg_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        n = ct.c_int()
        ms = ct.c_double()
        check(load().gj_rrcg_profile_read(self._h, ct.byref(n), ct.byref(ms)))
        return n.value, ms.value

    def close(self):
        if self._h is not None and self._h.value:
            load().gj_rrcg_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rrcg_joint_solve(ops: Sequence[Op], params: L.RRCGParams, dobs, sigma, w_depth, m, m_apr=None, w_hard=None,
                     history=False, stream=None) -> dict:
    """gj_rrcg_joint_solve on device tensors; m (two tensors) is updated in place."""
    lib = load()
    o = ops[0]
    hist = torch.zeros((params.kmax + 1, 9), dtype=torch.float64, device=m[0].device) if history else None
    handles = (ct.c_void_p * 2)(ops[0].handle.value, ops[1].handle.value)
    rep = L.RRCGReport()
    check(lib.gj_rrcg_joint_solve(handles, ct.byref(params), _pair(dobs, "dobs", o, o.s),
                                  _pair(sigma, "sigma", o, o.s), _pair(m_apr, "m_apr", o, o.n, True),
                                  _pair(w_depth, "w_depth", o, o.info.nz), _pair(w_hard, "w_hard", o, o.n, True),
                                  _pair(m, "m", o, o.n), _ptr(hist), ct.byref(rep), _stream(stream)))
    out = _report(rep)
    if hist is not None:
        out["history"] = _hist_rows(hist, out["iterations"] + 1)
    return out


def _host_vec(x, dtype, n: int, name: str, writable: bool = False):
    """A host buffer for the C ABI: a contiguous CPU tensor (e.g. page-locked) or numpy
    array of the op's dtype and length n; returns (keep-alive object, address)."""
    if isinstance(x, torch.Tensor):
        if x.is_cuda or x.dtype != dtype or not x.is_contiguous() or x.numel() != n:
            raise ValueError(f"{name} must be a contiguous CPU {dtype} tensor of {n} values")
        return x, x.data_ptr()
    a = np.asarray(x)
    want = np.float64 if dtype == torch.float64 else np.float32
    if a.dtype != want or not a.flags.c_contiguous or a.size != n or (writable and not a.flags.writeable):
        raise ValueError(f"{name} must be a contiguous writable {want.__name__} array of {n} values")
    return a, a.ctypes.data


def rrcg_joint_solve_host(ops: Sequence[Op], params: L.RRCGParams, dobs, sigma, w_depth, m, m_apr=None,
                          w_hard=None, stream=None) -> dict:
    """gj_rrcg_joint_solve_host: the solve with host buffers (CPU tensors or numpy arrays of
    the op's dtype); the library copies them in, solves and copies the models back into m.
    The report carries the bytes copied each way."""
    o = ops[0]
    keep = []

    def arr(vals, name, n, allow_none=False, writable=False):
        if vals is None:
            return None
        a = (ct.c_void_p * 2)()
        for i in range(2):
            if vals[i] is None:
                if not allow_none:
                    raise ValueError(f"{name}[{i}] is required")
                a[i] = None
            else:
                k, ptr = _host_vec(vals[i], o.dtype, n, f"{name}[{i}]", writable)
                keep.append(k)
                a[i] = ptr
        return a

    handles = (ct.c_void_p * 2)(ops[0].handle.value, ops[1].handle.value)
    rep = L.RRCGReport()
    args = (arr(dobs, "dobs", o.s), arr(sigma, "sigma", o.s), arr(m_apr, "m_apr", o.n, True),
            arr(w_depth, "w_depth", o.info.nz), arr(w_hard, "w_hard", o.n, True), arr(m, "m", o.n, writable=True))
    check(load().gj_rrcg_joint_solve_host(handles, ct.byref(params), *args, ct.byref(rep), _stream(stream)))
    es = 8 if o.dtype == torch.float64 else 4
    out = _report(rep)
    nin = 2 * (2 * o.s + o.info.nz + o.n) + (2 * o.n if m_apr is not None else 0) + (2 * o.n if w_hard is not None else 0)
    out["h2d_bytes"] = nin * es
    out["d2h_bytes"] = 2 * o.n * es
    return out


class Batch:
    """Several Solvers advanced together by one CUDA graph (gj_rrcg_batch_*)."""

    def __init__(self, solvers: Sequence[Solver], stream=None):
        lib = load()
        self.solvers = list(solvers)
        arr = (ct.c_void_p * len(self.solvers))(*[s._h.value for s in self.solvers])
        out = ct.c_void_p()
        check(lib.gj_rrcg_batch_create(arr, len(self.solvers), _stream(stream), ct.byref(out)))
        self._h = out

    def step(self, iters: int = 1, stream=None):
        check(load().gj_rrcg_batch_step(self._h, int(iters), _stream(stream)))

    def all_done(self, stream=None) -> bool:
        return all(s.done(stream) for s in self.solvers)

    def close(self):
        if self._h is not None and self._h.value:
            load().gj_rrcg_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
