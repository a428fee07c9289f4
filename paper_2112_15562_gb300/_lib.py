"""ctypes declarations of ``include/gj.h`` (argument marshalling only)."""
from __future__ import annotations

import ctypes as ct
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgj.so")

GJ_OK = 0
STATUS = {0: "GJ_OK", -1: "GJ_ERR_ARG", -2: "GJ_ERR_OOM", -3: "GJ_ERR_CUDA", -4: "GJ_ERR_NONFINITE",
          -5: "GJ_ERR_TIMEOUT", -6: "GJ_ERR_UNSUPPORTED"}
STATUS_CODE = {v: k for k, v in STATUS.items()}
GJ_GRAVITY, GJ_MAGNETIC = 1, 2
GJ_FP64, GJ_FP32_MIXED = 0, 1
GJ_SCALARS_AUTO, GJ_SCALARS_JOINT, GJ_SCALARS_PER_FIELD = 0, 1, 2
GJ_SETUP_RECOMPUTE_SPECTRA = 1


class GJError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(ct.Structure):
    _fields_ = [("sx", ct.c_int), ("sy", ct.c_int), ("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
                ("dx", ct.c_double), ("dy", ct.c_double), ("z_edges", ct.POINTER(ct.c_double)),
                ("station_z", ct.c_double), ("off_x", ct.c_int), ("off_y", ct.c_int)]


class Mag(ct.Structure):
    _fields_ = [("F_nT", ct.c_double), ("incl_deg", ct.c_double), ("decl_deg", ct.c_double)]


class OpInfo(ct.Structure):
    _fields_ = [("sx", ct.c_int), ("sy", ct.c_int), ("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
                ("Nx", ct.c_int), ("Ny", ct.c_int), ("ncol", ct.c_int), ("field", ct.c_int),
                ("precision", ct.c_int), ("spectrum_bytes", ct.c_int64), ("workspace_bytes", ct.c_int64),
                ("fast_path", ct.c_int), ("P_row", ct.c_int), ("C_col", ct.c_int), ("L_grp", ct.c_int),
                ("radix_order", ct.c_int), ("recompute", ct.c_int)]


class RRCGParams(ct.Structure):
    _fields_ = [("p", ct.c_int * 2), ("eps2", ct.c_double), ("alpha1", ct.c_double * 2), ("q", ct.c_double * 2),
                ("alpha_min", ct.c_double * 2), ("lambda_", ct.c_double * 2), ("lo", ct.c_double * 2),
                ("hi", ct.c_double * 2), ("kmax", ct.c_int), ("stop_on_chi2", ct.c_int), ("scalars", ct.c_int),
                ("anchor", ct.c_int), ("gramian_space", ct.c_int)]


class RRCGReport(ct.Structure):
    _fields_ = [("status", ct.c_int), ("iterations", ct.c_int), ("converged", ct.c_int),
                ("satisfied", ct.c_int * 2), ("phi", ct.c_double * 2), ("alpha", ct.c_double * 2),
                ("S_G", ct.c_double)]


class RRCGHist(ct.Structure):
    _fields_ = [("phi", ct.c_double * 2), ("alpha", ct.c_double * 2), ("S_G", ct.c_double),
                ("s", ct.c_double * 2), ("beta", ct.c_double * 2)]


_lib = None


def load() -> ct.CDLL:
    """Loads libgj.so; raises if the CUDA library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2112_15562_gb300.build.build() "
                          "(there is no CPU fallback)")
    L = ct.CDLL(LIB_PATH)
    vp, i32, i64, d = ct.c_void_p, ct.c_int, ct.c_int64, ct.c_double
    pp = ct.POINTER(vp)
    sig = {
        "gj_bttb_setup": (i32, [ct.POINTER(Grid), i32, ct.POINTER(Mag), i32, i32, i32, vp, pp]),
        "gj_bttb_setup_ex": (i32, [ct.POINTER(Grid), i32, ct.POINTER(Mag), i32, i32, i32, i32, vp, pp]),
        "gj_op_info": (i32, [vp, ct.POINTER(OpInfo)]),
        "gj_op_tune": (i32, [vp, i32, i32, i32, i32]),
        "gj_op_destroy": (None, [vp]),
        "gj_op_status": (i32, [vp, i32, vp]),
        "gj_selftest_bounded_wait": (i32, [i64, vp]),
        "gj_g_forward": (i32, [vp, vp, vp, vp]),
        "gj_g_adjoint": (i32, [vp, vp, vp, vp]),
        "gj_g_forward_pair": (i32, [pp, pp, pp, vp]),
        "gj_g_adjoint_pair": (i32, [pp, pp, pp, vp]),
        "gj_gramian_value_grad": (i32, [i64, i32, vp, vp, vp, vp, vp, vp]),
        "gj_gramian_value_grad_noalloc": (i32, [i64, i32, vp, vp, vp, vp, vp, vp]),
        "gj_rrcg_joint_solve": (i32, [pp, ct.POINTER(RRCGParams), pp, pp, pp, pp, pp, pp, vp,
                                      ct.POINTER(RRCGReport), vp]),
        "gj_rrcg_joint_solve_host": (i32, [pp, ct.POINTER(RRCGParams), pp, pp, pp, pp, pp, pp,
                                           ct.POINTER(RRCGReport), vp]),
        "gj_rrcg_create": (i32, [pp, ct.POINTER(RRCGParams), pp, pp, pp, pp, pp, pp, vp, vp, pp]),
        "gj_rrcg_iterate": (i32, [vp, i32, i32, vp]),
        "gj_rrcg_report_get": (i32, [vp, ct.POINTER(RRCGReport), vp]),
        "gj_rrcg_done": (i32, [vp, vp]),
        "gj_rrcg_report_device": (i32, [vp, vp, vp]),
        "gj_pearson": (i32, [i64, i32, vp, vp, vp, vp]),
        "gj_rrcg_profile": (i32, [vp, i32]),
        "gj_rrcg_profile_read": (i32, [vp, ct.POINTER(i32), ct.POINTER(d)]),
        "gj_rrcg_destroy": (None, [vp]),
        "gj_rrcg_batch_create": (i32, [pp, i32, vp, pp]),
        "gj_rrcg_batch_step": (i32, [vp, i32, vp]),
        "gj_rrcg_batch_destroy": (None, [vp]),
        "gj_probe_fma_rate": (i32, [i32, i32, ct.POINTER(d), ct.POINTER(d), vp]),
        "gj_last_error": (ct.c_char_p, []),
        "gj_version": (ct.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(status: int) -> None:
    if status != GJ_OK:
        raise GJError(status, load().gj_last_error().decode())
