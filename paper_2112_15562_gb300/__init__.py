"""GB300 joint gravity-magnetic inversion (arXiv 2112.15562).

Python binding of the CUDA library ``libgj.so`` (C ABI in ``include/gj.h``).
The binding only marshals arguments: every step of the BTTB/FFT products, the
Gramian and the RRCG solve runs in the library's kernels.  PyTorch supplies
device memory and streams.  There is no CPU fallback: if the library is not
built the calls raise.
"""
from ._lib import (GJ_FP32_MIXED, GJ_FP64, GJ_GRAVITY, GJ_MAGNETIC, GJ_SCALARS_AUTO, GJ_SCALARS_JOINT,
                   GJ_SCALARS_PER_FIELD, GJError)
from .api import (Batch, Op, Solver, bttb_setup, g_adjoint, g_adjoint_pair, g_forward, g_forward_pair,
                  gramian_value_grad,
                  rrcg_joint_solve, rrcg_joint_solve_host, solver_params)
from .autograd import G, GT, gramian
from .sweep import lambda_sweep, pearson

__all__ = ["lambda_sweep", "pearson", "Batch", "G", "GT", "gramian", "Op", "Solver", "bttb_setup", "g_forward", "g_adjoint", "g_forward_pair", "g_adjoint_pair", "gramian_value_grad", "rrcg_joint_solve",
           "rrcg_joint_solve_host", "solver_params", "GJError", "GJ_FP64", "GJ_FP32_MIXED",
           "GJ_GRAVITY", "GJ_MAGNETIC", "GJ_SCALARS_AUTO", "GJ_SCALARS_JOINT", "GJ_SCALARS_PER_FIELD"]
