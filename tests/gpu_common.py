"""Helpers for the GPU parity tests (test infrastructure)."""
import numpy as np
import pytest

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def lib():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2112_15562_gb300 as gj

    return gj


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def to_dev(x, prec):
    import torch

    dt = torch.float64 if prec == "fp64" else torch.float32
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(dt).cuda()
