"""The allocation-free Gramian entry point (gj_gramian_value_grad_noalloc).

Some callers cannot allocate device memory: hosts whose memory belongs to
another allocator, loops that forbid allocation.
This entry point serves them with a fixed scratch array inside the library.
The test calls it through the C ABI with buffers allocated beforehand and checks
two calls in a row (different sizes and data, so stale scratch from the first
call cannot pass for the second) against gj_gramian_value_grad, within the
tolerances of the other Gramian tests.  It runs last so that a failure here
leaves the rest of the suite already run.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

from tests.gpu_common import lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_allocating_entry_point_twice(prec):
    gj = lib()
    from paper_2112_15562_gb300 import _lib

    L = _lib.load()
    dt = torch.float64 if prec == "fp64" else torch.float32
    code = _lib.GJ_FP64 if prec == "fp64" else _lib.GJ_FP32_MIXED
    stol = 1e-12 if prec == "fp64" else 2e-6
    vtol = 1e-10 if prec == "fp64" else 1e-4
    rng = np.random.default_rng(42)
    for n in (300001, 5000):
        m1 = torch.from_numpy(rng.uniform(0, 1, n)).to(dt).cuda()
        m2 = (0.1 * m1 + 0.01 * torch.from_numpy(rng.standard_normal(n)).to(dt).cuda()).contiguous()
        S_ref, l1_ref, l2_ref = gj.gramian_value_grad(m1, m2)
        # outputs allocated before the call and poisoned
        S = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        l1 = torch.full_like(m1, float("nan"))
        l2 = torch.full_like(m2, float("nan"))
        stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = L.gj_gramian_value_grad_noalloc(n, code, ct.c_void_p(m1.data_ptr()), ct.c_void_p(m2.data_ptr()),
                                             ct.c_void_p(S.data_ptr()), ct.c_void_p(l1.data_ptr()),
                                             ct.c_void_p(l2.data_ptr()), stream)
        assert rc == 0, L.gj_last_error()
        torch.cuda.synchronize()
        scale = float((m1.double() @ m1.double()) * (m2.double() @ m2.double()))
        assert abs(S.item() - S_ref.item()) <= stol * scale
        for a, b in ((l1, l1_ref), (l2, l2_ref)):
            a64, b64 = a.double(), b.double()
            assert float(torch.linalg.norm(a64 - b64) / torch.linalg.norm(b64)) <= vtol


def test_noalloc_rejects_sizes_beyond_its_limit():
    lib()
    from paper_2112_15562_gb300 import _lib

    L = _lib.load()
    x = torch.zeros(4, device="cuda")
    p = ct.c_void_p(x.data_ptr())
    rc = L.gj_gramian_value_grad_noalloc(16777217, _lib.GJ_FP32_MIXED, p, p, p, None, None, None)
    assert rc == -1
    assert b"16777216" in L.gj_last_error()
