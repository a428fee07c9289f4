"""Failure paths on the GPU, made on the host (no fault, trap or hang): a NaN in
the observed data must stop the solve with GJ_ERR_NONFINITE (the non-finite check
of the chi^2 scalars, Eq. chi2) on both kernel families; the bounded mbarrier wait
must give up on a barrier that nothing completes and report GJ_ERR_TIMEOUT, with
the context still usable; and a healthy operator reports GJ_OK from gj_op_status."""
import ctypes as ct
import time

import numpy as np
import pytest
import torch

import synth
from oracle import operator as oop
from oracle import weights as owt
from tests.gpu_common import lib, to_dev

pytestmark = pytest.mark.gpu


def small_inputs():
    w = synth.small_joint()
    g = w.grid
    A = [oop.dense_matrix(g, oop.GRAVITY), oop.dense_matrix(g, oop.MAGNETIC, w.mag)]
    obs = [owt.noisy_data(A[i] @ w.m_true[i], 0.01, 0.01, w.noise[i]) for i in range(2)]
    wdep = [owt.depth_weights(g.z_edges, 2.0), owt.depth_weights(g.z_edges, 3.0)]
    return w, g, [o[0] for o in obs], [o[1] for o in obs], wdep


@pytest.mark.parametrize("path", [("fp64", (0, 0)), ("fp32", (512, 512))])
def test_nan_in_data_stops_with_nonfinite(path):
    gj = lib()
    from paper_2112_15562_gb300 import _lib

    prec, npad = path
    w, g, dob, sig, wdep = small_inputs()
    bad = [d.copy() for d in dob]
    bad[1][37] = np.nan
    ops = [gj.bttb_setup(g, "gravity", precision=prec, npad=npad),
           gj.bttb_setup(g, "magnetic", w.mag, precision=prec, npad=npad)]
    assert ops[0].info.fast_path == (1 if prec == "fp32" else 0)
    m = [to_dev(np.zeros(g.n), prec) for _ in range(2)]
    P = gj.solver_params(p=(1, 1), lam=(50.0, 1500.0), kmax=10, stop_on_chi2=False)
    with pytest.raises(gj.GJError) as ei:
        gj.rrcg_joint_solve(ops, P, [to_dev(x, prec) for x in bad], [to_dev(x, prec) for x in sig],
                            [to_dev(x, prec) for x in wdep], m)
    assert ei.value.status == _lib.STATUS_CODE["GJ_ERR_NONFINITE"]
    # the stepwise form reports it in rep.status and stops before any update
    sv = gj.Solver(ops, P, [to_dev(x, prec) for x in bad], [to_dev(x, prec) for x in sig],
                   [to_dev(x, prec) for x in wdep], m)
    sv.iterate(3)
    rep = sv.report()
    assert rep["status"] == _lib.STATUS_CODE["GJ_ERR_NONFINITE"] and rep["iterations"] == 0
    assert sv.done()
    sv.close()
    # the same operators still serve a clean solve
    m = [to_dev(np.zeros(g.n), prec) for _ in range(2)]
    rep = gj.rrcg_joint_solve(ops, P, [to_dev(x, prec) for x in dob], [to_dev(x, prec) for x in sig],
                              [to_dev(x, prec) for x in wdep], m)
    assert rep["status"] == 0 and rep["iterations"] == 10
    assert all(np.isfinite(t.cpu().numpy()).all() for t in m)


def test_bounded_wait_gives_up_and_reports_timeout():
    lib()
    from paper_2112_15562_gb300 import _lib

    L = _lib.load()
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    for limit_ns in (0, 20_000_000):
        t0 = time.perf_counter()
        rc = L.gj_selftest_bounded_wait(limit_ns, stream)
        dt = time.perf_counter() - t0
        assert rc == _lib.STATUS_CODE["GJ_ERR_TIMEOUT"], L.gj_last_error()
        assert dt >= limit_ns * 1e-9 and dt < 5.0
    # the context is still usable
    x = torch.arange(1000, device="cuda", dtype=torch.float64)
    assert float(x.sum()) == 499500.0
    assert L.gj_selftest_bounded_wait(-1, stream) == _lib.STATUS_CODE["GJ_ERR_ARG"]


def test_op_status_of_a_healthy_fast_operator():
    gj = lib()
    from paper_2112_15562_gb300 import _lib

    L = _lib.load()
    w, g, dob, sig, wdep = small_inputs()
    op = gj.bttb_setup(g, "magnetic", w.mag, precision="fp32", npad=(512, 512))
    assert op.info.fast_path == 1
    d = op.forward(to_dev(np.ones(g.n), "fp32"))
    op.adjoint(d)
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.gj_op_status(op.handle, 0, stream) == 0
    assert L.gj_op_status(op.handle, 1, stream) == 0
    slow = gj.bttb_setup(g, "gravity", precision="fp64")
    assert L.gj_op_status(slow.handle, 1, stream) == 0


def test_device_report_equals_host_report():
    """gj_rrcg_report_device writes the report into device memory without a host round
    trip; it must equal gj_rrcg_report_get."""
    gj = lib()
    from paper_2112_15562_gb300 import _lib

    L = _lib.load()
    w, g, dob, sig, wdep = small_inputs()
    ops = [gj.bttb_setup(g, "gravity", precision="fp64"), gj.bttb_setup(g, "magnetic", w.mag, precision="fp64")]
    m = [to_dev(np.zeros(g.n), "fp64") for _ in range(2)]
    sv = gj.Solver(ops, gj.solver_params(p=(1, 1), lam=(50.0, 1500.0), kmax=6, stop_on_chi2=False),
                   [to_dev(x, "fp64") for x in dob], [to_dev(x, "fp64") for x in sig],
                   [to_dev(x, "fp64") for x in wdep], m)
    sv.iterate(4)
    buf = torch.zeros(ct.sizeof(_lib.RRCGReport), dtype=torch.uint8, device="cuda")
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.gj_rrcg_report_device(sv._h, ct.c_void_p(buf.data_ptr()), stream) == 0
    host = bytes(buf.cpu().numpy().tobytes())
    dev = _lib.RRCGReport.from_buffer_copy(host)
    rep = sv.report()
    assert dev.iterations == rep["iterations"] == 4 and dev.status == rep["status"] == 0
    assert list(dev.phi) == rep["phi"] and dev.S_G == rep["S_G"] and list(dev.alpha) == rep["alpha"]
    sv.close()
