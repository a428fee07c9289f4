"""Parity of the fused FP32 joint solve on the 512 x 512 (and 256 x 512) kernels at the benchmark's
layer count (Eq. RRCG:1-8, Secs. 2.5, 2.6, 2.8): both fields interleaved in the
column passes with 40-layer columns split across warps, and the team row passes.

* 32x32 stations over 32x32x40 cells, 25 iterations, against the oracle with the
  dense matrices (assembled from the prism tables);
* the benchmark workload itself, 256x256 stations over 256x256x40 cells of 100 m,
  8 iterations, against the oracle with its FFT evaluation of the same products
  (oracle.operator.BCCB, pinned against the dense product on small grids).

Tolerances (the FP32 form's, set for FP32 vectors, spectra and FFTs with FP64
scalars): Phi of every iteration within 1e-4 relative, the models within 1e-3
relative L2.  The measured errors are printed (run with -s)."""
import numpy as np
import pytest

import synth
from oracle import operator as oop
from oracle import weights as owt
from oracle.rrcg import RRCGParams, rrcg_joint
from tests.gpu_common import lib, rel, to_dev

pytestmark = pytest.mark.gpu

KW = dict(p=(1, 1), alpha1=(2e4, 2e4), q=(0.95, 0.95), alpha_min=(5.0, 20.0), lam=(2.0, 100.0), lo=(0.0, 0.0),
          hi=(1.0, 0.1), stop_on_chi2=False)


def oracle_solve(fwd, adj, dob, sig, wdep, g, kmax):
    P = RRCGParams(kmax=kmax, **KW)
    return rrcg_joint(fwd, adj, dob, sig, [np.zeros(g.n)] * 2, [np.repeat(wdep[i], g.nx * g.ny) for i in range(2)], P)


def gpu_solve(gj, w, g, dob, sig, wdep, kmax, npad=(512, 512)):
    ops = [gj.bttb_setup(g, "gravity", precision="fp32", npad=npad),
           gj.bttb_setup(g, "magnetic", w.mag, precision="fp32", npad=npad)]
    kind = 2 if npad[0] == 1024 else 1
    assert ops[0].info.fast_path == kind and ops[1].info.fast_path == kind
    m = [to_dev(np.zeros(g.n), "fp32") for _ in range(2)]
    rep = gj.rrcg_joint_solve(ops, gj.solver_params(kmax=kmax, **KW), [to_dev(x, "fp32") for x in dob],
                              [to_dev(x, "fp32") for x in sig], [to_dev(x, "fp32") for x in wdep], m, history=True)
    return [t.cpu().numpy().astype(np.float64) for t in m], rep


def check(name, ref, m, rep, kmax):
    assert rep["iterations"] == ref.iterations == kmax
    phi_err = max(abs(rep["history"][k]["phi"][i] - ref.history[k]["phi"][i]) / ref.history[k]["phi"][i]
                  for k in range(kmax + 1) for i in range(2))
    m_err = [rel(m[i], ref.m[i]) for i in range(2)]
    print(f"\n{name}: max relative Phi error over {kmax + 1} iterations {phi_err:.2e}; "
          f"model relative L2 gravity {m_err[0]:.2e}, magnetic {m_err[1]:.2e}")
    assert phi_err <= 1e-4
    for i in range(2):
        assert m_err[i] <= 1e-3, (i, m_err[i])
        # the bounds as the FP32 path holds them (0.1 rounds up to 0.10000000149)
        assert m[i].min() >= np.float32(KW["lo"][i]) and m[i].max() <= np.float32(KW["hi"][i])


@pytest.mark.parametrize("npad", [(512, 512), (256, 512), (1024, 64), (1024, 1024)])
def test_fast_joint_solve_40_layers_against_dense_oracle(npad):
    gj = lib()
    w = synth.joint_256(n=32)
    g = w.grid
    A = [oop.dense_from_table(oop.kernel_table(g, oop.GRAVITY), g),
         oop.dense_from_table(oop.kernel_table(g, oop.MAGNETIC, w.mag), g)]
    obs = [owt.noisy_data(A[i] @ w.m_true[i], 0.01, 0.01, w.noise[i]) for i in range(2)]
    dob, sig = [o[0] for o in obs], [o[1] for o in obs]
    wdep = [owt.depth_weights(g.z_edges, 2.0), owt.depth_weights(g.z_edges, 3.0)]
    kmax = 25
    ref = oracle_solve([lambda x, i=i: A[i] @ x for i in range(2)], [lambda y, i=i: A[i].T @ y for i in range(2)],
                       dob, sig, wdep, g, kmax)
    m, rep = gpu_solve(gj, w, g, dob, sig, wdep, kmax, npad)
    check(f"32x32x40 padded {npad[0]}x{npad[1]}", ref, m, rep, kmax)


def test_fast_joint_solve_benchmark_workload_against_fft_oracle():
    gj = lib()
    w = synth.joint_256()
    g = w.grid
    B = [oop.BCCB(oop.kernel_table(g, oop.GRAVITY), g, 512, 512),
         oop.BCCB(oop.kernel_table(g, oop.MAGNETIC, w.mag), g, 512, 512)]
    obs = [owt.noisy_data(B[i].forward(w.m_true[i]), 0.01, 0.01, w.noise[i]) for i in range(2)]
    dob, sig = [o[0] for o in obs], [o[1] for o in obs]
    wdep = [owt.depth_weights(g.z_edges, 2.0), owt.depth_weights(g.z_edges, 3.0)]
    kmax = 8
    ref = oracle_solve([B[0].forward, B[1].forward], [B[0].adjoint, B[1].adjoint], dob, sig, wdep, g, kmax)
    m, rep = gpu_solve(gj, w, g, dob, sig, wdep, kmax)
    check("256x256x40", ref, m, rep, kmax)


def test_fast256_joint_solve_128x128x40_against_fft_oracle():
    """The largest grid of the 256-row kernels (128 x 128 stations over 128 x 128 x 40
    cells of 100 m, padded 256 x 512), 8 iterations against the FFT oracle at the
    same padded size."""
    gj = lib()
    w = synth.joint_256(n=128)
    g = w.grid
    B = [oop.BCCB(oop.kernel_table(g, oop.GRAVITY), g, 256, 512),
         oop.BCCB(oop.kernel_table(g, oop.MAGNETIC, w.mag), g, 256, 512)]
    obs = [owt.noisy_data(B[i].forward(w.m_true[i]), 0.01, 0.01, w.noise[i]) for i in range(2)]
    dob, sig = [o[0] for o in obs], [o[1] for o in obs]
    wdep = [owt.depth_weights(g.z_edges, 2.0), owt.depth_weights(g.z_edges, 3.0)]
    kmax = 8
    ref = oracle_solve([B[0].forward, B[1].forward], [B[0].adjoint, B[1].adjoint], dob, sig, wdep, g, kmax)
    m, rep = gpu_solve(gj, w, g, dob, sig, wdep, kmax, (256, 512))
    check("128x128x40 padded 256x512", ref, m, rep, kmax)
