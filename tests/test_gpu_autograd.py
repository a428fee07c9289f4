"""Differentiable forms (torch.autograd.Function) of G, G^T and the Gramian:
finite-difference gradchecks in FP64 at 32x32x8 and gradients against the dense
FP64 oracle (Eq. d=gm, Eq. Gramian, RRCG:2-3)."""
import numpy as np
import pytest
import torch

import synth
from oracle import gramian as ogm
from oracle import operator as oop
from tests.gpu_common import lib, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c5_small():
    gj = lib()
    g = synth.uniform_grid(32, 32, 32, 32, 8, 50.0)
    mag = synth.Mag(50000.0, 60.0, 10.0)
    ops = {f: gj.bttb_setup(g, f, mag if f == "magnetic" else None, precision="fp64")
           for f in ("gravity", "magnetic")}
    A = {"gravity": oop.dense_matrix(g, oop.GRAVITY), "magnetic": oop.dense_matrix(g, oop.MAGNETIC, mag)}
    return gj, g, ops, A


@pytest.mark.parametrize("field", ["gravity", "magnetic"])
def test_gradcheck_forward_and_adjoint(c5_small, field):
    gj, g, ops, A = c5_small
    op = ops[field]
    rng = np.random.default_rng(3)
    m = to_dev(rng.standard_normal(g.n), "fp64").requires_grad_(True)
    r = to_dev(rng.standard_normal(g.s), "fp64").requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: gj.G(op, x), (m,), fast_mode=True, eps=1e-6, atol=1e-7, rtol=1e-6)
    assert torch.autograd.gradcheck(lambda x: gj.GT(op, x), (r,), fast_mode=True, eps=1e-6, atol=1e-7, rtol=1e-6)


@pytest.mark.parametrize("field", ["gravity", "magnetic"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_misfit_gradient_matches_dense_oracle(c5_small, field, prec):
    gj, g, ops_fp64, A = c5_small
    op = ops_fp64[field] if prec == "fp64" else gj.bttb_setup(
        g, field, synth.Mag(50000.0, 60.0, 10.0) if field == "magnetic" else None, precision="fp32")
    rng = np.random.default_rng(4)
    m0 = rng.uniform(0, 1, g.n)
    d = rng.standard_normal(g.s)
    m = to_dev(m0, prec).requires_grad_(True)
    loss = 0.5 * torch.sum((gj.G(op, m) - to_dev(d, prec)) ** 2)
    loss.backward()
    ref = A[field].T @ (A[field] @ m0 - d)
    tol = 1e-10 if prec == "fp64" else 1e-4
    assert rel(m.grad.cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gramian_autograd(prec):
    gj = lib()
    rng = np.random.default_rng(5)
    n = 4097
    a, b = rng.uniform(0, 1, n), rng.uniform(0, 0.1, n)
    m1 = to_dev(a, prec).requires_grad_(True)
    m2 = to_dev(b, prec).requires_grad_(True)
    S = gj.gramian(m1, m2)
    assert S.dtype == torch.float64
    S.backward()
    l1, l2 = ogm.ascent_directions(a, b)
    tol = 1e-10 if prec == "fp64" else 1e-4
    assert rel(m1.grad.cpu().numpy(), 2 * l1) <= tol
    assert rel(m2.grad.cpu().numpy(), 2 * l2) <= tol
    if prec == "fp64":
        x1 = to_dev(rng.standard_normal(64), "fp64").requires_grad_(True)
        x2 = to_dev(rng.standard_normal(64), "fp64").requires_grad_(True)
        assert torch.autograd.gradcheck(gj.gramian, (x1, x2), eps=1e-6, atol=1e-6, rtol=1e-6)


@pytest.mark.parametrize("prec,npad", [("fp32", (512, 512)), ("fp32", (1024, 1024)), ("fp64", (0, 0))],
                         ids=["fast512", "fast1024", "general-fp64"])
def test_products_replay_in_a_cuda_graph(prec, npad):
    """A forward + backward step (G m and its adjoint through autograd) captured once
    with torch.cuda.graph and replayed gives the eager step's gradients: the
    products launch on the caller's stream with no host synchronisation."""
    gj = lib()
    g = synth.uniform_grid(32, 32, 32, 32, 8, 50.0)
    mag = synth.Mag(50000.0, 60.0, 10.0)
    ops = [gj.bttb_setup(g, "gravity", precision=prec, npad=npad),
           gj.bttb_setup(g, "magnetic", mag, precision=prec, npad=npad)]
    dt = torch.float64 if prec == "fp64" else torch.float32
    gen = torch.Generator(device="cuda").manual_seed(11)
    m = [torch.rand(g.n, device="cuda", dtype=dt, generator=gen, requires_grad=True) for _ in range(2)]
    gd = [torch.randn(g.s, device="cuda", dtype=dt, generator=gen) for _ in range(2)]

    def step():
        for t in m:
            t.grad = None
        for i in range(2):
            gj.G(ops[i], m[i]).backward(gd[i])

    step()
    ref = [t.grad.clone() for t in m]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for i in range(2):
        assert rel(m[i].grad.cpu().numpy(), ref[i].cpu().numpy()) <= 1e-12
    del graph
    for o in ops:
        o.close()
