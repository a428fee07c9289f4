"""Parity of gj_gramian_value_grad with the oracle (Eq. Gramian, RRCG:2-3)."""
import numpy as np
import pytest
import torch

from oracle import gramian as ogm
from tests.gpu_common import lib, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [1, 7, 1000, 300001])
def test_gramian_matches_oracle(prec, n):
    gj = lib()
    rng = np.random.default_rng(n)
    m1 = rng.uniform(0, 1, n)
    m2 = 0.1 * m1 + 0.01 * rng.standard_normal(n)
    S, l1, l2 = gj.gramian_value_grad(to_dev(m1, prec), to_dev(m2, prec))
    S_ref = ogm.gramian(m1, m2)
    r1, r2 = ogm.ascent_directions(m1, m2)
    scale = (m1 @ m1) * (m2 @ m2)
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert abs(S.item() - S_ref) <= tol * scale
    vtol = 1e-10 if prec == "fp64" else 1e-4
    if n > 1:
        assert rel(l1.cpu().numpy(), r1) <= vtol
        assert rel(l2.cpu().numpy(), r2) <= vtol


def test_gramian_collinear_is_zero():
    gj = lib()
    m1 = np.random.default_rng(1).uniform(0, 1, 5000)
    S, l1, l2 = gj.gramian_value_grad(to_dev(m1, "fp64"), to_dev(0.05 * m1, "fp64"))
    assert abs(S.item()) <= 1e-13 * (m1 @ m1) ** 2 * 0.05 ** 2


def test_pearson_on_the_device():
    """gj_pearson (the correlation measure of the lambda selection) against numpy's."""
    gj = lib()
    rng = np.random.default_rng(7)
    a, b = rng.standard_normal(50001), rng.standard_normal(50001)
    assert gj.pearson(a, b) == pytest.approx(np.corrcoef(a, b)[0, 1], abs=1e-12)
    assert gj.pearson(a, 3.0 * a - 2.0) == pytest.approx(1.0, abs=1e-12)
    assert gj.pearson(a, -0.5 * a + 7.0) == pytest.approx(-1.0, abs=1e-12)
    assert gj.pearson(a, np.full(a.size, 4.0)) == 0.0  # no spread: defined as 0
    assert gj.pearson(2 * a + 1, 5 * b - 3) == pytest.approx(gj.pearson(a, b), abs=1e-12)
    f = gj.pearson(torch.from_numpy(a).float().cuda(), torch.from_numpy(b).float().cuda())
    assert f == pytest.approx(np.corrcoef(a, b)[0, 1], abs=1e-6)
