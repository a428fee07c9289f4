"""Host-side logic of the binding, on the CPU: the autotuner's padded-size
candidates and the solver-option mapping.  None of these calls the GPU."""
import numpy as np
import pytest

import synth
from paper_2112_15562_gb300 import _lib as L
from paper_2112_15562_gb300 import autotune
from paper_2112_15562_gb300.api import solver_params


def _smooth(n, primes=(2, 3, 5, 7)):
    for p in primes:
        while n % p == 0:
            n //= p
    return n == 1


@pytest.mark.parametrize("minimum", [1, 7, 17, 100, 255, 511, 1023, 2040])
def test_smooth_sizes_are_the_next_7_smooth_integers(minimum):
    got = autotune.smooth_sizes(minimum, 3)
    want = [n for n in range(minimum, 2049) if _smooth(n)][:3]
    assert got == want


def test_candidates_cover_the_bccb_size_and_the_512_kernels():
    g = synth.uniform_grid(256, 256, 256, 256, 40, 100.0)
    c32 = autotune.candidates(g, "fp32")
    assert c32[:3] == [(512, 512), (525, 525), (540, 540)]
    assert (512, 512) in c32
    g2 = synth.uniform_grid(200, 130, 200, 130, 8, 50.0)  # s + n - 1 = 399 x 259
    c = autotune.candidates(g2, "fp64")
    assert all(ny >= 259 and nx >= 399 and _smooth(ny) and _smooth(nx) for ny, nx in c)
    assert (512, 512) not in c  # the 512 kernels are FP32 only
    assert (512, 512) in autotune.candidates(g2, "fp32")
    g3 = synth.uniform_grid(300, 300, 300, 300, 4, 50.0)  # beyond the 512 kernels' 256 per side
    assert (512, 512) not in autotune.candidates(g3, "fp32")


def test_solver_params_option_mapping():
    P = solver_params(p=(1, 2), lam=(2.0, 100.0), scalars="per_field", anchor="previous", gramian_space="weighted")
    assert list(P.p) == [1, 2] and list(P.lambda_) == [2.0, 100.0]
    assert P.scalars == L.GJ_SCALARS_PER_FIELD and P.anchor == 1 and P.gramian_space == 1
    Q = solver_params()
    assert Q.scalars == L.GJ_SCALARS_AUTO and Q.anchor == 0 and Q.gramian_space == 0 and Q.stop_on_chi2 == 1
    with pytest.raises(KeyError):
        solver_params(scalars="both")
