"""Orders of magnitude of the paper's Table II (Sec. III-A): after 10^4 steps
of the 1D advection, the error of the mixed store (c_0 in FP64, the other
coefficients in FP32: "# double = 1") against the FP64 store, in the
discrete L2 norm, and its mass error, for order 2 (k = 1) and order 4
(k = 3), a smooth and an oscillatory initial value.  The paper gives neither
N, the CFL number nor its initial values, so only orders of magnitude are
compared: errors of 1e-10 .. 1e-7 and mass errors of about 1e-14 there."""
import math

import numpy as np
import pytest

import paper_1603_07008_gb300 as S
from paper_1603_07008_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N = 256
STEPS = 10_000
SHIFT = 0.37
INITIAL = {
    # exp(-100 (x - 1/2)^2)
    "smooth": (np.array([1.0]), np.array([[[100.0, 0.5, 0.0, 0.0]]])),
    # 1 + cos(2 pi 8 x + 0.3): 32 cells per wavelength, mass 1
    "oscillatory": (np.array([1.0, 1.0]), np.array([[[0.0, 0.0, 0.0, 0.0]], [[0.0, 0.0, 2 * math.pi * 8, 0.3]]])),
}


def _run(storage, k, weights, params):
    g = W.Grid(n=(N,), lo=(0.0,), hi=(1.0,), pair=(-1,))
    with S.Context(g, k, storage) as ctx:
        ctx.project(8, weights, params)
        m0 = ctx.mass()
        for _ in range(STEPS):
            ctx.advect(0, -1, [SHIFT])
        return ctx.get_coeffs(), abs(ctx.mass() - m0) / abs(m0)


def _l2(u, k):
    w = np.array([2.0 / (2 * j + 1) for j in range(k + 1)]) / N / 2
    return math.sqrt(float(np.sum(u * u * w)))


@pytest.mark.parametrize("k", [1, 3])
@pytest.mark.parametrize("case", ["smooth", "oscillatory"])
def test_table2_orders_of_magnitude(k, case):
    w, prm = INITIAL[case]
    ref, mass64 = _run("fp64", k, w, prm)
    mix, mass32 = _run("mix_fp32", k, w, prm)
    err = _l2(mix - ref, k)
    print(f"order {k + 1} {case:11s}  error {err:.2e}  mass error (c_0 FP64) {mass32:.2e}  (all FP64) {mass64:.2e}")
    assert err < (1e-6 if case == "smooth" else 1e-5)
    assert mass32 < 1e-13
