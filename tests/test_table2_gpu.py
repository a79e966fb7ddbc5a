"""Orders of magnitude of the paper's Table II (Sec. III-A): after 10^4 steps
of the 1D advection, the error of every split store ("# double" = number of
coefficients c_0 .. c_{q-1} kept in FP64, the rest in FP32) against the FP64
store, in the discrete L2 norm, and its mass error, for order 2 (k = 1,
# double 0, 1) and order 4 (k = 3, # double 0 .. 3), a smooth and an
oscillatory initial value.  The paper gives neither N, the CFL number nor
its initial values, so only what its table shows is checked: the stores with
c_0 in FP64 conserve mass to about 1e-14 and the all-FP32 store does not
(about 1e-6 there), and every further coefficient in FP64 lowers the error.
"""
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


STORES = {1: ["fp32", "mix_fp32"], 3: ["fp32", "mix_fp32", "mix_fp32_d2", "mix_fp32_d3"]}
NDOUBLE = {"fp32": 0, "mix_fp32": 1, "mix_fp32_d2": 2, "mix_fp32_d3": 3}


@pytest.mark.parametrize("k", [1, 3])
@pytest.mark.parametrize("case", ["smooth", "oscillatory"])
def test_table2_orders_of_magnitude(k, case):
    w, prm = INITIAL[case]
    ref, mass64 = _run("fp64", k, w, prm)
    rows = {}
    for st in STORES[k]:
        u, me = _run(st, k, w, prm)
        rows[NDOUBLE[st]] = (_l2(u - ref, k), me)
    print(f"order {k + 1} {case:11s} all FP64: mass error {mass64:.2e}")
    for q in sorted(rows, reverse=True):
        print(f"order {k + 1} {case:11s} # double {q}  error {rows[q][0]:.2e}  mass error {rows[q][1]:.2e}")
    assert mass64 < 1e-13
    for q, (err, me) in rows.items():
        if q >= 1:
            assert me < 1e-13, q
        else:
            assert 1e-11 < me < 1e-4, me   # FP32 rounding of the mean (Table II: ~1e-6)
            assert err < 1e-3
    # every coefficient more in FP64 lowers the error
    qs = sorted(rows)
    for a, b in zip(qs, qs[1:]):
        assert rows[b][0] < rows[a][0], (a, b, rows)
    assert rows[1][0] < (1e-6 if case == "smooth" else 1e-5)
