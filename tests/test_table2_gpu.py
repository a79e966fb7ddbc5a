"""Table II (Sec. III-A) on the GPU: after 10^4 steps of the 1D advection,
the error of every split store ("# double" = number of coefficients
c_0 .. c_{q-1} kept in FP64, the rest in FP32) against the FP64 store, in the
function-space L2 norm, and its mass error, for order 2 (k = 1, # double 0,
1) and order 4 (k = 3, # double 0 .. 3), a smooth and an oscillatory initial
value (protocol: workloads.table2_protocol).

Each store runs twice: with its own arithmetic (rows of FP32 coefficients in
FP32) and with FP64 arithmetic (sl_set_arithmetic(SL_ARITH_FP64)).  The
FP64-arithmetic errors must agree with the oracle's FP64-arithmetic stores
(tests/test_table2_oracle.py) within a factor of 3 and, for # double >= 1,
lie within an order of magnitude of the printed values; the stores' own
FP32 arithmetic gives larger errors.  Mass: every store with c_0 in FP64
conserves it to about 1e-14 and the all-FP32 store does not.
"""
import numpy as np
import pytest

import oracle as O
import paper_1603_07008_gb300 as S
from paper_1603_07008_gb300 import workloads as W
from test_table2_oracle import fp64_arithmetic_table, golden_table2

pytestmark = pytest.mark.gpu

STORE = {0: "fp32", 1: "mix_fp32", 2: "mix_fp32_d2", 3: "mix_fp32_d3"}


def _run(P, storage, k, weights, params, arith):
    g = P.grid()
    with S.Context(g, k, storage) as ctx:
        ctx.project(P.nq, weights, params)
        ctx.set_arithmetic(arith)
        m0 = ctx.mass()
        for _ in range(P.steps):
            ctx.advect(0, -1, [P.shift])
        return ctx.get_coeffs(), abs(ctx.mass() - m0) / abs(m0)


@pytest.fixture(scope="module")
def oracle_table():
    return fp64_arithmetic_table(W.table2_protocol())


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("case", ["smooth", "oscillatory"])
def test_table2_orders_of_magnitude(order, case, oracle_table):
    P = W.table2_protocol()
    g = P.grid()
    k = order - 1
    paper = golden_table2()
    w, prm = P.initial[case]
    ref, mass64 = _run(P, "fp64", k, w, prm, "store")
    rows = {}
    for q in range(order):
        u32, m32 = _run(P, STORE[q], k, w, prm, "store")
        u64, m64 = _run(P, STORE[q], k, w, prm, "fp64")
        rows[q] = (O.l2_norm(u32 - ref, g, k), m32, O.l2_norm(u64 - ref, g, k), m64)
    print(f"\norder {order} {case}, N = {P.n}: all FP64 mass error {mass64:.2e}")
    print("#double  FP32 arith: error  mass   | FP64 arith: error  mass   | oracle error | paper error  mass")
    for q in sorted(rows, reverse=True):
        e32, m32, e64, m64 = rows[q]
        pe, pm = paper[(case, order, q)]
        print(f"{q:7d}  {e32:17.2e} {m32:.1e} | {e64:17.2e} {m64:.1e} | {oracle_table[(case, order, q)][0]:12.2e} |"
              f" {pe:.2e} {pm:.1e}")
    assert mass64 < 1e-13
    for q, (e32, m32, e64, m64) in rows.items():
        oe = oracle_table[(case, order, q)][0]
        assert oe / 3 <= e64 <= oe * 3, (q, e64, oe)
        if q >= 1:
            pe = paper[(case, order, q)][0]
            assert pe / 10 <= e64 <= pe * 10, (q, e64, pe)
            assert m32 < 1e-13 and m64 < 1e-13, (q, m32, m64)
            assert e64 < e32, (q, e64, e32)
        else:
            assert 1e-11 < m32 < 1e-4 and 1e-11 < m64 < 1e-4, (m32, m64)   # FP32 rounding of the mean
            assert e32 < 1e-3
    # every coefficient more in FP64 lowers the error, in both arithmetics
    for col in (0, 2):
        errs = [rows[q][col] for q in range(order)]
        assert all(b < a for a, b in zip(errs, errs[1:])), (col, errs)
