"""Table II (Sec. III-A) through the oracle, with FP64 arithmetic and FP32
storage: every sweep is the FP64 update rule, and the coefficients a store of
"# double" = q keeps in FP32 are rounded after every sweep
(oracle.stored_sweeps).  Sec. III-A states which coefficients are stored in
double precision, not the precision of the arithmetic; this test decides
between the two readings by the printed error column.

Protocol (workloads.table2_protocol): 10^4 steps of 1D periodic advection,
orders 2 and 4, the smooth and the oscillatory initial value, the error
against the FP64 scheme in the function-space L2 norm.  The paper gives
neither N nor the CFL number; with N = 512 and 0.37 cells per step every row
with c_0 in FP64 lands within an order of magnitude of the printed value
(tests/golden/table2.txt).  The all-FP32 rows are printed beside their
values: the paper's single precision implementation is not specified further.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1603_07008_gb300 import workloads as W


def golden_table2():
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "table2.txt")):
        if line.strip() and not line.startswith("#"):
            prof, order, q, err, merr = line.split()
            rows[(prof, int(order), int(q))] = (float(err), float(merr))
    return rows


def fp64_arithmetic_table(P):
    """{(profile, order, q): (error, mass error)} of the oracle's stores."""
    g = P.grid()
    out = {}
    for prof, (w, prm) in P.initial.items():
        for order in (2, 4):
            k = order - 1
            u0 = O.project(g, k, P.nq, w, prm)
            ref = u0
            for _ in range(P.steps):
                ref = O.sweep(ref, g.n, k, 0, -1, [P.shift])
            sweeps = [(0, -1, [P.shift])] * P.steps
            for q in range(order):
                held = O.round_storage(u0, k, 1, q)
                u = O.stored_sweeps(u0, g.n, k, q, sweeps)
                m0 = O.mass(held, g, k)
                out[(prof, order, q)] = (O.l2_norm(u - ref, g, k), abs(O.mass(u, g, k) - m0) / abs(m0))
    return out


@pytest.mark.slow
def test_table2_error_column_with_fp64_arithmetic():
    P = W.table2_protocol()
    paper = golden_table2()
    got = fp64_arithmetic_table(P)
    assert set(got) == set(paper)
    print(f"\nTable II, FP64 arithmetic + FP32 storage (oracle), N = {P.n}, shift {P.shift}, {P.steps} steps")
    print("profile      order #double   error (paper)          mass error (paper)")
    for key in sorted(paper, key=lambda t: (t[0], t[1], -t[2])):
        e, m = got[key]
        pe, pm = paper[key]
        print(f"{key[0]:12s} {key[1]:5d} {key[2]:7d}   {e:.2e} ({pe:.2e})    {m:.2e} ({pm:.2e})")
    for (prof, order, q), (e, m) in got.items():
        pe, _ = paper[(prof, order, q)]
        if q >= 1:
            # the printed orders of magnitude
            assert pe / 10 <= e <= pe * 10, (prof, order, q, e, pe)
            # mass error: the oracle's own FP64 drift (its A_00 + B_00 is 1 to
            # an ulp), not the store's
            assert m < 1e-11, (prof, order, q, m)
        else:
            assert 1e-9 < m < 1e-4, (prof, order, q, m)
    # every coefficient more in FP64 lowers the error
    for prof in P.initial:
        for order in (2, 4):
            errs = [got[(prof, order, q)][0] for q in range(order)]
            assert all(b < a for a, b in zip(errs, errs[1:])), (prof, order, errs)
