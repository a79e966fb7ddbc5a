"""FP64 arithmetic with FP32 storage (sl_set_arithmetic(SL_ARITH_FP64)) for
the stores of "# double" = 0 .. 3 (Sec. III-A), against the oracle that
applies the FP64 update rule and rounds the FP32 coefficients of the store
after every sweep (oracle.stored_sweeps).

Tolerances:
  * one sweep from a stored state: FP64 coefficients within 1e-13 of the
    oracle's (relative to the largest value; the GPU takes the conservation
    form of the mean row, the oracle the plain sums); every FP32 coefficient
    is the FP32 rounding of the oracle's FP64 value or one FP32 ulp from it
    (the two FP64 values differ by rounding order, so a value that close to a
    rounding boundary may round the other way), and nearly all are equal;
  * split steps: relative function-space L2 <= 1e-9 against the oracle with
    the same rounding after every sweep;
  * mass drift <= 1e-13 after 1000 steps for # double >= 1.
"""
import numpy as np
import pytest

import oracle as O
import paper_1603_07008_gb300 as S
from paper_1603_07008_gb300 import workloads as W

pytestmark = pytest.mark.gpu

Q = {"fp32": 0, "mix_fp32": 1, "mix_fp32_d2": 2, "mix_fp32_d3": 3}
CASES = [("mix_fp32", 0), ("mix_fp32", 1), ("mix_fp32", 2), ("mix_fp32", 3), ("fp32", 1), ("fp32", 2),
         ("fp32", 3), ("mix_fp32_d2", 2), ("mix_fp32_d2", 3), ("mix_fp32_d3", 3)]


def _grid(n, pair=None):
    d = len(n)
    return W.Grid(n=tuple(n), lo=(0.0,) * d, hi=(1.0,) * d, pair=tuple(pair or (-1,) * d))


def _check_stored(got, ref, k, d, q):
    """got: the GPU's state after a sweep; ref: the oracle's FP64 sweep of the
    same stored input (before rounding)."""
    mask = O.fp64_coefficients(k, d, q)
    scale = np.max(np.abs(ref))
    if mask.any():
        assert np.max(np.abs(got[:, mask] - ref[:, mask])) <= 1e-13 * scale
    r = ref[:, ~mask]
    r32 = r.astype(np.float32)
    g = got[:, ~mask]
    assert np.array_equal(g, g.astype(np.float32).astype(np.float64))   # what an FP32 plane holds
    ulp = np.spacing(np.abs(r32)).astype(np.float64)
    diff = np.abs(g - r32.astype(np.float64))
    assert np.all(diff <= ulp), float(np.max(diff / np.maximum(ulp, 1e-300)))
    assert np.count_nonzero(diff) <= 2 + r.size // 1000


@pytest.mark.parametrize("storage,k", CASES)
@pytest.mark.parametrize("n", [(37,), (9, 7), (5, 4, 3), (3, 4, 2, 3)])
def test_single_sweeps_match_the_oracle_rounded_to_the_store(storage, k, n):
    if (k + 1) ** len(n) > 512:
        pytest.skip("coefficient count covered by smaller shapes")
    q, d = Q[storage], len(n)
    rng = np.random.default_rng(11)
    u = O.round_storage(W.random_coefficients(int(np.prod(n)), k, d, 12), k, d, q)
    with S.Context(_grid(n), k, storage) as ctx:
        ctx.set_arithmetic("fp64")
        for dim in range(d):
            for sd in [-1] + [m for m in range(d) if m != dim]:
                cnt = 1 if sd < 0 else n[sd]
                s = rng.uniform(-2.5 * n[dim], 2.5 * n[dim], size=cnt)
                ctx.set_coeffs(u)
                ctx.advect(dim, sd, s)
                _check_stored(ctx.get_coeffs(), O.sweep(u, n, k, dim, sd, s), k, d, q)


@pytest.mark.parametrize("storage,k", [("mix_fp32", 2), ("fp32", 2), ("mix_fp32_d2", 2), ("mix_fp32_d3", 3)])
def test_strang_steps_match_the_stored_oracle(storage, k):
    q = Q[storage]
    p = W.config2(n=24, steps=10, storage=storage)
    sched = O.schedule(p.grid, "strang", p.dt, p.field_list())
    with S.Context(p.grid, k, storage) as ctx:
        ctx.project(p.nq, p.weights, p.params)
        u0 = ctx.get_coeffs()
        ctx.set_fields(p.field_list())
        ctx.set_arithmetic("fp64")
        ctx.step("strang", p.dt, p.steps)
        got = ctx.get_coeffs()
    ref = O.stored_sweeps(u0, p.grid.n, k, q, sched * p.steps)
    assert O.rel_l2(got, ref, k, 2) <= 1e-9


def test_fp64_arithmetic_is_closer_to_the_fp64_store():
    """After 50 Strang steps of the 2D workload the FP64-arithmetic mixed
    store is closer to the FP64 store than the FP32-arithmetic one."""
    p = W.config2(n=32, steps=50)
    out = {}
    for storage, arith in [("fp64", "store"), ("mix_fp32", "store"), ("mix_fp32", "fp64")]:
        with S.Context(p.grid, p.k, storage) as ctx:
            ctx.project(p.nq, p.weights, p.params)
            ctx.set_fields(p.field_list())
            ctx.set_arithmetic(arith)
            ctx.step("strang", p.dt, p.steps)
            out[(storage, arith)] = ctx.get_coeffs()
    ref = out[("fp64", "store")]
    e32 = O.rel_l2(out[("mix_fp32", "store")], ref, p.k, 2)
    e64 = O.rel_l2(out[("mix_fp32", "fp64")], ref, p.k, 2)
    assert e64 < e32 / 3, (e64, e32)
    assert e64 < 1e-7


@pytest.mark.parametrize("storage,k", [("mix_fp32", 1), ("mix_fp32", 3), ("mix_fp32_d2", 3), ("mix_fp32_d3", 3)])
def test_mass_is_conserved_over_1000_steps(storage, k):
    g = _grid((256,))
    with S.Context(g, k, storage) as ctx:
        ctx.set_coeffs(W.random_coefficients(256, k, 1, 13) + np.eye(1, (k + 1), 0))
        ctx.set_arithmetic("fp64")
        m0 = ctx.mass()
        for _ in range(1000):
            ctx.advect(0, -1, [0.37])
        assert abs(ctx.mass() - m0) / abs(m0) <= 1e-13


def test_graph_replay_and_switching_back():
    """A graph captured with FP64 arithmetic replays the same sweeps; the
    store's own arithmetic comes back with SL_ARITH_STORE."""
    import torch
    p = W.config2(n=16, steps=3)
    st = torch.cuda.Stream()
    res = {}
    for mode in ["eager", "graph", "back"]:
        with S.Context(p.grid, p.k, "mix_fp32", stream=st) as ctx:
            ctx.project(p.nq, p.weights, p.params)
            ctx.set_fields(p.field_list())
            ctx.set_arithmetic("fp64")
            if mode == "graph":
                ctx.graph_capture("strang", p.dt, p.steps)
                ctx.graph_launch()
            else:
                if mode == "back":
                    ctx.set_arithmetic("store")
                ctx.step("strang", p.dt, p.steps)
            res[mode] = ctx.get_coeffs()
    with S.Context(p.grid, p.k, "mix_fp32") as ctx:
        ctx.project(p.nq, p.weights, p.params)
        ctx.set_fields(p.field_list())
        ctx.step("strang", p.dt, p.steps)
        plain = ctx.get_coeffs()
    assert np.array_equal(res["eager"], res["graph"])
    assert np.array_equal(res["back"], plain)
    assert not np.array_equal(res["eager"], plain)


def test_arithmetic_argument_errors():
    g = _grid((8, 8), (1, -1))
    with S.Context(g, 1, "mix_bf16") as ctx:
        with pytest.raises(S.SlError) as e:
            ctx.set_arithmetic("fp64")
        assert e.value.status == S.SL_ENOTSUP
        ctx.set_arithmetic("store")
    with S.Context(g, 1, "fp64") as ctx:
        ctx.set_arithmetic("fp64")   # already FP64: accepted, no change
        ctx.set_arithmetic("store")
    with S.Context(g, 1, "mix_fp32") as ctx:
        with pytest.raises(S.SlError) as e:
            ctx.set_arithmetic(2)
        assert e.value.status == S.SL_EINVAL
        ctx.set_nodal_velocity(True)
        with pytest.raises(S.SlError) as e:
            ctx.set_arithmetic("fp64")
        assert e.value.status == S.SL_ENOTSUP
        ctx.set_nodal_velocity(False)
        ctx.set_arithmetic("fp64")
        for call in (lambda: ctx.set_nodal_velocity(True), lambda: ctx.advect_nodal(0, 0.1)):
            with pytest.raises(S.SlError) as e:
                call()
            assert e.value.status == S.SL_ENOTSUP
    with pytest.raises(Exception):
        S.sl_set_arithmetic(None, 1)


def test_fp64_rate_selftest():
    """The measured FP64 rate of the device, the FP64 store's roofline: the
    same for a longer run, and in the range of the GB300's nominal FP64 rate
    (about 1.25 TFLOP/s: 2 FMA per clock per SM at 2 GHz)."""
    r1 = S.sl_selftest_fp64_rate(1 << 12)
    r2 = S.sl_selftest_fp64_rate(1 << 14)
    assert 0.3e12 < r2 < 5e12, r2
    assert abs(r1 - r2) < 0.2 * r2
