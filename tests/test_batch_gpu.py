"""Batched sweeps (many independent problems, one persistent launch per
split substep): every problem must match the same problem advanced alone
(bit-exactly: the same arithmetic on the same tables) and the CPU oracle."""
import numpy as np
import pytest

import oracle as O
import paper_1603_07008_gb300 as S
from paper_1603_07008_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _problems(sizes, degrees, storage):
    out = []
    for (nx, nv), k in zip(sizes, degrees):
        p = W.config2(n=8, steps=1, storage=storage)
        g = W.Grid(n=(nx, nv), lo=p.grid.lo, hi=p.grid.hi, pair=p.grid.pair)
        q = W.config2(n=8, steps=1, storage=storage)
        q.grid = g
        q.k = k
        q.fields = {0: 0.1 * np.sin(0.5 * (g.lo[0] + (np.arange(nx) + 0.5) * (g.hi[0] - g.lo[0]) / nx))}
        out.append(q)
    return out


SIZES = [(64, 40), (33, 70), (128, 17), (5, 9), (96, 96), (1, 31)]
DEGS = [1, 2, 0, 2, 1, 2]


@pytest.mark.parametrize("storage", ["mix_fp32", "fp64"])
def test_batch_matches_single_problems_and_oracle(storage):
    probs = _problems(SIZES, DEGS, storage)
    steps = 3
    with S.Batch([p.grid for p in probs], [p.k for p in probs], storage) as b:
        for i, p in enumerate(probs):
            b.project(i, p.nq, p.weights, p.params)
        b.set_fields([p.field_list()[0] for p in probs])
        m0 = b.mass()
        b.step("strang", p.dt, steps)
        m1 = b.mass()
        got = [b.get_coeffs(i) for i in range(len(probs))]
    assert np.all(np.abs(m1 - m0) <= 1e-13 * np.abs(m0))
    for i, p in enumerate(probs):
        with S.Context(p.grid, p.k, storage) as c:
            c.project(p.nq, p.weights, p.params)
            c.set_fields(p.field_list())
            c.step("strang", p.dt, steps)
            alone = c.get_coeffs()
        assert np.array_equal(got[i], alone), i
        ref = O.step(O.project(p.grid, p.k, p.nq, p.weights, p.params), p.grid, p.k, "strang",
                     p.dt, steps, p.field_list())
        if storage == "fp64":
            assert O.rel_max(got[i], ref) <= 1e-12
        else:
            assert O.rel_l2(got[i], ref, p.k, 2) <= 1e-5


def test_batch_graph_and_autotune_keep_results():
    import torch
    probs = _problems(SIZES, DEGS, "mix_fp32")
    s = torch.cuda.Stream()
    res = []
    for mode in ("step", "graph"):
        with S.Batch([p.grid for p in probs], [p.k for p in probs], "mix_fp32", stream=s) as b:
            for i, p in enumerate(probs):
                b.project(i, p.nq, p.weights, p.params)
            b.set_fields([p.field_list()[0] for p in probs])
            if mode == "step":
                b.step("strang", 0.1, 4)
            else:
                b.autotune(2)
                b.graph_capture("strang", 0.1, 1)   # 3 sweeps: odd, two graphs
                for _ in range(4):
                    b.graph_launch()
            res.append([b.get_coeffs(i) for i in range(len(probs))])
    for a, c in zip(*res):
        assert np.array_equal(a, c)


def test_batch_profile_and_tune_readback():
    probs = _problems(SIZES, DEGS, "mix_fp32")
    with S.Batch([p.grid for p in probs], [p.k for p in probs], "mix_fp32") as b:
        for i, p in enumerate(probs):
            b.project(i, p.nq, p.weights, p.params)
        b.set_fields([p.field_list()[0] for p in probs])
        t0, t1 = b.get_tune(0), b.get_tune(1)
        assert t0["block"] == 128 and 1 <= t0["fibres_per_thread"] <= 3 and t0["chunk"] % 128 == 0
        assert 1 <= t1["fibres_per_thread"] <= 2 and t1["unroll"] in (1, 2, 4) and t1["chunk"] >= 1
        b.profile_enable(True)
        b.step("strang", 0.1, 2)          # x/2, v, x/2 per step
        n, ms, by = b.profile_query()
        nd, msd = b.profile_dims()
        assert n == 6 and nd[:2] == [4, 2] and sum(nd) == 6
        assert abs(sum(msd) - ms) <= 1e-6 * max(ms, 1.0)
        with pytest.raises(S.SlError):
            b.get_tune(2)


def test_batch_mass_matches_single_problem_mass():
    probs = _problems(SIZES, DEGS, "fp64")
    with S.Batch([p.grid for p in probs], [p.k for p in probs], "fp64") as b:
        for i, p in enumerate(probs):
            b.project(i, p.nq, p.weights, p.params)
        m = b.mass()
    for i, p in enumerate(probs):
        with S.Context(p.grid, p.k, "fp64") as c:
            c.project(p.nq, p.weights, p.params)
            assert abs(c.mass() - m[i]) <= 1e-13 * abs(m[i])


def test_batch_rejects_what_it_does_not_support():
    probs = _problems(SIZES[:2], [1, 1], "mix_fp32")
    with pytest.raises(S.SlError) as e:
        S.sl_batch_create([p.grid for p in probs], [1, 3], "mix_fp32")
    assert e.value.status == S.SL_ENOTSUP
    with pytest.raises(S.SlError) as e:
        S.sl_batch_create([p.grid for p in probs], [1, 1], "mix_bf16")
    assert e.value.status == S.SL_ENOTSUP
    g3 = W.Grid(n=(4, 4, 4), lo=(0.0,) * 3, hi=(1.0,) * 3, pair=(1, -1, -1))
    with pytest.raises(S.SlError) as e:
        S.sl_batch_create([probs[0].grid, g3], [1, 1], "mix_fp32")
    assert e.value.status == S.SL_EINVAL
    with S.Batch([p.grid for p in probs], [1, 1], "mix_fp32") as b:
        with pytest.raises(S.SlError) as e:
            b.step("strang", 0.1, 1)   # fields not set
        assert e.value.status == S.SL_EINVAL


def test_config4_full_size_batch():
    """256 problems, N_x, N_v in [64, 1024], k in {1, 2}, FP32 mixed: two
    Strang steps; every mass conserved, sampled problems match the oracle."""
    probs = W.config4()
    with S.Batch([p.grid for p in probs], [p.k for p in probs], "mix_fp32") as b:
        for i, p in enumerate(probs):
            b.project(i, p.nq, p.weights, p.params)
        b.set_fields([p.field_list()[0] for p in probs])
        m0 = b.mass()
        b.step("strang", 0.1, 2)
        m1 = b.mass()
        picks = [0, 17, 255, int(np.argmin([q.grid.cells for q in probs]))]
        got = {i: b.get_coeffs(i) for i in picks}
    assert np.all(np.abs(m1 - m0) <= 1e-13 * np.abs(m0))
    for i in picks:
        p = probs[i]
        ref = O.step(O.project(p.grid, p.k, p.nq, p.weights, p.params), p.grid, p.k, "strang",
                     0.1, 2, p.field_list())
        assert O.rel_l2(got[i], ref, p.k, 2) <= 1e-5


def test_batch_every_shape_gives_identical_results():
    """Every work-list shape (fibres per thread, cells per thread or per walk
    step, item size) changes only the work distribution."""
    probs = _problems(SIZES, DEGS, "mix_fp32")
    shapes0 = [dict(fibres_per_thread=f, unroll=u, chunk=128 * u * r)
               for f, u in [(1, 1), (2, 1), (3, 1), (1, 2), (3, 2), (1, 4), (2, 4)] for r in (1, 3)]
    shapes1 = [dict(fibres_per_thread=f, unroll=u, chunk=ch) for f in (1, 2) for u in (1, 2, 4) for ch in (1, 7, 1 << 30)]
    with S.Batch([p.grid for p in probs], [p.k for p in probs], "mix_fp32") as b:
        for i, p in enumerate(probs):
            b.project(i, p.nq, p.weights, p.params)
        b.set_fields([p.field_list()[0] for p in probs])
        init = [b.get_coeffs(i) for i in range(len(probs))]

        def run():
            for i in range(len(probs)):
                b.set_coeffs(i, init[i])
            b.step("strang", 0.1, 2)
            return [b.get_coeffs(i) for i in range(len(probs))]

        ref = run()
        for dim, shapes in ((0, shapes0), (1, shapes1)):
            keep = b.get_tune(dim)
            for sh in shapes:
                b.set_tune(dim, **sh)
                t = b.get_tune(dim)
                assert (t["fibres_per_thread"], t["unroll"], t["chunk"]) == (sh["fibres_per_thread"], sh["unroll"], sh["chunk"])
                got = run()
                for a, c in zip(got, ref):
                    assert np.array_equal(a, c), (dim, sh)
            b.set_tune(dim, **keep)
        for dim, sh in [(0, dict(fibres_per_thread=3, unroll=4, chunk=512)), (0, dict(fibres_per_thread=1, unroll=1, chunk=100)),
                        (0, dict(fibres_per_thread=1, unroll=1, chunk=128 * 9)), (1, dict(fibres_per_thread=3, unroll=1, chunk=8)),
                        (1, dict(fibres_per_thread=1, unroll=3, chunk=8)), (1, dict(fibres_per_thread=1, unroll=1, chunk=0)),
                        (1, dict(fibres_per_thread=1, unroll=1, chunk=8, block=64)), (2, dict(fibres_per_thread=1, unroll=1, chunk=8))]:
            with pytest.raises(S.SlError) as e:
                b.set_tune(dim, **sh)
            assert e.value.status == S.SL_EINVAL


def test_batch_lie_matches_single_problems():
    probs = _problems(SIZES, DEGS, "mix_fp32")
    with S.Batch([p.grid for p in probs], [p.k for p in probs], "mix_fp32") as b:
        for i, p in enumerate(probs):
            b.project(i, p.nq, p.weights, p.params)
        b.set_fields([p.field_list()[0] for p in probs])
        b.step("lie", 0.1, 3)
        got = [b.get_coeffs(i) for i in range(len(probs))]
    for i, p in enumerate(probs):
        with S.Context(p.grid, p.k, "mix_fp32") as c:
            c.project(p.nq, p.weights, p.params)
            c.set_fields(p.field_list())
            c.step("lie", 0.1, 3)
            assert np.array_equal(got[i], c.get_coeffs()), i


def test_batch_fields_changed_between_graph_replays_are_used():
    """The batch builds every problem's tables once per split step from the
    fields as they are then, also inside a captured step: after sl_set_fields
    a replayed graph uses the new fields, bit for bit as the problems stepped
    alone with the same fields."""
    import torch
    probs = _problems(SIZES, DEGS, "mix_fp32")
    f1 = [p.field_list()[0] for p in probs]
    f2 = [-2.0 * f + 0.03 for f in f1]
    st = torch.cuda.Stream()
    with S.Batch([p.grid for p in probs], [p.k for p in probs], "mix_fp32", stream=st) as b:
        for i, p in enumerate(probs):
            b.project(i, p.nq, p.weights, p.params)
        b.set_fields(f1)
        b.graph_capture("strang", 0.1, 1)
        b.graph_launch()
        b.set_fields(f2)
        b.graph_launch()
        got = [b.get_coeffs(i) for i in range(len(probs))]
    for i, p in enumerate(probs):
        with S.Context(p.grid, p.k, "mix_fp32") as c:
            c.project(p.nq, p.weights, p.params)
            c.set_fields([f1[i]])
            c.step("strang", 0.1, 1)
            c.set_fields([f2[i]])
            c.step("strang", 0.1, 1)
            alone = c.get_coeffs()
        assert np.array_equal(got[i], alone), i
