"""Parity of the stores of "# double" = 0, 2, 3 (Sec. III-A, Tables II-VI)
with the CPU oracle, through the C ABI.

Tolerances:
  * the store itself (set then get, raw planes, integer shifts): bit-exact
    against the oracle's round_storage / stored_sweeps;
  * rows of FP64 coefficients fed only by FP64 coefficients: max relative
    error <= 1e-13 against the FP64 oracle (FP64 arithmetic, another order);
  * split steps: relative function-space L2 <= 1e-6 against the oracle with
    the state rounded to the store after every sweep, and <= 1e-5 against the
    plain FP64 oracle (as for the mixed store);
  * mass drift <= 1e-13 for # double >= 1 (the FP64 conservation form of the
    mean row); the all-FP32 store conserves mass only to FP32 rounding.
"""
import numpy as np
import pytest

import oracle as O
import paper_1603_07008_gb300 as S
from paper_1603_07008_gb300 import workloads as W

pytestmark = pytest.mark.gpu

Q = {"fp32": 0, "mix_fp32_d2": 2, "mix_fp32_d3": 3}
# (storage, k) pairs built: # double = q needs k >= q
CASES = [("fp32", 1), ("fp32", 2), ("fp32", 3), ("mix_fp32_d2", 2), ("mix_fp32_d2", 3), ("mix_fp32_d3", 3)]
SHAPES = [(1,), (7,), (65,), (5, 3), (9, 4), (3, 5, 2), (2, 3, 2, 3), (2, 2, 1, 2, 2)]


def _grid(n, pair=None):
    d = len(n)
    return W.Grid(n=tuple(n), lo=(0.0,) * d, hi=(1.0,) * d, pair=tuple(pair or (-1,) * d))


def _rand(n, k, seed):
    return W.random_coefficients(int(np.prod(n)), k, len(n), seed)


def _skip_big(n, k):
    if (k + 1) ** len(n) > 512:
        pytest.skip("coefficient count covered by smaller shapes")


@pytest.mark.parametrize("storage,k", CASES)
@pytest.mark.parametrize("n", SHAPES)
def test_store_holds_the_rounded_state(storage, k, n):
    """set then get returns exactly what the store of # double = q holds:
    FP64 coefficients unchanged, the others rounded to FP32 (bit-exact), and
    the raw planes are the FP64 / FP32 blocks in coefficient order."""
    _skip_big(n, k)
    q, d = Q[storage], len(n)
    u = _rand(n, k, 3)
    want = O.round_storage(u, k, d, q)
    with S.Context(_grid(n), k, storage) as ctx:
        ctx.set_coeffs(u)
        assert np.array_equal(ctx.get_coeffs(), want)
        mean, hi, scale = S.sl_get_planes(ctx.handle)
        assert scale is None
        mask = O.fp64_coefficients(k, d, q)
        lo_ref = want[:, mask].T
        if mean is None:
            assert not mask.any()
        else:
            assert np.array_equal(mean.reshape(-1, want.shape[0]), lo_ref)
        assert hi.dtype == np.float32 and np.array_equal(hi.astype(np.float64), want[:, ~mask].T)
        # the planes written back reproduce the state
        ctx.set_coeffs(np.zeros_like(u))
        S.sl_set_planes(ctx.handle, mean, hi)
        ctx.synchronize()
        assert np.array_equal(ctx.get_coeffs(), want)


@pytest.mark.parametrize("storage,k", CASES)
@pytest.mark.parametrize("n", [(7,), (5, 3), (3, 4, 2), (2, 3, 2, 3)])
def test_integer_shifts_permute_the_stored_values(storage, k, n):
    _skip_big(n, k)
    q = Q[storage]
    u = _rand(n, k, 4)
    with S.Context(_grid(n), k, storage) as ctx:
        for dim in range(len(n)):
            for sd in [-1] + [m for m in range(len(n)) if m != dim]:
                cnt = 1 if sd < 0 else n[sd]
                s = np.array([(-1) ** c * (2 * c + 1) for c in range(cnt)], dtype=float)
                ctx.set_coeffs(u)
                ctx.advect(dim, sd, s)
                assert np.array_equal(ctx.get_coeffs(), O.stored_sweeps(u, n, k, q, [(dim, sd, s)])), (dim, sd)


@pytest.mark.parametrize("storage,k", [c for c in CASES if c[0] != "fp32"])
@pytest.mark.parametrize("n", [(33,), (6, 5), (4, 3, 5), (3, 2, 3, 2)])
def test_fp64_rows_are_computed_in_fp64(storage, k, n):
    """With every FP32 coefficient zero, a sweep's FP64 rows depend only on
    FP64 values: they must agree with the FP64 oracle to FP64 rounding (an
    FP32 step anywhere on that path would show as ~1e-8).  The FP32 rows are
    FP32 roundings of FP64 values."""
    _skip_big(n, k)
    q, d = Q[storage], len(n)
    mask = O.fp64_coefficients(k, d, q)
    u = _rand(n, k, 5)
    u[:, ~mask] = 0.0
    rng = np.random.default_rng(6)
    with S.Context(_grid(n), k, storage) as ctx:
        for dim in range(d):
            sd = (dim + 1) % d if d > 1 else -1
            cnt = 1 if sd < 0 else n[sd]
            s = rng.uniform(-2.5 * n[dim], 2.5 * n[dim], size=cnt)
            ctx.set_coeffs(u)
            ctx.advect(dim, sd, s)
            got = ctx.get_coeffs()
            ref = O.sweep(u, n, k, dim, sd, s)
            scale = np.max(np.abs(ref))
            assert np.max(np.abs(got[:, mask] - ref[:, mask])) <= 1e-13 * scale, dim
            assert np.max(np.abs(got[:, ~mask] - ref[:, ~mask])) <= 1e-6 * scale, dim


@pytest.mark.parametrize("storage,k", CASES)
@pytest.mark.parametrize("n", [(37,), (9, 7), (5, 4, 3), (3, 4, 2, 3)])
def test_single_sweeps_match_the_stored_oracle(storage, k, n):
    _skip_big(n, k)
    q, d = Q[storage], len(n)
    rng = np.random.default_rng(7)
    u = _rand(n, k, 8)
    with S.Context(_grid(n), k, storage) as ctx:
        for dim in range(d):
            for sd in [-1] + [m for m in range(d) if m != dim]:
                cnt = 1 if sd < 0 else n[sd]
                s = rng.uniform(-2.5 * n[dim], 2.5 * n[dim], size=cnt)
                ctx.set_coeffs(u)
                ctx.advect(dim, sd, s)
                got = ctx.get_coeffs()
                ref = O.stored_sweeps(u, n, k, q, [(dim, sd, s)])
                assert O.rel_l2(got, ref, k, d) <= 1e-6, (dim, sd)


def _strang(p, storage, steps):
    with S.Context(p.grid, p.k, storage) as ctx:
        ctx.project(p.nq, p.weights, p.params)
        ctx.set_fields(p.field_list())
        m0 = ctx.mass()
        ctx.step("strang", p.dt, steps)
        return ctx.get_coeffs(), abs(ctx.mass() - m0) / abs(m0)


@pytest.mark.parametrize("storage", ["fp32", "mix_fp32_d2"])
@pytest.mark.parametrize("cfg", ["2d", "4d"])
def test_strang_steps_match_oracle(storage, cfg):
    p = W.config2(n=48, steps=20) if cfg == "2d" else W.config3(n=6, steps=3)
    q = Q[storage]
    u0 = O.project(p.grid, p.k, p.nq, p.weights, p.params)
    sched = O.schedule(p.grid, "strang", p.dt, p.field_list())
    ref64 = O.step(u0, p.grid, p.k, "strang", p.dt, p.steps, p.field_list())
    refst = O.stored_sweeps(u0, p.grid.n, p.k, q, sched * p.steps)
    got, drift = _strang(p, storage, p.steps)
    assert O.rel_l2(got, refst, p.k, p.grid.ndim) <= 1e-6
    assert O.rel_l2(got, ref64, p.k, p.grid.ndim) <= 1e-5
    if q >= 1:
        assert drift <= 1e-13


def test_strang_d3_matches_oracle():
    p = W.config2(n=32, steps=10)
    p.k = 3
    u0 = O.project(p.grid, 3, p.nq, p.weights, p.params)
    sched = O.schedule(p.grid, "strang", p.dt, p.field_list())
    refst = O.stored_sweeps(u0, p.grid.n, 3, 3, sched * p.steps)
    got, drift = _strang(p, "mix_fp32_d3", p.steps)
    assert O.rel_l2(got, refst, 3, 2) <= 1e-6
    assert drift <= 1e-13


@pytest.mark.parametrize("storage,k", [("mix_fp32_d2", 2), ("mix_fp32_d2", 3), ("mix_fp32_d3", 3)])
def test_mass_drift_1000_steps(storage, k):
    p = W.config2(n=64, steps=1000)
    p.k = k
    with S.Context(p.grid, k, storage) as ctx:
        ctx.project(p.nq, p.weights, p.params)
        ctx.set_fields(p.field_list())
        m0 = ctx.mass()
        ctx.step("strang", p.dt, 1000)
        m1 = ctx.mass()
    assert abs(m1 - m0) / abs(m0) <= 1e-13


def test_fp32_mass_is_its_own_mean_plane():
    """The all-FP32 store has no FP64 plane: its mass reduction reads the FP32
    mean plane and must equal the oracle's mass of the stored state."""
    n, k = (40, 24), 2
    g = W.Grid(n=n, lo=(0.0, -1.0), hi=(2.0, 3.0), pair=(-1, -1))
    u = _rand(n, k, 9)
    with S.Context(g, k, "fp32") as ctx:
        ctx.set_coeffs(u)
        m = ctx.mass()
    ref = O.mass(O.round_storage(u, k, 2, 0), g, k)
    assert abs(m - ref) <= 1e-14 * abs(ref)


@pytest.mark.parametrize("storage,k", [("fp32", 2), ("mix_fp32_d2", 2), ("mix_fp32_d3", 3)])
@pytest.mark.parametrize("n", [(37, 5, 3), (8, 6, 4), (12, 3, 5)])
def test_every_launch_shape_gives_identical_results(storage, k, n):
    _skip_big(n, k)
    rng = np.random.default_rng(10)
    u = _rand(n, k, 11)
    with S.Context(_grid(n), k, storage) as ctx:
        for dim in range(len(n)):
            sd = (dim + 1) % len(n)
            s = rng.uniform(-2.5 * n[dim], 2.5 * n[dim], size=n[sd])
            ctx.set_coeffs(u)
            ctx.advect(dim, sd, s)
            ref = ctx.get_coeffs()
            if storage == "fp32":
                nfib = (k + 1) ** (len(n) - 1)
                if dim == 0:
                    shapes = [dict(block=b, fibres_per_thread=f) for f in (1, 2, 3) if f <= nfib for b in (64, 256)]
                    if n[0] % 4 == 0:
                        shapes += [dict(block=128, fibres_per_thread=f, unroll=4) for f in (1, 2) if f <= nfib]
                else:
                    shapes = [dict(block=128, fibres_per_thread=f, unroll=un, chunk=ch) for f, un in [(1, 1), (2, 2), (1, 4)]
                              if f <= nfib for ch in sorted({1, n[dim]})]
                    shapes.append(dict(block=64, fibres_per_thread=1, pipeline=4, chunk=n[dim]))
            else:
                if dim == 0:
                    shapes = [dict(block=b, fibres_per_thread=1) for b in (32, 128, 256)]
                else:
                    shapes = [dict(block=b, fibres_per_thread=1, unroll=un, chunk=ch) for b in (32, 128)
                              for un in (1, 2) for ch in sorted({1, 2, n[dim]})]
            for sh in shapes:
                ctx.set_tune(dim, **sh)
                ctx.set_coeffs(u)
                ctx.advect(dim, sd, s)
                assert np.array_equal(ctx.get_coeffs(), ref), (dim, sh)


def test_split_stores_reject_shapes_not_built():
    with S.Context(_grid((8, 6)), 2, "mix_fp32_d2") as ctx:
        for dim, sh in [(0, dict(block=128, fibres_per_thread=2)), (0, dict(block=128, fibres_per_thread=1, unroll=4)),
                        (1, dict(block=128, fibres_per_thread=1, unroll=4, chunk=3)),
                        (1, dict(block=128, fibres_per_thread=1, pipeline=4, chunk=3)),
                        (1, dict(block=128, fibres_per_thread=1, unroll=1, chunk=3, max_blocks_per_sm=4)),
                        (1, dict(block=256, fibres_per_thread=1, unroll=1, chunk=3))]:
            with pytest.raises(S.SlError):
                ctx.set_tune(dim, **sh)


def test_autotune_keeps_results():
    p = W.config2(n=40, steps=3)
    with S.Context(p.grid, p.k, "mix_fp32_d2") as a, S.Context(p.grid, p.k, "mix_fp32_d2") as b:
        for c in (a, b):
            c.project(p.nq, p.weights, p.params)
            c.set_fields(p.field_list())
        b.autotune(2)
        b.project(p.nq, p.weights, p.params)
        a.step("strang", p.dt, 3)
        b.step("strang", p.dt, 3)
        assert np.array_equal(a.get_coeffs(), b.get_coeffs())


def test_graph_replay_matches_step():
    import torch
    p = W.config2(n=24, steps=6)
    st = torch.cuda.Stream()
    with S.Context(p.grid, p.k, "mix_fp32_d2", stream=st) as a, \
            S.Context(p.grid, p.k, "mix_fp32_d2", stream=st) as b:
        for c in (a, b):
            c.project(p.nq, p.weights, p.params)
            c.set_fields(p.field_list())
        a.step("strang", p.dt, 6)
        b.graph_capture("strang", p.dt, 3)
        b.graph_launch()
        b.graph_launch()
        assert np.array_equal(a.get_coeffs(), b.get_coeffs())


def test_self_consistent_field_reads_the_fp64_mean():
    p = W.config2(n=32, steps=2)
    with S.Context(p.grid, p.k, "mix_fp32_d2") as a, S.Context(p.grid, p.k, "mix_fp32") as b:
        for c in (a, b):
            c.project(p.nq, p.weights, p.params)
            c.set_poisson(True)
        assert np.array_equal(a.field(), b.field())   # the same FP64 mean plane
    with S.Context(p.grid, p.k, "fp32") as c:
        with pytest.raises(S.SlError) as e:
            c.set_poisson(True)
        assert e.value.status == S.SL_ENOTSUP


@pytest.mark.parametrize("storage", ["mix_fp32_d2", "mix_fp32_d3", "fp32"])
def test_paper1d_full_size_sampled(storage):
    """The 1D workload of the paper's tables at the bench's size (order 4,
    N = 2^27, default shapes): one sweep, sampled target cells against the
    oracle applied to the stored source cells of each (a two-cell periodic
    problem with the same shift reproduces the update rule of one target)."""
    import math
    k, N, shift = 3, 1 << 27, 0.37
    q = Q[storage]
    g = W.Grid(n=(N,), lo=(0.0,), hi=(1.0,), pair=(-1,))
    rng = np.random.default_rng(12)
    cells = np.unique(np.concatenate([[0, 1, N - 1], rng.integers(0, N, size=61)])).astype(np.int64)
    with S.Context(g, k, storage) as ctx:
        ctx.project(k + 2, [1.0, 1.0], [[[0.0, 0.0, 0.0, 0.0]], [[0.0, 0.0, 2 * math.pi * 8, 0.3]]])
        src = ctx.get_cells(np.concatenate([cells, (cells - 1) % N]))
        m0 = ctx.mass()
        ctx.advect(0, -1, [shift])
        got = ctx.get_cells(cells)
        m1 = ctx.mass()
    a, b = src[: cells.size], src[cells.size:]
    ref = np.empty_like(got)
    for r in range(cells.size):
        u2 = np.stack([b[r], a[r]])          # cells i - 1, i of a two-cell line
        ref[r] = O.stored_sweeps(u2, (2,), k, q, [(0, -1, [shift])])[1]
    assert O.rel_l2(got, ref, k, 1) <= 1e-6
    if q >= 1:
        assert abs(m1 - m0) <= 1e-13 * abs(m0)
