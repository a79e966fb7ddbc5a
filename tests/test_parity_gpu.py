"""Parity of the CUDA sweep library (through its C ABI) with the CPU oracle.

Tolerances (stated for the method's outputs):
  * FP64 store:        max |gpu - oracle| / max |oracle| <= 1e-12
  * mixed FP32 store:  relative function-space L2 <= 1e-5 after 100 steps
  * BF16 / FP16 store: relative function-space L2 <= 1e-2
  * every store:       relative mass drift <= 1e-13 after 1000 steps
  * integer shifts:    bit-exact permutation.
All inputs are seeded; the oracle never sees a value computed on the GPU.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_1603_07008_gb300 as S
from paper_1603_07008_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIX_TOL = 1e-5
LP_TOL = 1e-2
MASS_TOL = 1e-13


def _grid(n, lo=None, hi=None, pair=None):
    d = len(n)
    return W.Grid(n=tuple(n), lo=tuple(lo or (0.0,) * d), hi=tuple(hi or (1.0,) * d),
                  pair=tuple(pair or (-1,) * d))


def _rand(n, k, seed):
    return W.random_coefficients(int(np.prod(n)), k, len(n), seed)


def _shifts(rng, n, dim, shift_dim, scale=2.5):
    cnt = 1 if shift_dim < 0 else n[shift_dim]
    return rng.uniform(-scale * n[dim], scale * n[dim], size=cnt)


SHAPES = [(1,), (2,), (7,), (33,), (64,), (5, 3), (31, 2), (3, 7, 2), (4, 3, 2, 3),
          (2, 3, 1, 2, 3), (2, 2, 3, 2, 1, 2)]


@pytest.mark.parametrize("n", SHAPES)
@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_fp64_single_sweeps_match_oracle(n, k):
    if (k + 1) ** len(n) > 1024:
        pytest.skip("large coefficient count covered elsewhere")
    rng = np.random.default_rng(hash((n, k)) % 2**32)
    u = _rand(n, k, 1)
    with S.Context(_grid(n), k, "fp64") as ctx:
        for dim in range(len(n)):
            for sd in [-1] + [m for m in range(len(n)) if m != dim]:
                s = _shifts(rng, n, dim, sd)
                ctx.set_coeffs(u)
                ctx.advect(dim, sd, s)
                got = ctx.get_coeffs()
                ref = O.sweep(u, n, k, dim, sd, s)
                assert O.rel_max(got, ref) <= FP64_TOL, (dim, sd)


@pytest.mark.parametrize("n", [(7,), (5, 3), (3, 4, 2), (2, 3, 2, 3)])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_integer_shifts_are_bit_exact(n, k):
    u = _rand(n, k, 2)
    with S.Context(_grid(n), k, "fp64") as ctx:
        for dim in range(len(n)):
            for sd in [-1] + [m for m in range(len(n)) if m != dim]:
                cnt = 1 if sd < 0 else n[sd]
                s = np.array([(-1) ** c * (3 * c + 1) for c in range(cnt)], dtype=float)
                ctx.set_coeffs(u)
                ctx.advect(dim, sd, s)
                assert np.array_equal(ctx.get_coeffs(), O.sweep(u, n, k, dim, sd, s))


@pytest.mark.parametrize("storage", ["mix_fp32", "mix_bf16", "mix_fp16"])
def test_integer_shifts_permute_the_stored_values(storage):
    """In the low-precision stores an integer shift moves stored values
    unchanged: the result is the periodic roll of what was stored."""
    n = (6, 5, 3)
    k = 1
    with S.Context(_grid(n), k, storage) as ctx:
        ctx.set_coeffs(_rand(n, k, 3))
        before = ctx.get_coeffs()
        for dim, sh in [(0, 2.0), (1, -7.0), (2, 4.0)]:
            ctx.advect(dim, -1, [sh])
            after = ctx.get_coeffs()
            B = before.reshape(tuple(reversed(n)) + (-1,))
            ref = np.roll(B, int(sh), axis=len(n) - 1 - dim).reshape(before.shape)
            assert np.array_equal(after, ref)
            before = after


def test_projection_matches_oracle():
    for p in [W.config1(), W.config2(n=48, steps=1), W.config3(n=6, steps=1),
              W.config5(n=3, steps=1)]:
        with S.Context(p.grid, p.k, "fp64") as ctx:
            ctx.project(p.nq, p.weights, p.params)
            got = ctx.get_coeffs()
        ref = O.project(p.grid, p.k, p.nq, p.weights, p.params)
        assert O.rel_max(got, ref) <= 1e-14, p.name


def test_config1_fp64_100_steps():
    """1D, N = 1024, k = 2, dt = 0.37/N, 100 steps, all FP64."""
    p = W.config1()
    g = p.grid
    h = (g.hi[0] - g.lo[0]) / g.n[0]
    s = p.velocity * p.dt / h
    u0 = O.project(g, p.k, p.nq, p.weights, p.params)
    ref = u0
    for _ in range(p.steps):
        ref = O.sweep(ref, g.n, p.k, 0, -1, s)
    with S.Context(g, p.k, p.storage) as ctx:
        ctx.project(p.nq, p.weights, p.params)
        m0 = ctx.mass()
        for _ in range(p.steps):
            ctx.advect(0, -1, [s])
        got = ctx.get_coeffs()
        m1 = ctx.mass()
    assert O.rel_max(got, ref) <= FP64_TOL
    assert abs(m1 - m0) / abs(m0) <= MASS_TOL


@pytest.mark.parametrize("n,k", [((5, 3), 2), ((7, 2, 3), 1), ((4, 3, 2, 3), 2), ((33,), 3)])
def test_mixed_fp32_single_sweeps(n, k):
    rng = np.random.default_rng(7)
    u = _rand(n, k, 4)
    with S.Context(_grid(n), k, "mix_fp32") as ctx:
        for dim in range(len(n)):
            for sd in [-1] + [m for m in range(len(n)) if m != dim]:
                s = _shifts(rng, n, dim, sd)
                ctx.set_coeffs(u)
                stored = ctx.get_coeffs()
                ctx.advect(dim, sd, s)
                got = ctx.get_coeffs()
                # against the oracle applied to exactly what was stored
                ref = O.sweep(stored, n, k, dim, sd, s)
                assert O.rel_l2(got, ref, k, len(n)) <= 1e-6
                # the mean row adds the FP32 higher coefficients' contribution
                # rounded in FP32: at most a few FP32 ulps of those terms
                assert np.max(np.abs(got[:, 0] - ref[:, 0])) <= 1e-6 * np.max(np.abs(stored[:, 1:]))


def _strang_oracle(p, steps):
    u = O.project(p.grid, p.k, p.nq, p.weights, p.params)
    return O.step(u, p.grid, p.k, "strang", p.dt, steps, p.field_list())


def _strang_gpu(p, storage, steps, graph=False):
    with S.Context(p.grid, p.k, storage) as ctx:
        ctx.project(p.nq, p.weights, p.params)
        ctx.set_fields(p.field_list())
        m0 = ctx.mass()
        ctx.step("strang", p.dt, steps)
        out = ctx.get_coeffs()
        m1 = ctx.mass()
    return out, abs(m1 - m0) / abs(m0)


@pytest.mark.parametrize("cfg", ["2d", "4d"])
def test_strang_fp64_matches_oracle(cfg):
    p = W.config2(n=40, steps=5) if cfg == "2d" else W.config3(n=8, steps=2)
    ref = _strang_oracle(p, p.steps)
    got, drift = _strang_gpu(p, "fp64", p.steps)
    assert O.rel_max(got, ref) <= FP64_TOL
    assert drift <= MASS_TOL


def test_config2_mixed_fp32_100_steps_full_size():
    """2D x-v, 512 x 512, k = 2, FP64 means + FP32 higher coefficients,
    Strang, dt = 0.1: relative L2 against the FP64 oracle after 100 steps."""
    p = W.config2(n=512, steps=100)
    ref = _strang_oracle(p, 100)
    got, drift = _strang_gpu(p, "mix_fp32", 100)
    err = O.rel_l2(got, ref, p.k, 2)
    assert err <= MIX_TOL, err
    assert drift <= MASS_TOL


def test_config2_fp64_full_size():
    p = W.config2(n=512, steps=20)
    ref = _strang_oracle(p, 20)
    got, drift = _strang_gpu(p, "fp64", 20)
    assert O.rel_max(got, ref) <= FP64_TOL
    assert drift <= MASS_TOL


@pytest.mark.parametrize("storage", ["mix_bf16", "mix_fp16"])
@pytest.mark.parametrize("cfg", ["6d", "4d", "2d"])
def test_scaled_stores_match_oracle(storage, cfg):
    if cfg == "6d":
        p = W.config5(n=4, steps=2)
    elif cfg == "4d":
        p = W.config3(n=6, steps=2)
    else:
        p = W.config2(n=64, steps=20)
    ref = _strang_oracle(p, p.steps)
    got, drift = _strang_gpu(p, storage, p.steps)
    err = O.rel_l2(got, ref, p.k, p.grid.ndim)
    assert err <= LP_TOL, err
    assert drift <= MASS_TOL


@pytest.mark.parametrize("storage", ["fp64", "mix_fp32", "mix_bf16", "mix_fp16"])
def test_mass_drift_1000_steps(storage):
    p = W.config2(n=64, steps=1000)
    k = 2 if storage in ("fp64", "mix_fp32") else 1
    p.k = k
    with S.Context(p.grid, k, storage) as ctx:
        ctx.project(p.nq, p.weights, p.params)
        ctx.set_fields(p.field_list())
        m0 = ctx.mass()
        ctx.step("strang", p.dt, 1000)
        m1 = ctx.mass()
    assert abs(m1 - m0) / abs(m0) <= MASS_TOL


@pytest.mark.parametrize("storage", ["fp64", "mix_fp32", "mix_bf16"])
def test_mass_drift_1d_1000_steps(storage):
    p = W.config1()
    k = 2 if storage != "mix_bf16" else 1
    h = 1.0 / 1024
    s = p.velocity * p.dt / h
    with S.Context(p.grid, k, storage) as ctx:
        ctx.project(p.nq, p.weights, p.params)
        m0 = ctx.mass()
        for _ in range(1000):
            ctx.advect(0, -1, [s])
        m1 = ctx.mass()
    assert abs(m1 - m0) / abs(m0) <= MASS_TOL


def test_config3_full_size_sampled_after_one_step():
    """4D 64^4, k = 2, mixed FP32: one Strang step (6 sweeps) on the GPU
    against the oracle evaluated on the dependency cones of sampled cells."""
    p = W.config3(n=64, steps=1)
    rng = np.random.default_rng(0)
    cells = np.concatenate([[0, p.grid.cells - 1], rng.integers(0, p.grid.cells, 10)])
    sched = O.schedule(p.grid, "strang", p.dt, p.field_list())
    ref = O.sample_after(p.grid, p.k, p.nq, p.weights, p.params, sched, cells)
    with S.Context(p.grid, p.k, "mix_fp32") as ctx:
        ctx.project(p.nq, p.weights, p.params)
        ctx.set_fields(p.field_list())
        m0 = ctx.mass()
        ctx.step("strang", p.dt, 1)
        got = ctx.get_cells(cells)
        m1 = ctx.mass()
    for i in range(len(cells)):
        assert O.rel_l2(got[i:i + 1], ref[i:i + 1], p.k, 4) <= 1e-5
    assert abs(m1 - m0) / abs(m0) <= MASS_TOL


@pytest.mark.parametrize("storage", ["mix_bf16", "mix_fp16"])
def test_config5_full_size_sampled_after_one_step(storage):
    """6D 20^6, k = 1, FP64 means + scaled BF16/FP16: one Strang step
    (9 sweeps) against the oracle on sampled dependency cones."""
    p = W.config5(n=20, steps=1)
    rng = np.random.default_rng(1)
    cells = np.concatenate([[0, p.grid.cells - 1], rng.integers(0, p.grid.cells, 4)])
    sched = O.schedule(p.grid, "strang", p.dt, p.field_list())
    ref = O.sample_after(p.grid, p.k, p.nq, p.weights, p.params, sched, cells)
    with S.Context(p.grid, p.k, storage) as ctx:
        ctx.project(p.nq, p.weights, p.params)
        ctx.set_fields(p.field_list())
        m0 = ctx.mass()
        ctx.step("strang", p.dt, 1)
        got = ctx.get_cells(cells)
        m1 = ctx.mass()
    assert O.rel_l2(got, ref, p.k, 6) <= LP_TOL
    assert abs(m1 - m0) / abs(m0) <= MASS_TOL


def test_graph_replay_matches_step():
    p = W.config2(n=48, steps=1)
    import torch
    s = torch.cuda.Stream()
    with S.Context(p.grid, p.k, "mix_fp32", stream=s) as a, \
            S.Context(p.grid, p.k, "mix_fp32", stream=s) as b:
        for c in (a, b):
            c.project(p.nq, p.weights, p.params)
            c.set_fields(p.field_list())
        a.step("strang", p.dt, 6)
        b.graph_capture("strang", p.dt, 3)   # 9 sweeps: odd, two graphs alternate
        b.graph_launch()
        b.graph_launch()
        assert np.array_equal(a.get_coeffs(), b.get_coeffs())


def test_codec_round_trip():
    n = (9, 4)
    k = 2
    u = _rand(n, k, 9)
    with S.Context(_grid(n), k, "fp64") as c:
        c.set_coeffs(u)
        assert np.array_equal(c.get_coeffs(), u)
    with S.Context(_grid(n), k, "mix_fp32") as c:
        c.set_coeffs(u)
        got = c.get_coeffs()
        assert np.array_equal(got[:, 0], u[:, 0])
        assert np.array_equal(got[:, 1:], u[:, 1:].astype(np.float32).astype(np.float64))
    for st, rel in (("mix_bf16", 2.0 ** -8), ("mix_fp16", 2.0 ** -11)):
        with S.Context(_grid(n), k, st) as c:
            c.set_coeffs(u)
            got = c.get_coeffs()
            assert np.array_equal(got[:, 0], u[:, 0])
            cmax = np.max(np.abs(u[:, 1:]), axis=1, keepdims=True)
            assert np.all(np.abs(got[:, 1:] - u[:, 1:]) <= rel * cmax)


def test_get_cells_matches_full_download():
    n = (5, 6, 7)
    u = _rand(n, 1, 12)
    with S.Context(_grid(n), 1, "mix_bf16") as c:
        c.set_coeffs(u)
        full = c.get_coeffs()
        idx = np.array([0, 7, 100, 209, 3])
        assert np.array_equal(c.get_cells(idx), full[idx])


def test_invalid_calls_leave_state_unchanged():
    n = (8, 4)
    u = _rand(n, 1, 13)
    with S.Context(_grid(n, pair=(1, -1)), 1, "fp64") as c:
        c.set_coeffs(u)
        for args, code in [((0, -1, [float("nan")]), S.SL_ENAN),
                           ((0, 1, [0.1, 0.2]), S.SL_EINVAL),
                           ((2, -1, [0.1]), S.SL_EINVAL),
                           ((0, 0, [0.1] * 8), S.SL_EINVAL)]:
            with pytest.raises(S.SlError) as e:
                c.advect(*args)
            assert e.value.status == code
        with pytest.raises(S.SlError) as e:
            c.step("strang", 0.1, 1)            # fields not set
        assert e.value.status == S.SL_EINVAL
        bad = u.copy()
        bad[3, 1] = np.inf
        with pytest.raises(S.SlError) as e:
            c.set_coeffs(bad)
        assert e.value.status == S.SL_ENAN
        assert np.array_equal(c.get_coeffs(), u)


def test_profile_counts_sweeps():
    p = W.config2(n=64, steps=1)
    with S.Context(p.grid, p.k, "mix_fp32") as c:
        c.project(p.nq, p.weights, p.params)
        c.set_fields(p.field_list())
        c.profile_enable(True)
        c.step("strang", p.dt, 4)
        n, ms, b = c.profile_query()
    assert n == 12 and ms > 0
    assert b == 12 * 2 * c.info["state_bytes"]


UNIT_FT = [1, 2, 3, 4, 9]
STRIDED_SHAPES = [(1, 1), (1, 2), (1, 4), (2, 1), (2, 2), (2, 4), (3, 1), (3, 2)]
ASYNC_SHAPES = [(1, 4), (1, 8), (2, 4), (2, 8), (3, 4)]


@pytest.mark.parametrize("storage", ["fp64", "mix_fp32"])
@pytest.mark.parametrize("n,k", [((37, 5, 3), 2), ((6, 9, 4), 1), ((3, 4, 5), 3), ((8, 3, 5), 2),
                                 ((4, 6, 2), 1), ((12, 2, 3), 3), ((16, 12), 2), ((20, 6), 1)])
def test_every_launch_shape_gives_identical_results(storage, n, k):
    """Fibres per thread, unroll, block size and chunk length change only the
    work distribution: every shape must give bit-identical output, and the
    output must match the oracle."""
    rng = np.random.default_rng(21)
    u = _rand(n, k, 22)
    g = _grid(n)
    with S.Context(g, k, storage) as ctx:
        for dim in range(len(n)):
            sd = (dim + 1) % len(n)
            s = _shifts(rng, n, dim, sd)
            ctx.set_coeffs(u)
            ctx.advect(dim, sd, s)
            ref_gpu = ctx.get_coeffs()
            ref = O.sweep(ctx_stored(u, storage), n, k, dim, sd, s)
            if storage == "fp64":
                assert O.rel_max(ref_gpu, ref) <= FP64_TOL
            else:
                assert O.rel_l2(ref_gpu, ref, k, len(n)) <= 1e-6
            shapes = []
            nfib = (k + 1) ** (len(n) - 1)
            if dim == 0:
                shapes = [dict(block=b, fibres_per_thread=f) for f in UNIT_FT if f <= nfib
                          for b in (64, 256)]
                vw = 4 if storage == "mix_fp32" else 2
                if n[0] % vw == 0:
                    shapes += [dict(block=b, fibres_per_thread=f, unroll=vw) for f in (1, 2, 3, 4)
                               if f <= nfib for b in (32, 256)]
            else:
                for f, un in STRIDED_SHAPES:
                    if f > nfib:
                        continue
                    for ch in sorted({1, min(3, n[dim]), n[dim]}):
                        shapes.append(dict(block=128, fibres_per_thread=f, unroll=un, chunk=ch))
                shapes.append(dict(block=32, fibres_per_thread=1, unroll=2, chunk=min(2, n[dim])))
                for occ in (4, 5, 6):   # at most occ blocks per SM
                    shapes.append(dict(block=128, fibres_per_thread=1, unroll=4, chunk=n[dim], max_blocks_per_sm=occ))
                for f, pl in ASYNC_SHAPES:
                    if f > nfib:
                        continue
                    for ch in sorted({1, min(2, n[dim]), n[dim]}):
                        for b in (64, 128):
                            shapes.append(dict(block=b, fibres_per_thread=f, pipeline=pl, chunk=ch))
            for sh in shapes:
                ctx.set_tune(dim, **sh)
                ctx.set_coeffs(u)
                ctx.advect(dim, sd, s)
                assert np.array_equal(ctx.get_coeffs(), ref_gpu), (dim, sh)


def ctx_stored(u, storage):
    if storage == "fp64":
        return u
    v = u.copy()
    v[:, 1:] = v[:, 1:].astype(np.float32).astype(np.float64)
    return v


SCALED_SPLITS = {((1, 6)): [32, 16, 8, 4], ((1, 5)): [16, 8, 4], ((2, 4)): [27, 9, 3],
                 ((2, 3)): [9, 3], ((3, 3)): [16, 4], ((1, 4)): [8]}


@pytest.mark.parametrize("storage", ["mix_bf16", "mix_fp16"])
@pytest.mark.parametrize("n,k", [((5, 7, 3, 2), 1), ((3, 2, 2, 3, 2, 2), 1), ((3, 4, 2, 3, 2), 1),
                                 ((4, 3, 3, 2), 2), ((4, 3, 5), 3), ((5, 3, 4), 2)])
def test_scaled_launch_shapes_identical(storage, n, k):
    """Every block size and every split of a cell's fibres over cooperating
    threads gives bit-identical results (the cell maximum does not depend
    on the order it is taken in)."""
    rng = np.random.default_rng(5)
    u = _rand(n, k, 6)
    splits = SCALED_SPLITS[(k, len(n))]
    with S.Context(_grid(n), k, storage) as ctx:
        if ctx.info["record_slots"]:
            splits = splits[:1]   # a cell record is always one thread's
        for dim in range(len(n)):
            s = _shifts(rng, n, dim, -1)
            ctx.set_coeffs(u)
            ctx.advect(dim, -1, s)
            ref = ctx.get_coeffs()
            shapes = []
            for f in splits:
                for b in (32, 64, 128, 256):
                    if b == 256 and (dim > 0 or ctx.info["record_slots"]):
                        continue
                    sh = dict(block=b, fibres_per_thread=f)
                    if dim > 0:
                        sh["chunk"] = min(2, n[dim])
                    shapes.append(sh)
            if ctx.info["record_slots"]:
                # record walks along every dimension, plain and prefetching
                for un in (1, 2):
                    for ch in sorted({1, min(2, n[dim]), n[dim]}):
                        shapes.append(dict(block=64, fibres_per_thread=splits[0], unroll=un, chunk=ch))
                if k == 1 and len(n) in (5, 6):
                    # lane groups: R/16 lanes share a cell, 1, 2 or 4 cells per walk step
                    for un in (1, 2, 4):
                        for ch in sorted({1, min(3, n[dim]), n[dim]}):
                            for b in (32, 256):
                                shapes.append(dict(block=b, fibres_per_thread=8, unroll=un, chunk=ch))
            for sh in shapes:
                ctx.set_tune(dim, **sh)
                ctx.set_coeffs(u)
                ctx.advect(dim, -1, s)
                assert np.array_equal(ctx.get_coeffs(), ref), (dim, sh)


def test_set_tune_rejects_shapes_not_built():
    with S.Context(_grid((3, 2, 2, 3, 2, 2)), 1, "mix_bf16") as ctx:   # cell records, lane groups
        assert ctx.info["record_slots"] == 64
        ctx.set_tune(0, block=256, fibres_per_thread=8, unroll=4, chunk=3)
        for dim, sh in [(0, dict(block=128, fibres_per_thread=8, unroll=1, chunk=0)),
                        (0, dict(block=128, fibres_per_thread=8, unroll=3, chunk=3)),
                        (1, dict(block=512, fibres_per_thread=8, unroll=1, chunk=2)),
                        (1, dict(block=256, fibres_per_thread=32, unroll=1, chunk=2)),
                        (1, dict(block=128, fibres_per_thread=4, unroll=1, chunk=2)),
                        (1, dict(block=128, fibres_per_thread=8, unroll=1, chunk=3))]:
            with pytest.raises(S.SlError) as e:
                ctx.set_tune(dim, **sh)
            assert e.value.status == S.SL_EINVAL
    with S.Context(_grid((4, 3, 5)), 3, "mix_bf16") as ctx:   # records without lane groups
        assert ctx.info["record_slots"] == 64
        with pytest.raises(S.SlError):
            ctx.set_tune(1, block=128, fibres_per_thread=8, unroll=1, chunk=2)
    with S.Context(_grid((4, 3, 3, 2)), 2, "mix_bf16") as ctx:
        for f in (1, 2, 5, 26):
            with pytest.raises(S.SlError) as e:
                ctx.set_tune(1, block=64, fibres_per_thread=f, chunk=2)
            assert e.value.status == S.SL_EINVAL
    with S.Context(_grid((8, 8)), 2, "mix_fp32") as ctx:
        for dim, sh in [(0, dict(block=512)), (0, dict(block=100)), (0, dict(block=128, fibres_per_thread=5)),
                        (1, dict(block=256, fibres_per_thread=1, unroll=1, chunk=8)),
                        (1, dict(block=128, fibres_per_thread=3, unroll=4, chunk=8)),
                        (1, dict(block=128, fibres_per_thread=1, unroll=1, chunk=0)),
                        (1, dict(block=128, fibres_per_thread=1, unroll=1, chunk=9)),
                        (1, dict(block=128, fibres_per_thread=3, pipeline=8, chunk=8)),
                        (0, dict(block=128, fibres_per_thread=1, pipeline=4)),
                        (0, dict(block=128, fibres_per_thread=1, unroll=2)),
                        (0, dict(block=128, fibres_per_thread=9, unroll=4)),
                        (1, dict(block=32, fibres_per_thread=1, pipeline=4, chunk=8)),
                        (1, dict(block=128, fibres_per_thread=1, unroll=1, chunk=8, max_blocks_per_sm=3)),
                        (1, dict(block=128, fibres_per_thread=1, pipeline=4, chunk=8, max_blocks_per_sm=5)),
                        (0, dict(block=128, fibres_per_thread=1, max_blocks_per_sm=5))]:
            with pytest.raises(S.SlError) as e:
                ctx.set_tune(dim, **sh)
            assert e.value.status == S.SL_EINVAL


def test_autotune_keeps_state_and_results():
    p = W.config3(n=10, steps=2)
    with S.Context(p.grid, p.k, "mix_fp32") as a, S.Context(p.grid, p.k, "mix_fp32") as b:
        for c in (a, b):
            c.project(p.nq, p.weights, p.params)
            c.set_fields(p.field_list())
        before = b.get_coeffs()
        b.autotune(2)
        assert np.array_equal(b.get_coeffs(), before)
        a.step("strang", p.dt, 2)
        b.step("strang", p.dt, 2)
        assert np.array_equal(a.get_coeffs(), b.get_coeffs())
        for d in range(4):
            t = b.get_tune(d)
            assert t["block"] >= 32


@pytest.mark.parametrize("storage", ["mix_bf16", "mix_fp16"])
@pytest.mark.parametrize("n,k", [((3, 4, 2, 3, 2), 1), ((4, 3, 5), 3), ((5, 2, 3, 2, 2, 2), 1),
                                 ((3, 4, 3, 2), 2), ((5, 3, 4), 2)])
def test_scaled_single_sweeps_every_fibre_split(storage, n, k):
    """Cells with more than 16 values are shared by several threads (a
    block-wide maximum for the scale); fewer are one thread's.  Both against
    the oracle applied to exactly the stored input; the FP64 mean row to
    rounding."""
    rng = np.random.default_rng(31)
    u = _rand(n, k, 32)
    with S.Context(_grid(n), k, storage) as ctx:
        for dim in range(len(n)):
            for sd in [-1, (dim + 1) % len(n)]:
                s = _shifts(rng, n, dim, sd)
                ctx.set_coeffs(u)
                stored = ctx.get_coeffs()
                ctx.advect(dim, sd, s)
                got = ctx.get_coeffs()
                ref = O.sweep(stored, n, k, dim, sd, s)
                assert O.rel_l2(got, ref, k, len(n)) <= 5e-3, (dim, sd)
                assert np.max(np.abs(got[:, 0] - ref[:, 0])) <= 1e-6 * np.max(np.abs(stored[:, 1:]))


@pytest.mark.parametrize("storage", ["mix_bf16", "mix_fp16"])
@pytest.mark.parametrize("n,k,slots", [((3, 2, 2, 3, 2, 2), 1, 64), ((3, 4, 2, 3, 2), 1, 32),
                                       ((4, 3, 5), 3, 64), ((4, 3, 3, 2), 2, 0)])
def test_record_layout_raw_planes(storage, n, k, slots):
    """Scaled shapes whose cells fill a record keep the higher coefficients
    in per-cell records: slot J is coefficient J, slot 0 and the padding are
    zero, and the raw planes round-trip."""
    u = _rand(n, k, 41)
    with S.Context(_grid(n), k, storage) as ctx:
        assert ctx.info["record_slots"] == slots
        ctx.set_coeffs(u)
        ctx.advect(0, -1, [0.3])
        ctx.advect(len(n) - 1, -1, [-1.7])
        want = ctx.get_coeffs()
        mean, hi, scale = S.sl_get_planes(ctx.handle)
        if slots:
            assert hi.shape == (int(np.prod(n)), slots)
            assert not hi[:, 0].any() and not hi[:, (k + 1) ** len(n):].any()
        # decode the raw planes on the host and compare
        x = hi.astype(np.uint32)
        if storage == "mix_bf16":
            vals = (x << 16).view(np.float32).astype(np.float64)
        else:
            vals = x.astype(np.uint16).view(np.float16).astype(np.float64)
        coef = vals[:, 1:(k + 1) ** len(n)] if slots else vals.T
        assert np.array_equal(coef * scale[:, None], want[:, 1:])
        assert np.array_equal(mean, want[:, 0])
        S.sl_set_planes(ctx.handle, mean, hi, scale)
        ctx.synchronize()
        assert np.array_equal(ctx.get_coeffs(), want)


@pytest.mark.parametrize("storage", ["fp64", "mix_fp32", "mix_bf16"])
def test_shift_edge_cases_match_oracle(storage):
    """Shifts at the edges of the split s = sigma + alpha, one per line:
    tiny negative shifts whose fractional part rounds to 1 (sigma + 1,
    alpha = 0: an exact copy), integers of both signs, shifts of many periods,
    alpha just below 1 and just above 0."""
    n = (10, 12)
    k = 2
    N = n[0]
    edge = [-1e-20, -2.0 ** -60, 1.0 - 2.0 ** -53, 3.0, -7.0, 1e6 + 0.37, -1e6 - 0.37, 0.5, 2.0 ** -40,
            N - 1e-15, -N + 1e-15, 2.5 * N]
    s = np.array(edge, dtype=float)
    u = _rand(n, k, 91)
    with S.Context(_grid(n), k, storage) as ctx:
        ctx.set_coeffs(u)
        stored = ctx.get_coeffs()
        ctx.advect(0, 1, s)
        got = ctx.get_coeffs()
    ref = O.sweep(stored, n, k, 0, 1, s)
    ncoef = (k + 1) ** 2
    G = got.reshape(n[1], n[0], ncoef)
    R = ref.reshape(n[1], n[0], ncoef)
    for line, sh in enumerate(edge):
        sig, alpha = O.shift_split(sh)
        if alpha == 0.0:   # exact copy: the stored values, rolled, bit for bit
            assert np.array_equal(G[line], np.roll(stored.reshape(n[1], n[0], ncoef)[line], sig, axis=0)), sh
        elif storage == "fp64":
            assert O.rel_max(G[line], R[line]) <= FP64_TOL, sh
        else:
            tol = 1e-6 if storage == "mix_fp32" else 1e-2
            assert np.sqrt(np.sum((G[line] - R[line]) ** 2)) <= tol * np.sqrt(np.sum(R[line] ** 2)), sh


def test_advect_graph_replay_matches_advect_calls():
    """A captured sequence of sweeps with fixed per-line shifts replays the
    same sweeps as the calls, and keeps its own copy of the shifts."""
    import torch
    n, k = (33, 5), 2
    rng = np.random.default_rng(17)
    u = _rand(n, k, 5)
    s = rng.uniform(-3, 3, size=n[1])
    st = torch.cuda.Stream()
    with S.Context(_grid(n), k, "mix_fp32", stream=st) as a, S.Context(_grid(n), k, "mix_fp32", stream=st) as b:
        a.set_coeffs(u)
        b.set_coeffs(u)
        for _ in range(5):
            a.advect(0, 1, s)
        b.graph_capture_advect(0, 1, s, 5)      # 5 sweeps: odd, two graphs
        b.advect(1, -1, [0.0])                  # an identity sweep (and other shifts) in between
        b.graph_launch()
        assert np.array_equal(a.get_coeffs(), b.get_coeffs())
        for _ in range(5):
            a.advect(0, 1, s)
        b.graph_launch()
        assert np.array_equal(a.get_coeffs(), b.get_coeffs())
        with pytest.raises(S.SlError):
            b.graph_capture_advect(0, 1, s[:3], 2)


def test_largest_grid_sampled_after_one_step():
    """The largest grid the library takes in 2D: 46340^2 = 2,147,395,600 cells
    (just below the 2^31 - 1 limit; k = 1, mixed FP32, 86 GB for the two
    copies of the state).  One Strang step against the oracle on the
    dependency cones of sampled cells, including the first and last cells,
    so that 32-bit cell indices and 64-bit plane offsets are exercised at
    their ends; mass conserved."""
    n = 46340
    p = W.config2(n=n, steps=1)
    g = p.grid
    assert g.cells < 2 ** 31 - 1
    rng = np.random.default_rng(7)
    cells = np.concatenate([[0, n - 1, g.cells - n, g.cells - 1], rng.integers(0, g.cells, 8)]).astype(np.int64)
    sched = O.schedule(g, "strang", p.dt, p.field_list())
    ref = O.sample_after(g, 1, p.nq, p.weights, p.params, sched, cells)
    with S.Context(g, 1, "mix_fp32") as ctx:
        ctx.project(p.nq, p.weights, p.params)
        ctx.set_fields(p.field_list())
        m0 = ctx.mass()
        ctx.step("strang", p.dt, 1)
        got = ctx.get_cells(cells)
        m1 = ctx.mass()
    for i in range(len(cells)):
        assert O.rel_l2(got[i:i + 1], ref[i:i + 1], 1, 2) <= 1e-5, cells[i]
    assert abs(m1 - m0) / abs(m0) <= MASS_TOL


@pytest.mark.parametrize("cfg", ["2d", "4d"])
@pytest.mark.parametrize("storage", ["fp64", "mix_fp32"])
def test_lie_splitting_matches_oracle(cfg, storage):
    """Lie splitting (x-dims then v-dims, each with dt) against the oracle."""
    p = W.config2(n=40, steps=5) if cfg == "2d" else W.config3(n=8, steps=2)
    u = O.project(p.grid, p.k, p.nq, p.weights, p.params)
    with S.Context(p.grid, p.k, storage) as ctx:
        ctx.project(p.nq, p.weights, p.params)
        ctx.set_fields(p.field_list())
        stored = ctx.get_coeffs()
        m0 = ctx.mass()
        ctx.step("lie", p.dt, p.steps)
        got = ctx.get_coeffs()
        drift = abs(ctx.mass() - m0) / abs(m0)
    ref = O.step(stored if storage != "fp64" else u, p.grid, p.k, "lie", p.dt, p.steps, p.field_list())
    if storage == "fp64":
        assert O.rel_max(got, ref) <= FP64_TOL
    else:
        assert O.rel_l2(got, ref, p.k, p.grid.ndim) <= 1e-5
    assert drift <= MASS_TOL


@pytest.mark.parametrize("storage,n,k", [("mix_fp32", (9, 6), 2), ("fp64", (7, 5, 3), 1),
                                         ("mix_bf16", (3, 2, 2, 3, 2, 2), 1), ("mix_fp16", (5, 4, 3), 2),
                                         ("fp32", (9, 6), 2), ("mix_fp32_d2", (7, 5, 3), 2),
                                         ("mix_fp32_d3", (6, 5), 3)])
def test_external_planes_give_the_same_results(storage, n, k):
    """A context over caller-owned planes (torch tensors) computes exactly
    what a context with library-owned state computes, and the current state
    is in the caller's memory."""
    import torch
    g = _grid(n)
    lay = S.sl_plane_layout(g, k, storage)
    bufs = []
    for _ in range(2):
        for key in ("mean_bytes", "hi_bytes", "scale_bytes"):
            nb = lay[key]
            # torch's allocator hands out 512-byte aligned blocks
            bufs.append(torch.zeros(max(nb, 1), dtype=torch.uint8, device="cuda") if nb else None)
    ptrs = [b.data_ptr() if b is not None else 0 for b in bufs]
    assert all(p % 256 == 0 for p in ptrs)
    u = _rand(n, k, 3)
    rng = np.random.default_rng(2)
    with S.Context(g, k, storage) as a, S.Context(g, k, storage, planes=ptrs) as b:
        for c in (a, b):
            c.set_coeffs(u)
        for dim in range(len(n)):
            s = _shifts(rng, n, dim, -1)
            a.advect(dim, -1, s)
            b.advect(dim, -1, s)
        assert np.array_equal(a.get_coeffs(), b.get_coeffs())
        cur = len(n) % 2                       # copy holding the state after len(n) sweeps
        if lay["mean_bytes"]:                  # the FP64 block starts with the cell means
            mean = bufs[3 * cur].view(torch.float64)[: int(np.prod(n))].cpu().numpy()
            assert np.array_equal(mean, b.get_coeffs()[:, 0])
        else:                                  # the all-FP32 store: the means are FP32 plane 0
            mean = bufs[3 * cur + 1].view(torch.float32)[: int(np.prod(n))].cpu().numpy()
            assert np.array_equal(mean.astype(np.float64), b.get_coeffs()[:, 0])
    del bufs


def test_shift_tables_are_sized_by_the_other_dimensions():
    """A sweep's shift classes follow one coordinate orthogonal to it, so the
    table of dimension m holds as many classes as the largest other extent
    (one in 1D): a 1D context of 2^22 cells at k = 3 allocates little beyond
    its two copies of the state (a table per cell would add 1.7 GB), and a 2D
    one tables of a line's length only."""
    g = _grid((1 << 22,))
    with S.Context(g, 3, "fp64") as ctx:
        info = ctx.info
        assert info["alloc_bytes"] <= 2 * info["state_bytes"] + (4 << 20)
    g2 = _grid((1 << 12, 1 << 10), pair=(1, -1))
    with S.Context(g2, 2, "mix_fp32") as ctx:
        info = ctx.info
        assert info["alloc_bytes"] <= 2 * info["state_bytes"] + (8 << 20)


@pytest.mark.parametrize("k", [1, 2])
def test_fibre_groups_side_by_side_over_many_tiles(k):
    """In the 2D mixed store the unit-stride sweep puts the fibre groups side by
    side in the launch order and loops over tiles when there are more than
    65535 of them (4096 x 1040 cells in blocks of 64 threads: 66 560 tiles).
    One fibre per thread that way must give the same bits as the whole cell per
    thread (one group, tiles in x)."""
    n = (4096, 1040)
    g = _grid(n)
    u = _rand(n, k, 23)
    s = np.random.default_rng(24).uniform(-3.0 * n[0], 3.0 * n[0], size=n[1])
    with S.Context(g, k, "mix_fp32") as ctx:
        outs = []
        for ft in (1, k + 1):
            ctx.set_tune(0, block=64, fibres_per_thread=ft)
            ctx.set_coeffs(u)
            ctx.advect(0, 1, s)
            outs.append(ctx.get_coeffs())
        assert np.array_equal(outs[0], outs[1])
        # and the sampled cells against the oracle on their own lines
        rows = [0, 517, n[1] - 1]
        for j in rows:
            line = u[j * n[0]:(j + 1) * n[0]]
            ref = O.sweep(ctx_stored(line, "mix_fp32"), [n[0], 1], k, 0, 1, [s[j]])
            got = outs[0][j * n[0]:(j + 1) * n[0]]
            assert O.rel_l2(got, ref, k, 2) <= 1e-6, j


@pytest.mark.parametrize("n,k", [(1024, 2), (1000, 3), (37, 1), (5, 0), (2048, 2)])
def test_one_launch_1d_graph_matches_advect_calls_bit_for_bit(n, k):
    """A captured advection of a short 1D line of the FP64 store runs every
    step in one thread-block cluster launch, each step building its matrices
    in the kernel: it must give the same bits as the same number of sl_advect
    calls (a table build and a sweep each), for shifts with and without a
    fractional part, negative ones, shifts of more than the line, and an odd
    number of steps (two graphs, one per buffer parity)."""
    import torch
    g = _grid((n,))
    u = _rand((n,), k, 31)
    st = torch.cuda.Stream()
    for s, steps in ((0.37, 100), (-2.75, 7), (3.0, 4), (2.5 * n + 0.4, 3)):
        with S.Context(g, k, "fp64", stream=st) as a, S.Context(g, k, "fp64", stream=st) as b:
            a.set_coeffs(u)
            b.set_coeffs(u)
            for _ in range(steps):
                a.advect(0, -1, [s])
            b.graph_capture_advect(0, -1, [s], steps)
            b.graph_launch()
            assert np.array_equal(a.get_coeffs(), b.get_coeffs()), (s, steps)
            b.graph_launch()
            for _ in range(steps):
                a.advect(0, -1, [s])
            assert np.array_equal(a.get_coeffs(), b.get_coeffs()), (s, steps)
    # against the oracle: the first configuration's 100 steps
    ref = u
    for _ in range(100):
        ref = O.sweep(ref, [n], k, 0, -1, [0.37])
    with S.Context(g, k, "fp64", stream=st) as b:
        b.set_coeffs(u)
        b.graph_capture_advect(0, -1, [0.37], 100)
        b.graph_launch()
        assert O.rel_max(b.get_coeffs(), ref) <= FP64_TOL


@pytest.mark.parametrize("storage,tol", [("fp64", FP64_TOL), ("mix_fp32", MIX_TOL)])
def test_fields_changed_between_steps_are_used(storage, tol):
    """Every split step builds its dimensions' shift tables from the fields as
    they are at that step (the v-tables on a side stream, joined before the
    v-sweeps): a step after sl_set_fields uses the new field.  4D, k = 2, two
    Strang steps with the default field, two with another one, against the
    oracle taking the same fields."""
    p = W.config3(n=8, steps=2)
    f1 = p.field_list()
    f2 = [-3.0 * f + 0.05 for f in f1]
    u0 = O.project(p.grid, p.k, p.nq, p.weights, p.params)
    ref = O.step(u0, p.grid, p.k, "strang", p.dt, 2, f1)
    ref = O.step(ref, p.grid, p.k, "strang", p.dt, 2, f2)
    with S.Context(p.grid, p.k, storage) as ctx:
        ctx.project(p.nq, p.weights, p.params)
        ctx.set_fields(f1)
        ctx.step("strang", p.dt, 2)
        ctx.set_fields(f2)
        ctx.step("strang", p.dt, 2)
        got = ctx.get_coeffs()
    if storage == "fp64":
        assert O.rel_max(got, ref) <= tol
    else:
        assert O.rel_l2(got, ref, p.k, 4) <= tol


@pytest.mark.parametrize("nv", [8192, 9001])
def test_table_of_many_classes(nv):
    """A table of up to 8192 classes is built one thread per matrix entry,
    a larger one one thread per class: both against the oracle (FP64 store,
    4 x nv cells, k = 2, per-line shifts from the orthogonal coordinate)."""
    n = (4, nv)
    k = 2
    u = _rand(n, k, 41)
    s = np.random.default_rng(42).uniform(-9.0, 9.0, size=nv)
    with S.Context(_grid(n), k, "fp64") as ctx:
        ctx.set_coeffs(u)
        ctx.advect(0, 1, s)
        got = ctx.get_coeffs()
    ref = O.sweep(u, n, k, 0, 1, s)
    assert O.rel_max(got, ref) <= FP64_TOL
