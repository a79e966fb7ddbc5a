"""Parity of the nodal-in-velocity x-sweep (sl_advect_nodal, and sl_step after
sl_set_nodal_velocity) with the oracle's sweep_nodal, through the C ABI.

Tolerances: FP64 store max-relative <= 1e-12; mixed FP32 store relative
function-space L2 <= 1e-6 for one sweep against the oracle applied to the
stored (rounded) input and <= 1e-5 after split steps against the FP64 oracle;
mass drift <= 1e-13 after 1000 steps in both stores.
"""
import numpy as np
import pytest

import oracle as O
import paper_1603_07008_gb300 as S
from paper_1603_07008_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# (extents, pair, v-box): x-dimension 0 or 1, with and without unpaired dimensions
XV = [((7, 5), (1, -1)), ((5, 6), (-1, 0)), ((4, 3, 5), (2, -1, -1)), ((3, 4, 2, 3), (2, 3, -1, -1)),
      ((6, 2, 4), (-1, 2, -1))]


def _grid(n, pair):
    d = len(n)
    lo = tuple(-3.0 if pair.count(m) else 0.0 for m in range(d))    # v-dimensions span [-3, 2)
    hi = tuple(2.0 if pair.count(m) else 1.0 for m in range(d))
    return W.Grid(n=tuple(n), lo=lo, hi=hi, pair=tuple(pair))


def _rand(n, k, seed):
    return W.random_coefficients(int(np.prod(n)), k, len(n), seed)


def _xdims(pair):
    return [m for m, p in enumerate(pair) if p >= 0]


@pytest.mark.parametrize("n,pair", XV)
@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_fp64_nodal_sweeps_match_oracle(n, pair, k):
    if (k + 1) ** len(n) > 512:
        pytest.skip("coefficient count covered by smaller shapes")
    g = _grid(n, pair)
    u = _rand(n, k, 31)
    with S.Context(g, k, "fp64") as ctx:
        for dim in _xdims(pair):
            for tau in (0.37, -1.3, 2.9):
                ctx.set_coeffs(u)
                ctx.advect_nodal(dim, tau)
                got = ctx.get_coeffs()
                ref = O.sweep_nodal(u, g, k, dim, tau)
                assert O.rel_max(got, ref) <= 1e-12, (dim, tau)


@pytest.mark.parametrize("n,pair", XV)
@pytest.mark.parametrize("k", [1, 2, 3])
def test_mixed_nodal_sweeps_match_oracle(n, pair, k):
    if (k + 1) ** len(n) > 512:
        pytest.skip("coefficient count covered by smaller shapes")
    g = _grid(n, pair)
    u = _rand(n, k, 32)
    stored = O.round_storage(u, k, len(n), 1)
    with S.Context(g, k, "mix_fp32") as ctx:
        for dim in _xdims(pair):
            for tau in (0.37, -1.3):
                ctx.set_coeffs(u)
                ctx.advect_nodal(dim, tau)
                got = ctx.get_coeffs()
                ref = O.sweep_nodal(stored, g, k, dim, tau)
                assert O.rel_l2(got, ref, k, len(n)) <= 1e-6, (dim, tau)
                # the mean gets the FP32 parts' rounding only
                assert np.max(np.abs(got[:, 0] - ref[:, 0])) <= 1e-6 * np.max(np.abs(stored[:, 1:]))


@pytest.mark.parametrize("store", ["fp64", "mix_fp32"])
def test_degree_zero_nodal_is_the_centre_sweep(store):
    """With one node per v-cell (k = 0) the node is the cell centre: the nodal
    sweep is the plain x-sweep with the centre velocity."""
    n, pair = (9, 6), (1, -1)
    g = _grid(n, pair)
    u = _rand(n, 0, 33)
    tau = 0.71
    hv, hx = 5.0 / 6, 1.0 / 9
    v = -3.0 + (np.arange(6) + 0.5) * hv
    with S.Context(g, 0, store) as a, S.Context(g, 0, store) as b:
        a.set_coeffs(u)
        b.set_coeffs(u)
        a.advect_nodal(0, tau)
        b.advect(0, 1, v * tau / hx)
        assert np.max(np.abs(a.get_coeffs() - b.get_coeffs())) <= 1e-14 * np.max(np.abs(u))


@pytest.mark.parametrize("store", ["fp64", "mix_fp32"])
@pytest.mark.parametrize("cfg", ["2d", "4d"])
def test_nodal_strang_steps_match_oracle(store, cfg):
    p = W.config2(n=32, steps=5) if cfg == "2d" else W.config3(n=6, steps=2)
    u0 = O.project(p.grid, p.k, p.nq, p.weights, p.params)
    ref = O.step(u0, p.grid, p.k, "strang", p.dt, p.steps, p.field_list(), nodal_v=True)
    with S.Context(p.grid, p.k, store) as ctx:
        ctx.project(p.nq, p.weights, p.params)
        ctx.set_fields(p.field_list())
        ctx.set_nodal_velocity(True)
        m0 = ctx.mass()
        ctx.step("strang", p.dt, p.steps)
        got = ctx.get_coeffs()
        drift = abs(ctx.mass() - m0) / abs(m0)
    if store == "fp64":
        assert O.rel_max(got, ref) <= 1e-12
    else:
        assert O.rel_l2(got, ref, p.k, p.grid.ndim) <= 1e-5
    assert drift <= 1e-13


@pytest.mark.parametrize("store", ["fp64", "mix_fp32"])
def test_nodal_mass_drift_1000_steps(store):
    p = W.config2(n=64, steps=1000)
    with S.Context(p.grid, p.k, store) as ctx:
        ctx.project(p.nq, p.weights, p.params)
        ctx.set_fields(p.field_list())
        ctx.set_nodal_velocity(True)
        m0 = ctx.mass()
        ctx.step("strang", p.dt, 1000)
        m1 = ctx.mass()
    assert abs(m1 - m0) / abs(m0) <= 1e-13


def test_nodal_graph_replay_matches_step():
    import torch
    p = W.config2(n=24, steps=6)
    st = torch.cuda.Stream()
    with S.Context(p.grid, p.k, "mix_fp32", stream=st) as a, \
            S.Context(p.grid, p.k, "mix_fp32", stream=st) as b:
        for c in (a, b):
            c.project(p.nq, p.weights, p.params)
            c.set_fields(p.field_list())
            c.set_nodal_velocity(True)
        a.step("strang", p.dt, 6)
        b.graph_capture("strang", p.dt, 3)
        b.graph_launch()
        b.graph_launch()
        assert np.array_equal(a.get_coeffs(), b.get_coeffs())


def test_nodal_free_streaming_beats_the_centre_velocity():
    """Free streaming over T = 1/2 (8 x-sweeps, 32 x 32 cells, k = 2): the
    nodal sweep on the GPU is as close to the exact solution as the oracle's
    and far closer than one velocity per v-cell."""
    import math
    k, N, T, steps = 2, 32, 0.5, 8
    g = W.Grid(n=(N, N), lo=(0.0, -1.0), hi=(1.0, 1.0), pair=(1, -1))
    w = np.array([1.0, 0.5, 0.5])
    terms = lambda t: np.array([[[0, 0, 0, 0], [1, 0, 0, 0]],
                                [[0, 0, 2 * math.pi, 0], [1, 0, 2 * math.pi * t, 0]],
                                [[0, 0, 2 * math.pi, -math.pi / 2], [1, 0, 2 * math.pi * t, -math.pi / 2]]],
                               dtype=float)
    ue = O.project(g, k, k + 3, w, terms(T))
    v = -1.0 + (np.arange(N) + 0.5) * (2.0 / N)
    with S.Context(g, k, "fp64") as a, S.Context(g, k, "fp64") as b:
        a.project(k + 3, w, terms(0.0))
        b.project(k + 3, w, terms(0.0))
        for _ in range(steps):
            a.advect_nodal(0, T / steps)
            b.advect(0, 1, v * (T / steps) * N)
        en = O.rel_l2(a.get_coeffs(), ue, k, 2)
        ec = O.rel_l2(b.get_coeffs(), ue, k, 2)
    assert en < 1e-5 and en < ec / 100, (en, ec)


def test_nodal_rejections():
    g1 = W.Grid(n=(8,), lo=(0.0,), hi=(1.0,), pair=(-1,))
    with S.Context(g1, 1, "fp64") as c:
        with pytest.raises(S.SlError) as e:
            c.set_nodal_velocity(True)
        assert e.value.status == S.SL_EINVAL
    g = _grid((6, 5), (1, -1))
    for store in ("mix_bf16", "fp32", "mix_fp32_d2"):
        with S.Context(g, 2, store) as c:
            with pytest.raises(S.SlError) as e:
                c.set_nodal_velocity(True)
            assert e.value.status == S.SL_ENOTSUP
    with S.Context(g, 2, "fp64") as c:
        with pytest.raises(S.SlError):
            c.advect_nodal(1, 0.3)          # dimension 1 is the v-dimension
        with pytest.raises(S.SlError):
            c.advect_nodal(0, float("nan"))


def test_nodal_full_size_sampled_after_one_x_sweep():
    """4D 64^4, k = 2, mixed store (the bench's nodal configuration): one
    nodal x-sweep along dimension 0 over dt / 2, sampled target cells against
    the oracle on a small (x, v) problem cut out around each: the x-cells that
    the target's nodes read, one v-cell with the same velocity range, and the
    nine fibres of the other two indices one by one."""
    p = W.config3(n=64, steps=1)
    g, k, o = p.grid, p.k, p.k + 1
    n = g.n
    hx = (g.hi[0] - g.lo[0]) / n[0]
    hv = (g.hi[2] - g.lo[2]) / n[2]
    tau = 0.5 * p.dt
    eta, _ = O.gauss_legendre(o)
    rng = np.random.default_rng(21)
    cells = rng.integers(0, int(np.prod(n)), size=40).astype(np.int64)
    cells = np.concatenate([cells, [0, int(np.prod(n)) - 1]])
    with S.Context(g, k, "mix_fp32") as ctx:
        ctx.project(p.nq, p.weights, p.params)
        ctx.set_fields(p.field_list())
        plans, need = [], []
        for c in cells:
            i0, i1, i2, i3 = c % 64, (c // 64) % 64, (c // 4096) % 64, c // 262144
            sig = [O.shift_split((g.lo[2] + (i2 + 0.5 + 0.5 * e) * hv) * tau / hx)[0] for e in eta]
            dlo, dhi = min(min(sig), 0), max(max(sig) + 1, 0)
            xs = [(i0 - d) % 64 for d in range(dhi, dlo - 1, -1)]       # mini index 0 .. W-1
            win = [x + 64 * (i1 + 64 * (i2 + 64 * i3)) for x in xs]
            plans.append((i2, dhi, len(win)))
            need.extend(win)
        src = ctx.get_cells(np.array(need, dtype=np.int64))
        ctx.advect_nodal(0, tau)
        got = ctx.get_cells(cells)
    ref = np.empty_like(got)
    pos = 0
    for r, (j, dhi, wlen) in enumerate(plans):
        block = src[pos:pos + wlen]
        pos += wlen
        mini = W.Grid(n=(wlen, 1), lo=(0.0, g.lo[2] + j * hv), hi=(wlen * hx, g.lo[2] + (j + 1) * hv), pair=(1, -1))
        for j1 in range(o):
            for j3 in range(o):
                idx = [j0 + o * j1 + o * o * j2 + o ** 3 * j3 for j2 in range(o) for j0 in range(o)]
                u2 = block[:, idx]                        # mini coefficient j0 + o j2
                out = O.sweep_nodal(u2, mini, k, 0, tau)
                ref[r, idx] = out[dhi]
    assert O.rel_l2(got, ref, k, 4) <= 1e-6
    assert np.max(np.abs(got[:, 0] - ref[:, 0])) <= 1e-6 * np.max(np.abs(ref[:, 1:]))


def _swap01(u, n, k):
    """The coefficients of a 4D state with dimensions 0 and 1 exchanged (cells
    and coefficient indices), in the layout of the swapped grid."""
    o = k + 1
    t = u.reshape(n[3], n[2], n[1], n[0], o, o, o, o)    # axes i3 i2 i1 i0 j3 j2 j1 j0
    return np.ascontiguousarray(t.transpose(0, 1, 3, 2, 4, 5, 7, 6)).reshape(u.shape)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_nodal_runs_match_one_target_per_thread_bit_for_bit(k):
    """The FP32 fibres of the mixed store take runs of consecutive targets
    per thread: four along x-dimension 1 (lanes on neighbouring x-lines), two
    along x-dimension 0 (lanes on neighbouring runs of one line), and one
    target at a time where the nodes of a v-cell do not share sigma.  Every
    form keeps the same order of every sum, so the sweep along dimension 1
    equals, bit for bit, the sweep along dimension 0 of the state with
    dimensions 0 and 1 exchanged: runs cut by the line end (9 = 4 + 4 + 1 and
    2 + 2 + 2 + 2 + 1), wrapped sources, and v-cells whose nodes do and do
    not share sigma."""
    n = (7, 9, 5, 4)
    g = W.Grid(n=n, lo=(0.0, 0.0, -3.0, -3.0), hi=(1.0, 2.0, 2.0, 2.0), pair=(2, 3, -1, -1))
    ns = (9, 7, 5, 4)
    gs = W.Grid(n=ns, lo=(0.0, 0.0, -3.0, -3.0), hi=(2.0, 1.0, 2.0, 2.0), pair=(3, 2, -1, -1))
    u = _rand(n, k, 60 + k)
    us = _swap01(u, n, k)
    with S.Context(g, k, "mix_fp32") as a, S.Context(gs, k, "mix_fp32") as b:
        for tau in (0.05, 0.37, -1.3, 2.9):
            a.set_coeffs(u)
            b.set_coeffs(us)
            a.advect_nodal(1, tau)
            b.advect_nodal(0, tau)
            assert np.array_equal(_swap01(a.get_coeffs(), n, k), b.get_coeffs()), tau


def _nodal_windows(g, k, xdim, tau, cells):
    """For each sampled target cell of a 4D grid: the cells along x that its
    nodes read in a nodal x-sweep over tau (a window around it), and the plan
    (v-cell, target position in the window, window length)."""
    n = g.n
    o = k + 1
    vdim = g.pair[xdim]
    st = [1, n[0], n[0] * n[1], n[0] * n[1] * n[2]]
    hx = (g.hi[xdim] - g.lo[xdim]) / n[xdim]
    hv = (g.hi[vdim] - g.lo[vdim]) / n[vdim]
    eta, _ = O.gauss_legendre(o)
    plans, need = [], []
    for c in cells:
        ix, j = (c // st[xdim]) % n[xdim], (c // st[vdim]) % n[vdim]
        sig = [O.shift_split((g.lo[vdim] + (j + 0.5 + 0.5 * e) * hv) * tau / hx)[0] for e in eta]
        dlo, dhi = min(min(sig), 0), max(max(sig) + 1, 0)
        base = c - ix * st[xdim]
        win = [base + ((ix - d) % n[xdim]) * st[xdim] for d in range(dhi, dlo - 1, -1)]
        plans.append((j, dhi, len(win)))
        need.extend(win)
    return plans, np.array(need, dtype=np.int64)


def _nodal_sampled_reference(g, k, xdim, tau, plans, src):
    """The oracle's nodal x-sweep at the sampled targets, each on a cut-out
    (x, v) problem: its window along x, one v-cell of the same velocity range,
    and the o^2 fibres of the other two indices one by one."""
    o = k + 1
    vdim = g.pair[xdim]
    others = [m for m in range(4) if m not in (xdim, vdim)]
    hx = (g.hi[xdim] - g.lo[xdim]) / g.n[xdim]
    hv = (g.hi[vdim] - g.lo[vdim]) / g.n[vdim]
    ref = np.empty((len(plans), o ** 4))
    pos = 0
    for r, (j, dhi, wlen) in enumerate(plans):
        block = src[pos:pos + wlen]
        pos += wlen
        mini = W.Grid(n=(wlen, 1), lo=(0.0, g.lo[vdim] + j * hv), hi=(wlen * hx, g.lo[vdim] + (j + 1) * hv),
                      pair=(1, -1))
        for ja in range(o):
            for jb in range(o):
                idx = []
                for jv in range(o):
                    for jx in range(o):       # mini coefficient jx + o jv
                        jj = [0, 0, 0, 0]
                        jj[xdim], jj[vdim], jj[others[0]], jj[others[1]] = jx, jv, ja, jb
                        idx.append(jj[0] + o * jj[1] + o * o * jj[2] + o ** 3 * jj[3])
                ref[r, idx] = O.sweep_nodal(block[:, idx], mini, k, 0, tau)[dhi]
    return ref


@pytest.mark.parametrize("xdim", [0, 1])
def test_nodal_sampled_with_64_bit_plane_offsets(xdim):
    """4D 64 x 64 x 96 x 72, k = 2, mixed store: 80 FP32 planes of 28.3M
    cells, more than 2^31 elements, so both nodal forms (one target per thread
    along dimension 0, runs along dimension 1) address the FP32 block with
    64-bit offsets.  One x-sweep over dt / 2; sampled targets against the
    oracle on cut-out (x, v) problems."""
    p = W.config3(n=64, steps=1)
    n = (64, 64, 96, 72)
    g = W.Grid(n=n, lo=p.grid.lo, hi=p.grid.hi, pair=p.grid.pair)
    k, tau = p.k, 0.5 * p.dt
    rng = np.random.default_rng(70 + xdim)
    cells = np.concatenate([rng.integers(0, int(np.prod(n)), size=30), [0, int(np.prod(n)) - 1]]).astype(np.int64)
    plans, need = _nodal_windows(g, k, xdim, tau, cells)
    with S.Context(g, k, "mix_fp32") as ctx:
        assert ctx.info["plane_stride"] * (ctx.info["ncoef"] - 1) >= 2 ** 31
        ctx.project(p.nq, p.weights, p.params)
        src = ctx.get_cells(need)
        ctx.advect_nodal(xdim, tau)
        got = ctx.get_cells(cells)
    ref = _nodal_sampled_reference(g, k, xdim, tau, plans, src)
    assert O.rel_l2(got, ref, k, 4) <= 1e-6
    assert np.max(np.abs(got[:, 0] - ref[:, 0])) <= 1e-6 * np.max(np.abs(ref[:, 1:]))
