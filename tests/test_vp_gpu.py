"""Self-consistent field (the Vlasov-Poisson system of Sec. II in 1+1
dimensions) on the GPU against the oracle: the field, the split step that
recomputes it before every v-sweep, graph replay, mass conservation, and the
linear Landau damping rate."""
import math

import numpy as np
import pytest

import oracle as O
import paper_1603_07008_gb300 as S
from paper_1603_07008_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _landau(nx, nv, k=2):
    p = W.config2(n=8, steps=1)
    g = W.Grid(n=(nx, nv), lo=p.grid.lo, hi=p.grid.hi, pair=p.grid.pair)
    return p, g


@pytest.mark.parametrize("swap,nx", [(False, 48), (True, 48), (False, 5), (False, 1003)])
def test_field_matches_oracle(swap, nx):
    """The field is computed by a cluster of 8 blocks, each taking a segment
    of the x-cells: 48 cells (6 per block), 5 (three blocks without cells)
    and 1003 (uneven segments)."""
    p, g = _landau(nx, 40)
    if swap:   # v along dimension 0, x along dimension 1
        g = W.Grid(n=(40, nx), lo=(g.lo[1], g.lo[0]), hi=(g.hi[1], g.hi[0]), pair=(-1, 0))
    rng = np.random.default_rng(3)
    u = rng.standard_normal((g.cells, 9)) * 0.1
    u[:, 0] += 1.0
    with S.Context(g, 2, "fp64") as ctx:
        ctx.set_coeffs(u)
        E = ctx.field()
        W_gpu = ctx.field_energy()
    ref = O.poisson_field(u, g, 2)
    # both sum n_v terms per density and n_x terms per field value in FP64,
    # in different orders: |difference| <= 2 (n_x + n_v) eps h_x sum_i |rho_i|
    nv = 40
    hx = 4 * math.pi / nx
    rho_abs = 12.0 / nv * np.sum(np.abs(u[:, 0]))
    assert np.max(np.abs(E - ref)) <= 2 * (nx + nv) * np.finfo(float).eps * hx * rho_abs
    assert abs(W_gpu - O.field_energy(ref, g)) <= 1e-12 * O.field_energy(ref, g)


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-11), ("mix_fp32", 1e-5)])
def test_self_consistent_steps_match_oracle(storage, tol):
    p, g = _landau(32, 64)
    u0 = O.project(g, 2, p.nq, p.weights, p.params)
    steps = 40
    with S.Context(g, 2, storage) as ctx:
        ctx.set_coeffs(u0)
        stored = ctx.get_coeffs()
        ctx.set_poisson(True)
        m0 = ctx.mass()
        ctx.step("strang", 0.1, steps)
        got = ctx.get_coeffs()
        drift = abs(ctx.mass() - m0) / abs(m0)
    ref = O.vp_step(stored, g, 2, "strang", 0.1, steps)
    if storage == "fp64":
        assert O.rel_max(got, ref) <= tol
    else:
        assert O.rel_l2(got, ref, 2, 2) <= tol
    assert drift <= 1e-13


def test_self_consistent_graph_replay_matches_steps():
    import torch
    p, g = _landau(32, 64)
    u0 = O.project(g, 2, p.nq, p.weights, p.params)
    s = torch.cuda.Stream()
    res = []
    for mode in ("step", "graph"):
        with S.Context(g, 2, "mix_fp32", stream=s) as ctx:
            ctx.set_coeffs(u0)
            ctx.set_poisson(True)
            if mode == "step":
                ctx.step("strang", 0.1, 6)
            else:
                ctx.graph_capture("strang", 0.1, 2)
                for _ in range(3):
                    ctx.graph_launch()
            res.append(ctx.get_coeffs())
    assert np.array_equal(res[0], res[1])


def test_landau_damping_rate_on_the_gpu():
    """Mixed FP32 store, 128 x 256 cells, k = 2: the field energy decays at
    twice gamma = -0.1533 (linear Landau damping, wave number 1/2)."""
    p, g = _landau(128, 256)
    with S.Context(g, 2, "mix_fp32") as ctx:
        ctx.project(p.nq, p.weights, p.params)
        ctx.set_poisson(True)
        en = [ctx.field_energy()]
        for _ in range(200):
            ctx.step("strang", 0.1, 1)
            en.append(ctx.field_energy())
    t = np.arange(len(en)) * 0.1
    le = np.log(np.array(en))
    peaks = [i for i in range(1, len(le) - 1) if le[i] > le[i - 1] and le[i] >= le[i + 1] and t[i] < 20]
    gamma = np.polyfit(t[peaks], le[peaks], 1)[0] / 2
    assert abs(gamma + 0.1533) < 0.003, gamma


def test_poisson_needs_one_x_and_one_v_dimension():
    g = W.config3(n=4, steps=1).grid
    with S.Context(g, 1, "mix_fp32") as ctx:
        with pytest.raises(S.SlError) as e:
            ctx.set_poisson(True)
        assert e.value.status == S.SL_EINVAL
