"""Failure detection and recovery on the GPU, without a GPU fault: simulated
allocation failures (every allocation the library makes, one at a time),
guard-band canaries after sweeps in every store and launch form, and
checkpoint/resume continuing bit for bit."""
import numpy as np
import pytest

import paper_1603_07008_gb300 as S
from paper_1603_07008_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _free():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _session(p, store):
    """A context's life through the calls that allocate: create, project
    (workspace), set/get (staging), self-consistent field or nodal tables."""
    with S.Context(p.grid, p.k, store) as ctx:
        ctx.project(p.nq, p.weights, p.params)
        u = ctx.get_coeffs()
        ctx.set_coeffs(u)
        ctx.set_nodal_velocity(True)
        ctx.set_poisson(True)
        ctx.set_fields(p.field_list())
        ctx.step("strang", p.dt, 1)
        return ctx.mass()


@pytest.mark.parametrize("store", ["fp64", "mix_fp32"])
def test_every_allocation_failure_is_reported_and_leaks_nothing(store):
    p = W.config2(n=32, steps=1)
    ref = _session(p, store)
    free0 = _free()
    n = 1
    while True:
        S.sl_debug_fail_alloc(n)
        try:
            m = _session(p, store)
        except S.SlError as e:
            assert e.status == S.SL_ENOMEM, (n, str(e))
            n += 1
            continue
        finally:
            S.sl_debug_fail_alloc(0)
        assert m == ref          # the hook was past the last allocation: the session ran through
        break
    assert n >= 5                # create (state, pinned mass), workspace, staging, field, nodal tables
    assert abs(_free() - free0) <= 4 << 20


def test_batch_allocation_failures_clean_up():
    probs = W.config4(nprob=6, nmin=16, nmax=64)
    grids, ks = [q.grid for q in probs], [q.k for q in probs]
    free0 = _free()
    failures = 0
    for n in range(1, 40):
        S.sl_debug_fail_alloc(n)
        try:
            b = S.Batch(grids, ks, "mix_fp32")
        except S.SlError as e:
            assert e.status == S.SL_ENOMEM, str(e)
            failures += 1
            continue
        finally:
            S.sl_debug_fail_alloc(0)
        b.close()
        break
    assert failures >= 6 * 2
    assert abs(_free() - free0) <= 4 << 20


CASES = [("fp64", (9, 7), 2, (1, -1)), ("mix_fp32", (12, 5, 3), 2, (-1, -1, -1)),
         ("mix_bf16", (5, 3, 2, 3), 1, (2, 3, -1, -1)), ("mix_fp16", (3, 2, 2, 3, 2, 2), 1, (3, 4, 5, -1, -1, -1)),
         ("fp32", (10, 6), 3, (1, -1)), ("mix_fp32_d2", (7, 4, 3), 2, (2, -1, -1)), ("mix_fp32_d3", (9, 5), 3, (1, -1))]


@pytest.mark.parametrize("store,n,k,pair", CASES)
def test_guards_hold_after_sweeps_in_every_form(store, n, k, pair):
    """Every dimension swept with several launch shapes (the autotuner's
    candidates included), with split steps and nodal x-sweeps where the store
    takes them: no byte past any array or plane may change."""
    d = len(n)
    g = W.Grid(n=n, lo=(0.0,) * d, hi=(1.0,) * d, pair=pair)
    u = W.random_coefficients(int(np.prod(n)), k, d, 41)
    with S.Context(g, k, store) as ctx:
        assert ctx.check_guards() == 0
        ctx.set_coeffs(u)
        rng = np.random.default_rng(42)
        for dim in range(d):
            sd = (dim + 1) % d
            ctx.advect(dim, sd, rng.uniform(-3 * n[dim], 3 * n[dim], size=n[sd]))
        ctx.autotune(1)
        if any(q >= 0 for q in pair):
            nf = sum(n[m] for m in range(d) if pair[m] >= 0)
            ctx.set_fields(rng.uniform(-1, 1, size=nf))
            ctx.step("lie", 0.3, 2)
            if store in ("fp64", "mix_fp32"):
                ctx.set_nodal_velocity(True)
                ctx.step("strang", 0.3, 2)
        ctx.mass()
        ctx.get_coeffs()
        assert ctx.check_guards() == 0
        # the check sees a changed byte
        S.sl_debug_corrupt_guard(ctx.handle)
        assert ctx.check_guards() == 1


@pytest.mark.parametrize("store", ["fp64", "mix_fp32", "mix_bf16", "fp32", "mix_fp32_d2"])
def test_checkpoint_resume_is_bit_exact(store, tmp_path):
    p = W.config2(n=24, steps=1)
    k = 1 if store == "mix_bf16" else 2
    with S.Context(p.grid, k, store) as a:
        a.project(p.nq, p.weights, p.params)
        a.set_fields(p.field_list())
        a.step("strang", p.dt, 3)
        S.save_checkpoint(a, tmp_path / "c.npz", step=3, time=3 * p.dt, extra={"run": "t"})
        a.step("strang", p.dt, 4)
        want = a.get_coeffs()
    b, meta = S.load_checkpoint(tmp_path / "c.npz")
    with b:
        assert meta["step"] == 3 and meta["extra"] == {"run": "t"}
        b.set_fields(p.field_list())
        b.step("strang", p.dt, 4)
        assert np.array_equal(b.get_coeffs(), want)


def test_tune_cache_reuses_the_autotuners_choice(tmp_path):
    p = W.config3(n=12, steps=1)
    path = tmp_path / "tunes.json"
    with S.Context(p.grid, p.k, "mix_fp32") as a:
        assert S.autotune_cached(a, path) is False
        first = [a.get_tune(d) for d in range(4)]
    with S.Context(p.grid, p.k, "mix_fp32") as b:
        assert S.autotune_cached(b, path) is True
        assert [b.get_tune(d) for d in range(4)] == first
