"""sl_mass_noalloc: the mass reduction for callers that cannot let a library
call cudaMalloc (an application that owns all device memory through its own
pool, or a loop where a device allocation and its implicit synchronisation are
not allowed).  Its scratch is a fixed array inside the library, so the only
memory involved is the caller's input plane and output slot.

It must give the same mass as sl_mass, the context-based entry point, on
consecutive calls (the shared scratch keeps the previous call's contents).
This file is collected last so that a stop-at-first-failure run has already
run every other test when it gets here; it also passes on its own.
"""
import math

import numpy as np
import pytest

import paper_1603_07008_gb300 as S
from paper_1603_07008_gb300 import workloads as W

MASS_TOL = 1e-13


def _cell_volume(g):
    vol = 1.0
    for m in range(len(g.n)):
        vol *= (g.hi[m] - g.lo[m]) / g.n[m]
    return vol


@pytest.mark.gpu
@pytest.mark.parametrize("storage", ["mix_fp32", "fp64"])
def test_noalloc_mass_matches_sl_mass_on_consecutive_calls(storage):
    import torch
    stream = torch.cuda.Stream()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    # two different problems, so the second call sees the first call's
    # leftover partial sums in the shared scratch
    for p in (W.config2(n=700, steps=1, storage=storage), W.config3(n=12, steps=1, storage=storage)):
        vol = _cell_volume(p.grid)
        with S.Context(p.grid, p.k, storage, stream=stream) as ctx:
            ctx.project(p.nq, p.weights, p.params)
            ctx.set_fields(p.field_list())
            for call in range(2):
                ref = ctx.mass()
                mean, _, _ = S.sl_get_planes(ctx.handle)
                d_mean = torch.from_numpy(mean).to("cuda")
                torch.cuda.synchronize()
                S.sl_mass_noalloc(d_mean.data_ptr(), mean.size, vol, out.data_ptr(), stream)
                stream.synchronize()
                got = float(out.item())
                assert abs(got - ref) <= MASS_TOL * abs(ref), (p.name, call, got, ref)
                ctx.step("strang", p.dt, 2)


@pytest.mark.gpu
def test_noalloc_mass_at_the_block_cap_matches_the_exact_sum():
    """3 000 000 seeded values, more than 1024 blocks of 256 threads and 8
    cells each: every one of the 1024 scratch slots is used and the
    reduction strides over the plane.  Two calls in a row, the second on a
    shorter prefix, against the correctly rounded sum times the volume."""
    import torch
    rng = np.random.default_rng(31)
    vals = rng.uniform(0.5, 1.5, 3_000_000)
    vol = 0.013
    d_mean = torch.from_numpy(vals).to("cuda")
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    for cells in (vals.size, 2_500_001):
        S.sl_mass_noalloc(d_mean.data_ptr(), cells, vol, out.data_ptr(), stream)
        stream.synchronize()
        exact = vol * math.fsum(vals[:cells].tolist())
        assert abs(float(out.item()) - exact) <= 1e-14 * exact, (cells, float(out.item()), exact)


def _library_or_skip():
    try:
        S.lib()
    except Exception as e:   # no nvcc build on this host
        pytest.skip(f"libsl.so not available: {e}")


def test_noalloc_rejects_bad_sizes_without_device_work():
    _library_or_skip()
    for cells in (0, -5, 2 ** 31):
        with pytest.raises(S.SlError) as e:
            S.sl_mass_noalloc(0x1000, cells, 1.0, 0x2000)
        assert e.value.status == S.SL_EINVAL
    with pytest.raises(S.SlError) as e:
        S.sl_mass_noalloc(0, 10, 1.0, 0x2000)
    assert e.value.status == S.SL_EINVAL
    with pytest.raises(S.SlError) as e:
        S.sl_mass_noalloc(0x1000, 10, float("nan"), 0x2000)
    assert e.value.status == S.SL_ENAN
