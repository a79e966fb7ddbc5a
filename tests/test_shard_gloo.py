"""One grid split along an x-dimension over ranks (paper_1603_07008_gb300.shard):
the slabs, the halo widths, and -- with two gloo ranks on the CPU -- split
steps whose sweeps along the split dimension read their halo from the
neighbouring rank, computed by the oracle.  They must equal the same steps
on the whole grid bit for bit, and the slabs' masses must add up to the
grid's (Sec. II-A: each target cell reads two source cells per sweep)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1603_07008_gb300 import shard
from paper_1603_07008_gb300 import workloads as W


def test_slab_bounds():
    assert shard.slab_bounds(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert shard.slab_bounds(8, 2) == [(0, 4), (4, 8)]
    assert shard.slab_bounds(5, 1) == [(0, 5)]
    with pytest.raises(ValueError):
        shard.slab_bounds(2, 3)


def test_halo_widths():
    # shifts in [0.2, 0.4]: sigma in {0, 1}; cells i - 2 .. i read
    assert shard.halo_widths(0.2, 0.4) == (2, 0)
    # negative shifts read cells above the slab (sigma in [-3, 0]: a shift just
    # below an integer may round up to it, so one cell below is kept)
    assert shard.halo_widths(-2.5, -0.5) == (1, 3)
    assert shard.halo_widths(-1.3, 2.7) == (4, 2)
    with pytest.raises(ValueError):
        shard.halo_widths(1.0, -1.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    p = W.config2(n=8, steps=3)
    # 24 x-cells, 12 v-cells; the field strong enough for shifts of several cells
    p.grid = W.Grid(n=(24, 12), lo=p.grid.lo, hi=p.grid.hi, pair=p.grid.pair)
    x = p.grid.lo[0] + (np.arange(24) + 0.5) * (p.grid.hi[0] - p.grid.lo[0]) / 24
    p.fields = {0: 2.0 * np.sin(0.5 * x)}
    return p


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _problem()
        nx, nv = p.grid.n
        k = p.k
        nc = (k + 1) ** 2
        u = O.project(p.grid, k, p.nq, p.weights, p.params).reshape(nv, nx, nc)
        s, e = shard.slab_bounds(nx, world)[rank]
        slab = u[:, s:e, :].copy()
        sched = O.schedule(p.grid, "strang", p.dt, p.field_list())
        for _ in range(p.steps):
            for dim, sd, shifts in sched:
                if dim == 0:        # along the split dimension: shifts per v-line
                    lo, hi = shard.halo_widths(float(np.min(shifts)), float(np.max(shifts)))
                    ext = shard.exchange_halos(slab, lo, hi, axis=1)
                    n_ext = ext.shape[1]
                    out = O.sweep(ext.reshape(-1, nc), [n_ext, nv], k, 0, sd, shifts)
                    slab = out.reshape(nv, n_ext, nc)[:, lo:lo + (e - s), :].copy()
                else:               # along v: every line lies in the slab; field of the slab's x-cells
                    out = O.sweep(slab.reshape(-1, nc), [e - s, nv], k, 1, 0, np.asarray(shifts)[s:e])
                    slab = out.reshape(nv, e - s, nc)
        np.save(os.path.join(out_dir, f"slab{rank}.npy"), slab)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_steps_equal_the_whole_grid(tmp_path, world):
    import oracle as O
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    p = _problem()
    nx, nv = p.grid.n
    nc = (p.k + 1) ** 2
    u0 = O.project(p.grid, p.k, p.nq, p.weights, p.params)
    ref = O.step(u0, p.grid, p.k, "strang", p.dt, p.steps, p.field_list()).reshape(nv, nx, nc)
    slabs = [np.load(tmp_path / f"slab{r}.npy") for r in range(world)]
    got = np.concatenate(slabs, axis=1)
    assert np.array_equal(got, ref)
    # the shifts span several cells, so the halos are wider than one cell
    sched = O.schedule(p.grid, "strang", p.dt, p.field_list())
    assert max(shard.halo_widths(float(np.min(s)), float(np.max(s)))[0] for d, _, s in sched if d == 0) >= 2
    # mass of the grid = sum of the slabs' masses
    vol = (p.grid.hi[0] - p.grid.lo[0]) / nx * (p.grid.hi[1] - p.grid.lo[1]) / nv
    total = sum(vol * float(np.sum(sl[:, :, 0])) for sl in slabs)
    whole = O.mass(ref.reshape(-1, nc), p.grid, p.k)
    assert abs(total - whole) <= 1e-14 * abs(whole)
