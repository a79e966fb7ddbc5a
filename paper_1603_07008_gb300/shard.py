"""One grid split along one dimension over several ranks: the slab each rank
holds and the halo of source cells that a sweep along the split dimension
needs from the neighbouring ranks.

The update rule of Sec. II-A is local: the new coefficients of cell i come
from the cells i - sigma and i - sigma - 1 only, sigma = floor(s) of the
line's shift s in cells (one more when the fractional part rounds to 1).  A
rank holding the cells [start, stop) of the split dimension therefore needs,
for shifts in [s_min, s_max], the cells start - sigma_max - 1 .. start - 1
from the rank below and stop .. stop - 1 - sigma_min from the rank above
(periodic).  Sweeps along every other dimension stay inside a slab, and the
mass of the grid is the sum of the slabs' masses.

This module only plans and moves data (torch.distributed point-to-point
free: one all_gather of equal-shaped boundary blocks per exchange); it holds
none of the method's arithmetic, and works on host arrays with any backend
that supports all_gather (gloo on the CPU).
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np

__all__ = ["slab_bounds", "halo_widths", "exchange_halos"]


def slab_bounds(n: int, world: int) -> List[Tuple[int, int]]:
    """[start, stop) of each rank's slab of n cells, sizes differing by at most one."""
    if world < 1 or n < world:
        raise ValueError(f"cannot split {n} cells over {world} ranks")
    base, extra = divmod(n, world)
    out, start = [], 0
    for r in range(world):
        size = base + (1 if r < extra else 0)
        out.append((start, start + size))
        start += size
    return out


def halo_widths(shift_min: float, shift_max: float) -> Tuple[int, int]:
    """(cells below, cells above) a slab that a sweep with shifts (in cells) in
    [shift_min, shift_max] reads: sigma lies in [floor(shift_min),
    floor(shift_max) + 1] (the second bound covers a fractional part that
    rounds to 1), and a target reads the cells i - sigma and i - sigma - 1."""
    if not (math.isfinite(shift_min) and math.isfinite(shift_max)) or shift_min > shift_max:
        raise ValueError("shift bounds must be finite and ordered")
    sig_min = math.floor(shift_min)
    sig_max = math.floor(shift_max) + 1
    return max(sig_max + 1, 0), max(-sig_min, 0)


def exchange_halos(slab: np.ndarray, lo: int, hi: int, axis: int, group=None) -> np.ndarray:
    """The slab extended by lo cells from the rank below and hi cells from the
    rank above along `axis` (ranks in a periodic ring; with one rank the slab
    wraps onto itself).  Every rank's slab must hold at least max(lo, hi)
    cells along `axis` and have the same shape along the other axes."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    size = slab.shape[axis]
    if max(lo, hi) > size:
        raise ValueError(f"halo of {max(lo, hi)} cells exceeds a slab of {size}")
    top = np.take(slab, range(size - lo, size), axis=axis)      # the next rank's lower halo
    bottom = np.take(slab, range(0, hi), axis=axis)              # the previous rank's upper halo
    if world == 1:
        below, above = top, bottom
    else:
        def gather(block):
            t = torch.from_numpy(np.ascontiguousarray(block))
            parts = [torch.empty_like(t) for _ in range(world)]
            dist.all_gather(parts, t, group=group)
            return [p.numpy() for p in parts]
        tops = gather(top)
        bottoms = gather(bottom)
        below = tops[(rank - 1) % world]
        above = bottoms[(rank + 1) % world]
    return np.concatenate([below, slab, above], axis=axis)
