"""Checkpoint/resume of a context's state, and a file cache of the autotuner's
launch shapes.  Host-side bookkeeping around the C ABI (sl_get_planes,
sl_set_planes, sl_get_tune, sl_set_tune, sl_autotune); no arithmetic of the
method happens here.

Checkpoint: an ``.npz`` with the store's raw planes (the FP64 block, the
low-precision planes or cell records, the per-cell scales) and the context's
grid, degree and store, plus the caller's step counter, time and a JSON
``extra``.  Raw planes make a resumed run continue bit for bit in every store:
decoding to FP64 and encoding again would round the per-cell scales of the
scaled stores differently.  Fields, the self-consistent-field switch and the
nodal-velocity switch are settings, not state: the caller sets them again.

Tune cache: a JSON file mapping a key of (device, extents, pairs, degree,
store) to the launch shape of every dimension.  A hit sets the shapes without
timing anything; a miss runs sl_autotune and stores its choice.
"""
from __future__ import annotations

import json
import os
import tempfile
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np

CHECKPOINT_VERSION = 1


@dataclass(frozen=True)
class Box:
    """The grid of a checkpoint: periodic box, extents and x/v pairs."""
    n: Tuple[int, ...]
    lo: Tuple[float, ...]
    hi: Tuple[float, ...]
    pair: Tuple[int, ...]


def write_checkpoint(path, meta: dict, mean, hi, scale) -> None:
    """Write the planes and the metadata (a JSON-serialisable dict) to path,
    atomically (a temporary file in the same directory, then a rename)."""
    arrays = {"meta": np.frombuffer(json.dumps(meta, sort_keys=True).encode(), dtype=np.uint8),
              "hi": np.ascontiguousarray(hi)}
    if mean is not None:
        arrays["mean"] = np.ascontiguousarray(mean)
    if scale is not None:
        arrays["scale"] = np.ascontiguousarray(scale)
    d = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(dir=d, suffix=".npz.tmp")
    os.close(fd)
    try:
        with open(tmp, "wb") as f:
            np.savez(f, **arrays)
        os.replace(tmp, path)
    finally:
        if os.path.exists(tmp):
            os.unlink(tmp)


def read_checkpoint(path):
    """(meta, mean, hi, scale) of a checkpoint file; mean / scale may be None."""
    with np.load(path, allow_pickle=False) as z:
        meta = json.loads(bytes(z["meta"]).decode())
        if meta.get("version") != CHECKPOINT_VERSION:
            raise ValueError(f"checkpoint version {meta.get('version')} is not {CHECKPOINT_VERSION}")
        mean = z["mean"] if "mean" in z.files else None
        hi = z["hi"]
        scale = z["scale"] if "scale" in z.files else None
    return meta, mean, hi, scale


def checkpoint_meta(grid, degree: int, storage, step: int, time: float, extra=None) -> dict:
    return {"version": CHECKPOINT_VERSION,
            "grid": {"n": [int(x) for x in grid.n], "lo": [float(x) for x in grid.lo],
                     "hi": [float(x) for x in grid.hi], "pair": [int(x) for x in grid.pair]},
            "degree": int(degree), "storage": storage if isinstance(storage, str) else int(storage),
            "step": int(step), "time": float(time), "extra": extra}


def save_checkpoint(ctx, path, step: int = 0, time: float = 0.0, extra=None) -> None:
    """Checkpoint a Context's current state (synchronises its stream)."""
    from . import sl_get_planes
    mean, hi, scale = sl_get_planes(ctx.handle)
    write_checkpoint(path, checkpoint_meta(ctx.grid, ctx.degree, ctx.storage, step, time, extra), mean, hi, scale)


def load_checkpoint(path, stream=None):
    """(Context holding the checkpointed state, meta).  The caller sets fields
    and switches again before stepping."""
    from . import Context, sl_set_planes
    meta, mean, hi, scale = read_checkpoint(path)
    g = meta["grid"]
    box = Box(tuple(g["n"]), tuple(g["lo"]), tuple(g["hi"]), tuple(g["pair"]))
    ctx = Context(box, meta["degree"], meta["storage"], stream=stream)
    try:
        sl_set_planes(ctx.handle, mean, hi, scale)
        ctx.synchronize()
    except Exception:
        ctx.close()
        raise
    return ctx, meta


# ---------------------------------------------------------------------------
# tune cache
# ---------------------------------------------------------------------------

def device_name() -> str:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_name(torch.cuda.current_device())
    except Exception:
        pass
    return "unknown"


def tune_key(device: str, n: Sequence[int], pair: Sequence[int], degree: int, storage) -> str:
    return json.dumps({"device": device, "n": [int(x) for x in n], "pair": [int(x) for x in pair],
                       "degree": int(degree), "storage": storage if isinstance(storage, str) else int(storage)},
                      sort_keys=True)


def _load_cache(path) -> dict:
    if not os.path.exists(path):
        return {}
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def _store_cache(path, data: dict) -> None:
    d = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(dir=d, suffix=".json.tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def autotune_cached(ctx, path, reps: int = 3, device: Optional[str] = None) -> bool:
    """Set ctx's launch shapes from the cache file at path, or autotune and
    record them.  Returns True on a cache hit.  ctx needs grid, degree,
    storage, get_tune, set_tune and autotune (a Context)."""
    g = ctx.grid
    key = tune_key(device or device_name(), g.n, g.pair, ctx.degree, ctx.storage)
    data = _load_cache(path)
    shapes = data.get(key)
    if shapes is not None and len(shapes) == len(g.n):
        try:
            for d, sh in enumerate(shapes):
                ctx.set_tune(d, **sh)
            return True
        except Exception:     # a shape this library does not provide: tune again
            pass
    ctx.autotune(reps)
    data[key] = [dict(ctx.get_tune(d)) for d in range(len(g.n))]
    _store_cache(path, data)
    return False
