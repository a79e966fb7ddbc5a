"""GB300 (sm_103a) semi-Lagrangian discontinuous Galerkin projection sweep.

Python binding of ``libsl.so`` (declared in ``include/sl.h``).  The functions
below carry the C names and only marshal arguments: every step of the sweep,
the matrix construction, the mass reduction, the codec and the projection run
in the library's CUDA kernels.  There is no CPU fallback: if the library
cannot be built or loaded, ``lib()`` raises.

Method: L. Einkemmer, "A mixed precision semi-Lagrangian algorithm and its
performance on accelerators", HPCS 2016 (arXiv:1603.07008), Sec. II-A.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "SL_OK", "SL_EINVAL", "SL_ENOMEM", "SL_ECUDA", "SL_ETIMEOUT", "SL_ENAN", "SL_ENOTSUP",
    "SL_FP64", "SL_MIX_FP32", "SL_MIX_BF16", "SL_MIX_FP16", "SL_FP32", "SL_MIX_FP32_D2", "SL_MIX_FP32_D3",
    "N_DOUBLE", "plane_counts", "SL_LIE", "SL_STRANG", "STORAGE",
    "SlError", "sl_grid", "make_grid", "lib", "library_path", "Context",
    "sl_create", "sl_destroy", "sl_last_error", "sl_get_info", "sl_state_bytes", "sl_ab_host",
    "sl_set_coeffs", "sl_get_coeffs", "sl_get_cells", "sl_set_planes", "sl_get_planes", "sl_project", "sl_advect",
    "sl_set_fields", "sl_step", "sl_mass", "sl_graph_capture", "sl_graph_launch",
    "sl_synchronize", "sl_profile_enable", "sl_profile_query", "sl_mass_noalloc",
    "sl_get_tune", "sl_set_tune", "sl_autotune", "sl_profile_dims", "Batch",
    "sl_batch_create", "sl_batch_destroy", "sl_batch_last_error", "sl_batch_info", "sl_batch_project",
    "sl_batch_set_coeffs", "sl_batch_get_coeffs", "sl_batch_set_fields", "sl_batch_step",
    "sl_batch_mass", "sl_batch_graph_capture", "sl_batch_graph_launch", "sl_batch_synchronize",
    "sl_batch_autotune", "sl_batch_profile_enable", "sl_batch_profile_query", "sl_batch_profile_dims",
    "sl_batch_get_tune", "sl_batch_set_tune", "sl_selftest_conversions", "sl_set_poisson", "sl_get_field",
    "sl_field_energy", "sl_graph_capture_advect", "sl_create_external", "sl_plane_layout",
    "sl_set_nodal_velocity", "sl_advect_nodal", "sl_check_guards", "sl_debug_fail_alloc",
    "sl_debug_corrupt_guard", "save_checkpoint", "load_checkpoint", "autotune_cached", "sl_selftest_sub_widened",
    "sl_set_arithmetic", "sl_selftest_fp64_rate",
]

SL_OK, SL_EINVAL, SL_ENOMEM, SL_ECUDA, SL_ETIMEOUT, SL_ENAN, SL_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
SL_FP64, SL_MIX_FP32, SL_MIX_BF16, SL_MIX_FP16 = 0, 1, 2, 3
SL_FP32, SL_MIX_FP32_D2, SL_MIX_FP32_D3 = 4, 5, 6
SL_LIE, SL_STRANG = 0, 1
SL_ARITH_STORE, SL_ARITH_FP64 = 0, 1
ARITH = {"store": SL_ARITH_STORE, "fp64": SL_ARITH_FP64}
STORAGE = {"fp64": SL_FP64, "mix_fp32": SL_MIX_FP32, "mix_bf16": SL_MIX_BF16, "mix_fp16": SL_MIX_FP16,
           "fp32": SL_FP32, "mix_fp32_d2": SL_MIX_FP32_D2, "mix_fp32_d3": SL_MIX_FP32_D3}
# Coefficients per dimension kept in FP64 ("# double" of Sec. III-A) of the
# stores that keep a block of them (the mixed stores keep the mean: 1).
N_DOUBLE = {SL_FP32: 0, SL_MIX_FP32: 1, SL_MIX_FP32_D2: 2, SL_MIX_FP32_D3: 3}
SPLITTING = {"lie": SL_LIE, "strang": SL_STRANG}
MAX_DIM = 6


class SlError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"sl status {status}: {msg}")
        self.status = status


class sl_tune(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("fibres_per_thread", ctypes.c_int32),
                ("unroll", ctypes.c_int32), ("pipeline", ctypes.c_int32), ("chunk", ctypes.c_int64),
                ("max_blocks_per_sm", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class sl_layout(ctypes.Structure):
    _fields_ = [("plane_stride", ctypes.c_int64), ("record_slots", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("mean_bytes", ctypes.c_int64), ("hi_bytes", ctypes.c_int64), ("scale_bytes", ctypes.c_int64)]


class sl_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("n", ctypes.c_int64 * MAX_DIM),
                ("lo", ctypes.c_double * MAX_DIM), ("hi", ctypes.c_double * MAX_DIM),
                ("pair", ctypes.c_int32 * MAX_DIM)]


class sl_info(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_int64), ("ncoef", ctypes.c_int64), ("dof", ctypes.c_int64),
                ("plane_stride", ctypes.c_int64), ("state_bytes", ctypes.c_int64),
                ("alloc_bytes", ctypes.c_int64), ("degree", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("record_slots", ctypes.c_int32)]


def make_grid(g) -> sl_grid:
    """sl_grid from any object with n, lo, hi, pair sequences (or an sl_grid)."""
    if isinstance(g, sl_grid):
        return g
    s = sl_grid()
    nd = len(g.n)
    s.ndim = nd
    for m in range(MAX_DIM):
        s.n[m] = int(g.n[m]) if m < nd else 1
        s.lo[m] = float(g.lo[m]) if m < nd else 0.0
        s.hi[m] = float(g.hi[m]) if m < nd else 1.0
        s.pair[m] = int(g.pair[m]) if m < nd else -1
    return s


_lock = threading.Lock()
_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


def library_path() -> str:
    from . import build as _b
    return _b.LIB


def lib():
    """Load libsl.so, building it with nvcc first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _b
        try:
            path = _b.build()
        except Exception as e:  # no silent fallback: the CUDA library is the product
            raise RuntimeError(f"libsl.so could not be built: {e}") from e
        L = ctypes.CDLL(path)
        st = ctypes.c_int
        sig = {
            "sl_create": (st, [ctypes.POINTER(sl_grid), ctypes.c_int, ctypes.c_int, _vp,
                               ctypes.POINTER(_vp)]),
            "sl_destroy": (None, [_vp]),
            "sl_last_error": (ctypes.c_char_p, [_vp]),
            "sl_get_info": (st, [_vp, ctypes.POINTER(sl_info)]),
            "sl_state_bytes": (st, [ctypes.POINTER(sl_grid), ctypes.c_int, ctypes.c_int, _i64p]),
            "sl_ab_host": (st, [ctypes.c_int, ctypes.c_double, _dp, _dp]),
            "sl_set_coeffs": (st, [_vp, _dp]),
            "sl_get_coeffs": (st, [_vp, _dp]),
            "sl_get_cells": (st, [_vp, _i64p, ctypes.c_int64, _dp]),
            "sl_set_planes": (st, [_vp, _dp, _vp, ctypes.POINTER(ctypes.c_float)]),
            "sl_get_planes": (st, [_vp, _dp, _vp, ctypes.POINTER(ctypes.c_float)]),
            "sl_project": (st, [_vp, ctypes.c_int, ctypes.c_int, _dp, _dp]),
            "sl_advect": (st, [_vp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int64]),
            "sl_set_fields": (st, [_vp, _dp, ctypes.c_int64]),
            "sl_step": (st, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_int]),
            "sl_mass": (st, [_vp, _dp]),
            "sl_graph_capture": (st, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_int]),
            "sl_graph_launch": (st, [_vp]),
            "sl_synchronize": (st, [_vp]),
            "sl_profile_enable": (st, [_vp, ctypes.c_int]),
            "sl_profile_query": (st, [_vp, _i64p, _dp, _dp]),
            "sl_profile_dims": (st, [_vp, _i64p, _dp]),
            "sl_get_tune": (st, [_vp, ctypes.c_int, ctypes.POINTER(sl_tune)]),
            "sl_set_tune": (st, [_vp, ctypes.c_int, ctypes.POINTER(sl_tune)]),
            "sl_autotune": (st, [_vp, ctypes.c_int]),
            "sl_batch_create": (st, [ctypes.c_int, ctypes.POINTER(sl_grid), ctypes.POINTER(ctypes.c_int),
                                     ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
            "sl_batch_destroy": (None, [_vp]),
            "sl_batch_last_error": (ctypes.c_char_p, [_vp]),
            "sl_batch_info": (st, [_vp, _i64p, _i64p, _i64p]),
            "sl_batch_project": (st, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]),
            "sl_batch_set_coeffs": (st, [_vp, ctypes.c_int, _dp]),
            "sl_batch_get_coeffs": (st, [_vp, ctypes.c_int, _dp]),
            "sl_batch_set_fields": (st, [_vp, _dp, ctypes.c_int64]),
            "sl_batch_step": (st, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_int]),
            "sl_batch_mass": (st, [_vp, _dp]),
            "sl_batch_graph_capture": (st, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_int]),
            "sl_batch_graph_launch": (st, [_vp]),
            "sl_batch_synchronize": (st, [_vp]),
            "sl_batch_autotune": (st, [_vp, ctypes.c_int]),
            "sl_batch_profile_enable": (st, [_vp, ctypes.c_int]),
            "sl_batch_profile_query": (st, [_vp, _i64p, _dp, _dp]),
            "sl_batch_profile_dims": (st, [_vp, _i64p, _dp]),
            "sl_batch_get_tune": (st, [_vp, ctypes.c_int, ctypes.POINTER(sl_tune)]),
            "sl_batch_set_tune": (st, [_vp, ctypes.c_int, ctypes.POINTER(sl_tune)]),
            "sl_mass_noalloc": (st, [_vp, ctypes.c_int64, ctypes.c_double, _vp, _vp]),
            "sl_set_poisson": (st, [_vp, ctypes.c_int]),
            "sl_set_nodal_velocity": (st, [_vp, ctypes.c_int]),
            "sl_set_arithmetic": (st, [_vp, ctypes.c_int]),
            "sl_selftest_fp64_rate": (st, [ctypes.c_int64, _vp, _dp]),
            "sl_check_guards": (st, [_vp, _i64p]),
            "sl_selftest_sub_widened": (st, [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                             ctypes.c_int64, _dp, _i64p]),
            "sl_debug_fail_alloc": (st, [ctypes.c_int64]),
            "sl_debug_corrupt_guard": (st, [_vp]),
            "sl_advect_nodal": (st, [_vp, ctypes.c_int, ctypes.c_double]),
            "sl_create_external": (st, [ctypes.POINTER(sl_grid), ctypes.c_int, ctypes.c_int, _vp,
                                        ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
            "sl_plane_layout": (st, [ctypes.POINTER(sl_grid), ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(sl_layout)]),
            "sl_graph_capture_advect": (st, [_vp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int64, ctypes.c_int]),
            "sl_get_field": (st, [_vp, _dp]),
            "sl_field_energy": (st, [_vp, _dp]),
            "sl_selftest_conversions": (st, [_dp, ctypes.POINTER(ctypes.c_float), ctypes.c_int64,
                                             ctypes.POINTER(ctypes.c_float), _dp, _i64p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray, t=_dp):
    return a.ctypes.data_as(t)


def sl_last_error(ctx=None) -> str:
    r = lib().sl_last_error(ctx)
    return r.decode() if r else ""


def _check(status: int, ctx=None):
    if status != SL_OK:
        raise SlError(status, sl_last_error(ctx))


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def sl_create(grid, degree: int, storage, stream=None):
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    g = make_grid(grid)
    out = _vp()
    _check(lib().sl_create(ctypes.byref(g), int(degree), st, _stream_handle(stream), ctypes.byref(out)))
    return out


def sl_destroy(ctx):
    if ctx:
        lib().sl_destroy(ctx)


def sl_get_info(ctx) -> dict:
    i = sl_info()
    _check(lib().sl_get_info(ctx, ctypes.byref(i)), ctx)
    return {k: getattr(i, k) for k, _ in sl_info._fields_}


def sl_state_bytes(grid, degree: int, storage) -> int:
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    b = ctypes.c_int64()
    g = make_grid(grid)
    _check(lib().sl_state_bytes(ctypes.byref(g), int(degree), st, ctypes.byref(b)))
    return b.value


def sl_ab_host(degree: int, alpha: float) -> Tuple[np.ndarray, np.ndarray]:
    o = degree + 1
    A = np.zeros((o, o))
    B = np.zeros((o, o))
    _check(lib().sl_ab_host(int(degree), float(alpha), _ptr(A), _ptr(B)))
    return A, B


def sl_set_coeffs(ctx, u: np.ndarray):
    u_ = _f64(u)
    info = sl_get_info(ctx)
    if u_.size != info["dof"]:
        raise ValueError(f"expected {info['dof']} coefficients, got {u_.size}")
    _check(lib().sl_set_coeffs(ctx, _ptr(u_)), ctx)


def sl_get_coeffs(ctx) -> np.ndarray:
    info = sl_get_info(ctx)
    out = np.empty((info["cells"], info["ncoef"]))
    _check(lib().sl_get_coeffs(ctx, _ptr(out)), ctx)
    return out


def sl_get_cells(ctx, cells) -> np.ndarray:
    info = sl_get_info(ctx)
    c = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.empty((c.size, info["ncoef"]))
    _check(lib().sl_get_cells(ctx, _ptr(c, _i64p), c.size, _ptr(out)), ctx)
    return out


_ELEM = {SL_FP64: np.float64, SL_MIX_FP32: np.float32, SL_MIX_BF16: np.uint16,
         SL_MIX_FP16: np.uint16, SL_FP32: np.float32, SL_MIX_FP32_D2: np.float32, SL_MIX_FP32_D3: np.float32}


def plane_counts(ndim: int, degree: int, storage) -> Tuple[int, int]:
    """(FP64 planes, low-precision planes) of one copy of the state: q^d and
    o^d - q^d for the stores of # double = q (0, 2, 3), else 1 and o^d - 1."""
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    nc = (degree + 1) ** ndim
    nlo = N_DOUBLE[st] ** ndim if st in (SL_FP32, SL_MIX_FP32_D2, SL_MIX_FP32_D3) else 1
    return nlo, nc - nlo


def plane_arrays(ctx):
    """Host numpy arrays (mean, hi, scale) shaped for sl_get_planes / sl_set_planes:
    mean is [cells] (one FP64 plane), [n_lo, cells] (several) or None (SL_FP32)."""
    info = sl_get_info(ctx)
    st = info["storage"]
    if st in (SL_FP32, SL_MIX_FP32_D2, SL_MIX_FP32_D3):
        # state bytes = cells (8 n_lo + 4 n_hi), n_lo + n_hi = o^d
        nlo = (info["state_bytes"] // info["cells"] - 4 * info["ncoef"]) // 4
    else:
        nlo = 1
    nhi = info["ncoef"] - nlo
    if nlo == 0:
        mean = None
    elif nlo == 1:
        mean = np.empty(info["cells"], dtype=np.float64)
    else:
        mean = np.empty((nlo, info["cells"]), dtype=np.float64)
    if info["record_slots"]:
        hi = np.empty((info["cells"], info["record_slots"]), dtype=_ELEM[st])
    else:
        hi = np.empty((nhi, info["cells"]), dtype=_ELEM[st])
    scale = np.empty(info["cells"], dtype=np.float32) if st in (SL_MIX_BF16, SL_MIX_FP16) else None
    return mean, hi, scale


def sl_set_planes(ctx, mean, hi, scale=None):
    """Enqueue the copy of raw planes (host arrays or raw host addresses).
    The memory must stay valid until the context's stream passes the copy."""
    fp = ctypes.POINTER(ctypes.c_float)
    if mean is None:
        m = None
    else:
        m = mean if isinstance(mean, int) else _ptr(mean)
        m = ctypes.cast(m, _dp) if isinstance(mean, int) else m
    h = hi if isinstance(hi, int) else hi.ctypes.data
    s = None if scale is None else (ctypes.cast(scale, fp) if isinstance(scale, int) else scale.ctypes.data_as(fp))
    _check(lib().sl_set_planes(ctx, m, ctypes.c_void_p(h), s), ctx)


def sl_get_planes(ctx, mean=None, hi=None, scale=None):
    if hi is None:
        mean, hi, scale = plane_arrays(ctx)
    fp = ctypes.POINTER(ctypes.c_float)
    s = None if scale is None else scale.ctypes.data_as(fp)
    m = None if mean is None else _ptr(mean)
    _check(lib().sl_get_planes(ctx, m, ctypes.c_void_p(hi.ctypes.data), s), ctx)
    return mean, hi, scale


def sl_project(ctx, nq: int, weights, params):
    w = _f64(weights)
    p = _f64(params)
    _check(lib().sl_project(ctx, int(nq), int(w.size), _ptr(w), _ptr(p)), ctx)


def sl_advect(ctx, dim: int, shift_dim: int, shifts):
    s = _f64(np.atleast_1d(shifts))
    _check(lib().sl_advect(ctx, int(dim), int(shift_dim), _ptr(s), s.size), ctx)


def sl_set_fields(ctx, fields):
    if isinstance(fields, (list, tuple)):
        f = _f64(np.concatenate([np.ravel(x) for x in fields])) if fields else np.zeros(0)
    else:
        f = _f64(fields)
    _check(lib().sl_set_fields(ctx, _ptr(f), f.size), ctx)


def _split(s) -> int:
    return SPLITTING[s] if isinstance(s, str) else int(s)


def sl_step(ctx, splitting, dt: float, nsteps: int):
    _check(lib().sl_step(ctx, _split(splitting), float(dt), int(nsteps)), ctx)


def sl_mass(ctx) -> float:
    m = ctypes.c_double()
    _check(lib().sl_mass(ctx, ctypes.byref(m)), ctx)
    return m.value


def sl_graph_capture(ctx, splitting, dt: float, nsteps: int):
    _check(lib().sl_graph_capture(ctx, _split(splitting), float(dt), int(nsteps)), ctx)


def sl_graph_launch(ctx):
    _check(lib().sl_graph_launch(ctx), ctx)


def sl_synchronize(ctx):
    _check(lib().sl_synchronize(ctx), ctx)


def sl_profile_enable(ctx, enable: bool = True):
    _check(lib().sl_profile_enable(ctx, 1 if enable else 0), ctx)


def sl_profile_query(ctx) -> Tuple[int, float, float]:
    n = ctypes.c_int64()
    ms = ctypes.c_double()
    b = ctypes.c_double()
    _check(lib().sl_profile_query(ctx, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(b)), ctx)
    return n.value, ms.value, b.value


def sl_profile_dims(ctx):
    """(launches[6], ms[6]) per sweep dimension of the last sl_profile_query."""
    n = (ctypes.c_int64 * MAX_DIM)()
    ms = (ctypes.c_double * MAX_DIM)()
    _check(lib().sl_profile_dims(ctx, n, ms), ctx)
    return list(n), list(ms)


def sl_get_tune(ctx, dim: int) -> dict:
    t = sl_tune()
    _check(lib().sl_get_tune(ctx, int(dim), ctypes.byref(t)), ctx)
    return {k: getattr(t, k) for k, _ in sl_tune._fields_ if k != "reserved"}


def sl_set_tune(ctx, dim: int, block: int, fibres_per_thread: int = 1, unroll: int = 1,
                chunk: int = 0, pipeline: int = 0, max_blocks_per_sm: int = 0):
    t = sl_tune(int(block), int(fibres_per_thread), int(unroll), int(pipeline), int(chunk),
                int(max_blocks_per_sm), 0)
    _check(lib().sl_set_tune(ctx, int(dim), ctypes.byref(t)), ctx)


def sl_autotune(ctx, reps: int = 3):
    _check(lib().sl_autotune(ctx, int(reps)), ctx)


def sl_selftest_conversions(d_in, f_in):
    """(fl32(d), fl32(-d), double(f), mismatches) from the library's device
    conversions; mismatches counts elements where its two forms disagree."""
    d = np.ascontiguousarray(d_in, dtype=np.float64)
    f = np.ascontiguousarray(f_in, dtype=np.float32)
    if d.size != f.size:
        raise ValueError("d_in and f_in differ in length")
    fo = np.empty(2 * d.size, dtype=np.float32)
    do = np.empty(d.size, dtype=np.float64)
    mm = ctypes.c_int64()
    st = lib().sl_selftest_conversions(d.ctypes.data_as(_dp), f.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                       d.size, fo.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                       do.ctypes.data_as(_dp), ctypes.byref(mm))
    if st != SL_OK:
        raise SlError(st, "sl_selftest_conversions failed")
    return fo[0::2], fo[1::2], do, mm.value


def sl_graph_capture_advect(ctx, dim: int, shift_dim: int, shifts, nsteps: int):
    s = np.ascontiguousarray(np.atleast_1d(shifts), dtype=np.float64)
    _check(lib().sl_graph_capture_advect(ctx, int(dim), int(shift_dim), s.ctypes.data_as(_dp), s.size,
                                         int(nsteps)), ctx)


def sl_plane_layout(grid, degree: int, storage) -> dict:
    """Layout of one copy of the state (see sl.h)."""
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    g = make_grid(grid)
    lay = sl_layout()
    _check(lib().sl_plane_layout(ctypes.byref(g), int(degree), st, ctypes.byref(lay)))
    return {k: getattr(lay, k) for k, _ in sl_layout._fields_ if k != "reserved"}


def sl_create_external(grid, degree: int, storage, planes, stream=None):
    """Context over six caller-owned device addresses (integers or 0):
    mean_0, hi_0, scale_0, mean_1, hi_1, scale_1."""
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    g = make_grid(grid)
    arr = (_vp * 6)(*[_vp(int(p)) if p else _vp() for p in planes])
    h = _vp()
    _check(lib().sl_create_external(ctypes.byref(g), int(degree), st, _stream_handle(stream), arr,
                                    ctypes.byref(h)))
    return h


def sl_set_poisson(ctx, enable=True):
    _check(lib().sl_set_poisson(ctx, 1 if enable else 0), ctx)


def sl_set_nodal_velocity(ctx, enable=True):
    _check(lib().sl_set_nodal_velocity(ctx, 1 if enable else 0), ctx)


def sl_advect_nodal(ctx, dim: int, tau: float):
    _check(lib().sl_advect_nodal(ctx, int(dim), float(tau)), ctx)


def sl_selftest_fp64_rate(iters: int = 1 << 14, stream=None) -> float:
    """Measured FP64 FLOP/s of the current device."""
    out = ctypes.c_double()
    _check(lib().sl_selftest_fp64_rate(int(iters), _stream_handle(stream), ctypes.byref(out)))
    return out.value


def sl_set_arithmetic(ctx, arith):
    """"store" (SL_ARITH_STORE) or "fp64" (SL_ARITH_FP64), or the number."""
    a = ARITH[arith] if isinstance(arith, str) else int(arith)
    _check(lib().sl_set_arithmetic(ctx, a), ctx)


def sl_selftest_sub_widened(a, b):
    """(float64(a) - float64(b) as the library's mean row forms it, mismatches
    between its integer-pipe and FP64 forms)."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    out = np.empty(a.size, dtype=np.float64)
    mm = ctypes.c_int64()
    fp = ctypes.POINTER(ctypes.c_float)
    _check(lib().sl_selftest_sub_widened(a.ctypes.data_as(fp), b.ctypes.data_as(fp), a.size, _ptr(out),
                                         ctypes.byref(mm)))
    return out, mm.value


def sl_check_guards(ctx) -> int:
    """Bytes of the context's guard bands and plane padding that lost their
    canary value (0 after a sound run)."""
    n = ctypes.c_int64()
    _check(lib().sl_check_guards(ctx, ctypes.byref(n)), ctx)
    return n.value


def sl_debug_fail_alloc(n: int):
    _check(lib().sl_debug_fail_alloc(int(n)))


def sl_debug_corrupt_guard(ctx):
    _check(lib().sl_debug_corrupt_guard(ctx), ctx)


def sl_get_field(ctx, nx: int) -> np.ndarray:
    out = np.empty(int(nx), dtype=np.float64)
    _check(lib().sl_get_field(ctx, out.ctypes.data_as(_dp)), ctx)
    return out


def sl_field_energy(ctx) -> float:
    w = ctypes.c_double()
    _check(lib().sl_field_energy(ctx, ctypes.byref(w)), ctx)
    return w.value


def sl_mass_noalloc(d_mean: int, cells: int, cell_volume: float, d_out: int, stream=None):
    """Allocation-free mass reduction on raw device addresses (integers):
    enqueues d_out[0] = cell_volume * sum(d_mean[:cells]) on `stream`."""
    st = lib().sl_mass_noalloc(ctypes.c_void_p(int(d_mean)), int(cells), float(cell_volume),
                               ctypes.c_void_p(int(d_out)), _stream_handle(stream))
    if st != SL_OK:
        why = {SL_EINVAL: "NULL pointer or cells outside [1, 2^31 - 1]",
               SL_ENAN: "cell_volume is NaN",
               SL_ECUDA: "scratch address lookup or kernel launch failed"}.get(st, "failed")
        raise SlError(st, f"sl_mass_noalloc: {why}")


class Context:
    """Owns one sl_ctx handle; methods forward to the functions above."""

    def __init__(self, grid, degree: int, storage, stream=None, planes=None):
        """planes: six device addresses for sl_create_external (the caller
        keeps that memory alive), or None for library-owned state."""
        self.grid = grid
        self.degree = degree
        self.storage = storage
        if planes is None:
            self.handle = sl_create(grid, degree, storage, stream)
        else:
            self.handle = sl_create_external(grid, degree, storage, planes, stream)
        self.info = sl_get_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            sl_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_coeffs(self, u):
        sl_set_coeffs(self.handle, u)

    def get_coeffs(self) -> np.ndarray:
        return sl_get_coeffs(self.handle)

    def get_cells(self, cells) -> np.ndarray:
        return sl_get_cells(self.handle, cells)

    def project(self, nq, weights, params):
        sl_project(self.handle, nq, weights, params)

    def advect(self, dim, shift_dim, shifts):
        sl_advect(self.handle, dim, shift_dim, shifts)

    def set_fields(self, fields):
        sl_set_fields(self.handle, fields)

    def step(self, splitting, dt, nsteps=1):
        sl_step(self.handle, splitting, dt, nsteps)

    def mass(self) -> float:
        return sl_mass(self.handle)

    def graph_capture(self, splitting, dt, nsteps):
        sl_graph_capture(self.handle, splitting, dt, nsteps)

    def graph_launch(self):
        sl_graph_launch(self.handle)

    def synchronize(self):
        sl_synchronize(self.handle)

    def autotune(self, reps=3):
        sl_autotune(self.handle, reps)

    def get_tune(self, dim):
        return sl_get_tune(self.handle, dim)

    def set_tune(self, dim, **kw):
        sl_set_tune(self.handle, dim, **kw)

    def profile_enable(self, on=True):
        sl_profile_enable(self.handle, on)

    def profile_query(self):
        return sl_profile_query(self.handle)

    def profile_dims(self):
        return sl_profile_dims(self.handle)

    def graph_capture_advect(self, dim, shift_dim, shifts, nsteps):
        sl_graph_capture_advect(self.handle, dim, shift_dim, shifts, nsteps)

    def set_poisson(self, enable=True):
        sl_set_poisson(self.handle, enable)

    def set_nodal_velocity(self, enable=True):
        sl_set_nodal_velocity(self.handle, enable)

    def advect_nodal(self, dim, tau):
        sl_advect_nodal(self.handle, dim, tau)

    def set_arithmetic(self, arith):
        sl_set_arithmetic(self.handle, arith)

    def check_guards(self):
        return sl_check_guards(self.handle)

    def field(self):
        nx = [n for n, pr in zip(self.grid.n, self.grid.pair) if pr >= 0][0]
        return sl_get_field(self.handle, nx)

    def field_energy(self):
        return sl_field_energy(self.handle)


# ---------------------------------------------------------------------------
# batches


def _bcheck(status: int, b):
    if status != SL_OK:
        r = lib().sl_batch_last_error(b)
        raise SlError(status, r.decode() if r else "")


def sl_batch_create(grids, degrees, storage, stream=None):
    n = len(grids)
    arr = (sl_grid * n)(*[make_grid(g) for g in grids])
    deg = (ctypes.c_int * n)(*[int(d) for d in degrees])
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    out = _vp()
    _check(lib().sl_batch_create(n, arr, deg, st, _stream_handle(stream), ctypes.byref(out)))
    return out


def sl_batch_destroy(b):
    if b:
        lib().sl_batch_destroy(b)


def sl_batch_last_error(b=None) -> str:
    r = lib().sl_batch_last_error(b)
    return r.decode() if r else ""


def sl_batch_info(b):
    c, d, s = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _bcheck(lib().sl_batch_info(b, ctypes.byref(c), ctypes.byref(d), ctypes.byref(s)), b)
    return {"cells": c.value, "dof": d.value, "state_bytes": s.value}


def sl_batch_project(b, prob, nq, weights, params):
    w = _f64(weights)
    p = _f64(params)
    _bcheck(lib().sl_batch_project(b, int(prob), int(nq), int(w.size), _ptr(w), _ptr(p)), b)


def sl_batch_set_coeffs(b, prob, u):
    u_ = _f64(u)
    _bcheck(lib().sl_batch_set_coeffs(b, int(prob), _ptr(u_)), b)


def sl_batch_get_coeffs(b, prob, cells, ncoef):
    out = np.empty((cells, ncoef))
    _bcheck(lib().sl_batch_get_coeffs(b, int(prob), _ptr(out)), b)
    return out


def sl_batch_set_fields(b, fields):
    f = _f64(np.concatenate([np.ravel(x) for x in fields])) if len(fields) else np.zeros(0)
    _bcheck(lib().sl_batch_set_fields(b, _ptr(f), f.size), b)


def sl_batch_step(b, splitting, dt, nsteps):
    _bcheck(lib().sl_batch_step(b, _split(splitting), float(dt), int(nsteps)), b)


def sl_batch_mass(b, nprob):
    out = np.empty(nprob)
    _bcheck(lib().sl_batch_mass(b, _ptr(out)), b)
    return out


def sl_batch_graph_capture(b, splitting, dt, nsteps):
    _bcheck(lib().sl_batch_graph_capture(b, _split(splitting), float(dt), int(nsteps)), b)


def sl_batch_graph_launch(b):
    _bcheck(lib().sl_batch_graph_launch(b), b)


def sl_batch_synchronize(b):
    _bcheck(lib().sl_batch_synchronize(b), b)


def sl_batch_autotune(b, reps=3):
    _bcheck(lib().sl_batch_autotune(b, int(reps)), b)


def sl_batch_profile_enable(b, enable=True):
    _bcheck(lib().sl_batch_profile_enable(b, 1 if enable else 0), b)


def sl_batch_profile_query(b):
    n, ms, by = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    _bcheck(lib().sl_batch_profile_query(b, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)), b)
    return n.value, ms.value, by.value


def sl_batch_profile_dims(b):
    n = (ctypes.c_int64 * MAX_DIM)()
    ms = (ctypes.c_double * MAX_DIM)()
    _bcheck(lib().sl_batch_profile_dims(b, n, ms), b)
    return list(n), list(ms)


def sl_batch_get_tune(b, dim: int):
    t = sl_tune()
    _bcheck(lib().sl_batch_get_tune(b, int(dim), ctypes.byref(t)), b)
    return dict(block=t.block, fibres_per_thread=t.fibres_per_thread, unroll=t.unroll,
                pipeline=t.pipeline, chunk=t.chunk)


def sl_batch_set_tune(b, dim: int, fibres_per_thread: int, unroll: int, chunk: int, block: int = 128,
                      pipeline: int = 0, max_blocks_per_sm: int = 0):
    t = sl_tune(int(block), int(fibres_per_thread), int(unroll), int(pipeline), int(chunk),
                int(max_blocks_per_sm), 0)
    _bcheck(lib().sl_batch_set_tune(b, int(dim), ctypes.byref(t)), b)


class Batch:
    """Owns one sl_batch handle for a list of problems (objects with .grid, .k)."""

    def __init__(self, grids, degrees, storage, stream=None):
        self.grids = list(grids)
        self.degrees = list(degrees)
        self.handle = sl_batch_create(self.grids, self.degrees, storage, stream)
        self.info = sl_batch_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            sl_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def project(self, prob, nq, weights, params):
        sl_batch_project(self.handle, prob, nq, weights, params)

    def set_coeffs(self, prob, u):
        sl_batch_set_coeffs(self.handle, prob, u)

    def get_coeffs(self, prob):
        g = self.grids[prob]
        cells = int(np.prod(g.n))
        return sl_batch_get_coeffs(self.handle, prob, cells, (self.degrees[prob] + 1) ** len(g.n))

    def set_fields(self, fields):
        sl_batch_set_fields(self.handle, fields)

    def step(self, splitting, dt, nsteps=1):
        sl_batch_step(self.handle, splitting, dt, nsteps)

    def mass(self):
        return sl_batch_mass(self.handle, len(self.grids))

    def graph_capture(self, splitting, dt, nsteps):
        sl_batch_graph_capture(self.handle, splitting, dt, nsteps)

    def graph_launch(self):
        sl_batch_graph_launch(self.handle)

    def synchronize(self):
        sl_batch_synchronize(self.handle)

    def autotune(self, reps=3):
        sl_batch_autotune(self.handle, reps)

    def profile_enable(self, on=True):
        sl_batch_profile_enable(self.handle, on)

    def profile_query(self):
        return sl_batch_profile_query(self.handle)

    def profile_dims(self):
        return sl_batch_profile_dims(self.handle)

    def get_tune(self, dim):
        return sl_batch_get_tune(self.handle, dim)

    def set_tune(self, dim, **kw):
        sl_batch_set_tune(self.handle, dim, **kw)


from .state_io import autotune_cached, load_checkpoint, save_checkpoint  # noqa: E402
