"""CPU FP64 oracle for the sLdG projection sweep (Einkemmer, arXiv:1603.07008).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
and the CPU-baseline leg of the benchmark may import this package.  It shares
no code with the CUDA library and never receives values computed there.

The arithmetic lives in plain C (``sl_oracle.c``, FP64, built with
``-ffp-contract=off``).  This module compiles and loads it with ctypes and
adds the host-side pieces that are plain bookkeeping:

* ``schedule``      -- the order of one-dimensional sweeps in a split step
                       (Sec. II: time splitting reduces the Vlasov equation to
                       one-dimensional advections, eq. (advection)).  Reading:
                       Strang = x-dims with dt/2, v-dims with dt, x-dims with
                       dt/2; Lie = x-dims then v-dims, each with dt; the
                       x-sweep along m uses the cell-centre velocity of its
                       paired v-dimension, the v-sweep uses E_m(x_m).
* ``sample_after``  -- coefficients of a few cells after a sequence of sweeps
                       on a grid too big to hold: every sweep needs only two
                       source cells per target cell (Sec. II-A, locality),
                       so the dependency cone is evaluated cell by cell.

Functions and the paper passages they follow:
  gauss_legendre, legendre   -- Gauss-Legendre quadrature used by eq. (cj)
  shift_split                -- integer/fractional part of the CFL number (Sec. II-A)
  ab_matrices                -- A, B of the update rule (Sec. II-A)
  sweep                      -- update rule applied along one dimension (Sec. II-A)
  bruteforce_sweep           -- translate + L2-project without A, B (Sec. II-A)
  project / project_cells    -- eq. (cj)
  mass                       -- c0 is the cell mean (Sec. II-A, III-A)
  step                       -- split time step (Sec. II)
  poisson_field, vp_step     -- self-consistent field of the Vlasov equation of
                                Sec. II in 1+1 dimensions (reading: d_x E =
                                rho - rho_bar, rho = int f dv) and the split
                                step that recomputes it before every v-sweep
  sweep_nodal,               -- x-sweep with the velocity at the Gauss nodes of
  bruteforce_nodal,             every v-cell (reading of v d_x f with v varying
  node_sigma,                   inside a v-cell), the same without A, B, and its
  apply_cell_nodal              per-cell form for the dependency cones of
                                sample_after
  fp64_coefficients,         -- which coefficients a store of "# double" = q
  storage_bytes,                keeps in FP64 (Sec. III-A, Tables II-VI;
  round_storage,                reading for d > 1: every index j_m < q), its
  stored_sweeps                 bytes per cell, the state as that store holds
                                it, and sweeps with the state rounded to the
                                store after each (FP64 arithmetic)
  l2_norm, rel_l2, rel_max   -- error measures; l2_norm is the function-space
                                L2 norm of the expansion, the reading of the
                                "discrete L2 norm" of Table II (Sec. III-A)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from typing import Dict, List, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsl_oracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.or_legendre.restype = ctypes.c_double
            L.or_legendre.argtypes = [ctypes.c_int, ctypes.c_double]
            L.or_gauss_legendre.restype = ctypes.c_int
            L.or_gauss_legendre.argtypes = [ctypes.c_int, _dp, _dp]
            L.or_shift_split.restype = None
            L.or_shift_split.argtypes = [ctypes.c_double, _i64p, _dp]
            L.or_ab_matrices.restype = ctypes.c_int
            L.or_ab_matrices.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp]
            L.or_sweep.restype = ctypes.c_int
            L.or_sweep.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   _dp, _dp, _dp]
            L.or_bruteforce_sweep.restype = ctypes.c_int
            L.or_bruteforce_sweep.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, _dp, ctypes.c_int, _dp, _dp]
            L.or_sweep_nodal.restype = ctypes.c_int
            L.or_sweep_nodal.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp]
            L.or_bruteforce_nodal.restype = ctypes.c_int
            L.or_bruteforce_nodal.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                              _dp, _dp]
            L.or_project.restype = ctypes.c_int
            L.or_project.argtypes = [ctypes.c_int, _i64p, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, _dp, _dp, _i64p, ctypes.c_int64, _dp]
            L.or_mass.restype = ctypes.c_double
            L.or_mass.argtypes = [ctypes.c_int, _i64p, _dp, _dp, ctypes.c_int, _dp]
            L.or_node_sigma.restype = ctypes.c_int
            L.or_node_sigma.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int64, _i64p]
            L.or_apply_cell_nodal.restype = ctypes.c_int
            L.or_apply_cell_nodal.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                              ctypes.POINTER(_dp), ctypes.POINTER(_dp), _dp]
            L.or_apply_cell.restype = ctypes.c_int
            L.or_apply_cell.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp,
                                        _dp, _dp]
            L.or_set_mutation.restype = None
            L.or_set_mutation.argtypes = [ctypes.c_int]
            L.or_get_mutation.restype = ctypes.c_int
            L.or_get_mutation.argtypes = []
            _lib = L
    return _lib


def _p(a: np.ndarray, t=_dp):
    return a.ctypes.data_as(t)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int64)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


# --------------------------------------------------------------------------
# scalar pieces
# --------------------------------------------------------------------------

class planted_mistake:
    """Context manager for the test of the pins: inside it the C oracle runs
    with planted mistake m (see MUTATION m in sl_oracle.c); 0 is the oracle."""

    def __init__(self, m: int):
        self.m = int(m)

    def __enter__(self):
        lib().or_set_mutation(self.m)
        return self

    def __exit__(self, *exc):
        lib().or_set_mutation(0)
        return False


def legendre(j: int, x: float) -> float:
    return lib().or_legendre(j, float(x))


def gauss_legendre(n: int) -> Tuple[np.ndarray, np.ndarray]:
    x = np.zeros(n)
    w = np.zeros(n)
    _check(lib().or_gauss_legendre(n, _p(x), _p(w)), "gauss_legendre")
    return x, w


def shift_split(s: float) -> Tuple[int, float]:
    sg = ctypes.c_int64()
    a = ctypes.c_double()
    lib().or_shift_split(float(s), ctypes.byref(sg), ctypes.byref(a))
    return sg.value, a.value


def ab_matrices(k: int, alpha: float) -> Tuple[np.ndarray, np.ndarray]:
    o = k + 1
    A = np.zeros((o, o))
    B = np.zeros((o, o))
    _check(lib().or_ab_matrices(k, float(alpha), _p(A), _p(B)), "ab_matrices")
    return A, B


# --------------------------------------------------------------------------
# whole-grid operations; u is [cells, o^d] float64, dimension 0 fastest
# --------------------------------------------------------------------------

def sweep(u: np.ndarray, n: Sequence[int], k: int, dim: int, shift_dim: int,
          shifts) -> np.ndarray:
    n_ = _i64(n)
    u_ = _f64(u)
    s_ = _f64(np.atleast_1d(shifts))
    expect = 1 if shift_dim < 0 else int(n_[shift_dim])
    if s_.size != expect:
        raise ValueError(f"expected {expect} shifts, got {s_.size}")
    out = np.empty_like(u_)
    _check(lib().or_sweep(len(n_), _p(n_, _i64p), k, dim, shift_dim, _p(s_), _p(u_), _p(out)),
           "sweep")
    return out


def bruteforce_sweep(u: np.ndarray, n: Sequence[int], k: int, dim: int, shift_dim: int,
                     shifts, nq: int = 12) -> np.ndarray:
    n_ = _i64(n)
    u_ = _f64(u)
    s_ = _f64(np.atleast_1d(shifts))
    out = np.empty_like(u_)
    _check(lib().or_bruteforce_sweep(len(n_), _p(n_, _i64p), k, dim, shift_dim, _p(s_), nq,
                                     _p(u_), _p(out)), "bruteforce_sweep")
    return out


def _nodal_args(grid, dim: int, tau: float):
    vdim = grid.pair[dim]
    if vdim < 0:
        raise ValueError(f"dimension {dim} has no paired v-dimension")
    h = [(grid.hi[m] - grid.lo[m]) / grid.n[m] for m in range(len(grid.n))]
    return vdim, float(grid.lo[vdim]), h[vdim], float(tau) / h[dim]


def sweep_nodal(u: np.ndarray, grid, k: int, dim: int, tau: float) -> np.ndarray:
    """x-sweep along `dim` over time tau with the velocity of the paired
    v-dimension taken at the o Gauss-Legendre nodes of every v-cell (see
    or_sweep_nodal)."""
    n_ = _i64(grid.n)
    u_ = _f64(u)
    vdim, vlo, hv, toh = _nodal_args(grid, dim, tau)
    out = np.empty_like(u_)
    _check(lib().or_sweep_nodal(len(n_), _p(n_, _i64p), k, dim, vdim, vlo, hv, toh, _p(u_), _p(out)),
           "sweep_nodal")
    return out


def node_sigma(grid, k: int, dim: int, tau: float, j: int) -> List[int]:
    """sigma_q of the o node shifts of v-cell j in the nodal x-sweep along dim."""
    vdim, vlo, hv, toh = _nodal_args(grid, dim, tau)
    out = np.zeros(k + 1, dtype=np.int64)
    _check(lib().or_node_sigma(k, vlo, hv, toh, int(j), _p(out, _i64p)), "node_sigma")
    return [int(x) for x in out]


def apply_cell_nodal(grid, k: int, dim: int, tau: float, j: int, ua, ub) -> np.ndarray:
    """New coefficients of one cell of v-cell j in the nodal x-sweep along dim
    from its source cells: ua[q], ub[q] the coefficients of the cells
    i - sigma_q and i - sigma_q - 1 (the same bits as sweep_nodal)."""
    vdim, vlo, hv, toh = _nodal_args(grid, dim, tau)
    o = k + 1
    a_ = [_f64(x) for x in ua]
    b_ = [_f64(x) for x in ub]
    pa = (_dp * o)(*[_p(x) for x in a_])
    pb = (_dp * o)(*[_p(x) for x in b_])
    out = np.empty_like(a_[0])
    _check(lib().or_apply_cell_nodal(len(grid.n), k, dim, vdim, vlo, hv, toh, int(j), pa, pb, _p(out)),
           "apply_cell_nodal")
    return out


def bruteforce_nodal(u: np.ndarray, grid, k: int, dim: int, tau: float, nq: int = 12) -> np.ndarray:
    n_ = _i64(grid.n)
    u_ = _f64(u)
    vdim, vlo, hv, toh = _nodal_args(grid, dim, tau)
    out = np.empty_like(u_)
    _check(lib().or_bruteforce_nodal(len(n_), _p(n_, _i64p), k, dim, vdim, vlo, hv, toh, nq, _p(u_),
                                     _p(out)), "bruteforce_nodal")
    return out


def project(grid, k: int, nq: int, weights, params) -> np.ndarray:
    """Coefficients of all cells, eq. (cj), of u0 = sum_t w_t prod_m g_{t,m}."""
    return project_cells(grid, k, nq, weights, params, None)


def project_cells(grid, k: int, nq: int, weights, params, cells) -> np.ndarray:
    n_ = _i64(grid.n)
    lo = _f64(grid.lo)
    hi = _f64(grid.hi)
    w_ = _f64(weights)
    p_ = _f64(params)
    nterms = w_.size
    if p_.shape != (nterms, len(n_), 4):
        raise ValueError("params must be [nterms, ndim, 4]")
    ncoef = (k + 1) ** len(n_)
    if cells is None:
        total = int(np.prod(n_))
        out = np.empty((total, ncoef))
        cp = None
        nc = total
    else:
        c_ = _i64(cells)
        out = np.empty((c_.size, ncoef))
        cp = _p(c_, _i64p)
        nc = c_.size
    _check(lib().or_project(len(n_), _p(n_, _i64p), _p(lo), _p(hi), k, nq, nterms, _p(w_),
                            _p(p_), cp, nc, _p(out)), "project")
    return out


def mass(u: np.ndarray, grid, k: int) -> float:
    n_ = _i64(grid.n)
    u_ = _f64(u)
    return lib().or_mass(len(n_), _p(n_, _i64p), _p(_f64(grid.lo)), _p(_f64(grid.hi)), k, _p(u_))


def apply_cell(ndim: int, k: int, dim: int, A, B, ua, ub) -> np.ndarray:
    A_, B_, a_, b_ = _f64(A), _f64(B), _f64(ua), _f64(ub)
    out = np.empty_like(a_)
    _check(lib().or_apply_cell(ndim, k, dim, _p(A_), _p(B_), _p(a_), _p(b_), _p(out)),
           "apply_cell")
    return out


# --------------------------------------------------------------------------
# splitting schedule and time stepping (host bookkeeping)
# --------------------------------------------------------------------------

def line_shifts(grid, dim: int, tau: float, fields: Sequence[np.ndarray]):
    """(shift_dim, shifts in cells) of the sweep along `dim` over time tau.

    x-dim m (pair[m] = p >= 0): velocity = cell centre of v-dim p,
        v_j = lo_p + (j + 1/2) h_p; shift = v_j * tau / h_m, one per v-line.
    v-dim p (= pair[m] of x-dim m): velocity = E_m at the x_m cell centres;
        shift = E * tau / h_p, one per x_m-line.  fields are ordered by x-dim."""
    ndim = len(grid.n)
    h = [(grid.hi[m] - grid.lo[m]) / grid.n[m] for m in range(ndim)]
    xd = [m for m in range(ndim) if grid.pair[m] >= 0]
    if grid.pair[dim] >= 0:
        p = grid.pair[dim]
        v = grid.lo[p] + (np.arange(grid.n[p], dtype=np.float64) + 0.5) * h[p]
        return p, v * tau / h[dim]
    for idx, m in enumerate(xd):
        if grid.pair[m] == dim:
            E = _f64(fields[idx])
            return m, E * tau / h[dim]
    raise ValueError(f"dimension {dim} is neither an x- nor a v-dimension")


def schedule(grid, splitting: str, dt: float, fields) -> List[Tuple[int, int, np.ndarray]]:
    """List of (dim, shift_dim, shifts) for one split time step."""
    xd = [m for m in range(len(grid.n)) if grid.pair[m] >= 0]
    vd = [grid.pair[m] for m in xd]
    if splitting == "strang":
        plan = [(m, 0.5 * dt) for m in xd] + [(p, dt) for p in vd] + [(m, 0.5 * dt) for m in xd]
    elif splitting == "lie":
        plan = [(m, dt) for m in xd] + [(p, dt) for p in vd]
    else:
        raise ValueError(f"unknown splitting {splitting!r}")
    out = []
    for dim, tau in plan:
        sd, s = line_shifts(grid, dim, tau, fields)
        out.append((dim, sd, s))
    return out


def schedule_nodal(grid, splitting: str, dt: float, fields) -> List[tuple]:
    """schedule() with every x-sweep a nodal one: ("nodal", dim, tau) in place
    of (dim, shift_dim, shifts) for the x-dimensions."""
    sched = schedule(grid, splitting, dt, fields)
    taus = _plan_taus(grid, splitting, dt)
    return [("nodal", dim, tau) if grid.pair[dim] >= 0 else (dim, sd, s)
            for (dim, sd, s), tau in zip(sched, taus)]


def step(u: np.ndarray, grid, k: int, splitting: str, dt: float, nsteps: int, fields,
         nodal_v: bool = False) -> np.ndarray:
    """nsteps split steps; nodal_v: the x-sweeps take the velocity at the
    Gauss nodes of every v-cell (sweep_nodal) instead of its centre."""
    sched = schedule(grid, splitting, dt, fields)
    taus = _plan_taus(grid, splitting, dt)
    for _ in range(nsteps):
        for (dim, sd, s), tau in zip(sched, taus):
            if nodal_v and grid.pair[dim] >= 0:
                u = sweep_nodal(u, grid, k, dim, tau)
            else:
                u = sweep(u, grid.n, k, dim, sd, s)
    return u


def _plan_taus(grid, splitting: str, dt: float) -> List[float]:
    xd = [m for m in range(len(grid.n)) if grid.pair[m] >= 0]
    if splitting == "strang":
        return [0.5 * dt] * len(xd) + [dt] * len(xd) + [0.5 * dt] * len(xd)
    return [dt] * (2 * len(xd))


# --------------------------------------------------------------------------
# split storage: "# double" of Sec. III-A (Table II and Tables III-VI)
# --------------------------------------------------------------------------

def fp64_coefficients(k: int, ndim: int, ndouble: int) -> np.ndarray:
    """Boolean mask over the o^d coefficients J = sum_m j_m o^m of a cell:
    True for those a store of "# double" = ndouble keeps in FP64.  Sec. III-A
    counts, in one dimension, the coefficients c_0 .. c_{q-1} stored in double
    precision (q = 1: only the cell mean).  Reading for d dimensions: the
    tensor-product coefficients with every per-dimension index j_m < q."""
    o = k + 1
    if not 0 <= ndouble <= o:
        raise ValueError(f"# double must be in 0..{o}")
    mask = np.ones(o ** ndim, dtype=bool)
    for J in range(o ** ndim):
        r = J
        for _ in range(ndim):
            mask[J] &= (r % o) < ndouble
            r //= o
    return mask


def storage_bytes(k: int, ndim: int, ndouble: int) -> int:
    """Bytes per cell of that store: 8 per FP64 and 4 per FP32 coefficient."""
    n64 = int(fp64_coefficients(k, ndim, ndouble).sum())
    return 8 * n64 + 4 * ((k + 1) ** ndim - n64)


def round_storage(u: np.ndarray, k: int, ndim: int, ndouble: int) -> np.ndarray:
    """The state [cells, o^d] as that store holds it: FP64 coefficients as
    they are, the others rounded to FP32 (round to nearest, ties to even)."""
    mask = fp64_coefficients(k, ndim, ndouble)
    v = np.array(u, dtype=np.float64, copy=True)
    v[:, ~mask] = v[:, ~mask].astype(np.float32).astype(np.float64)
    return v


def stored_sweeps(u: np.ndarray, n: Sequence[int], k: int, ndouble: int, sweeps) -> np.ndarray:
    """Apply sweeps (dim, shift_dim, shifts) in turn, each in FP64, rounding
    the state to the store of "# double" = ndouble after every sweep: what a
    store of that precision holds when its arithmetic is exact."""
    u = round_storage(u, k, len(n), ndouble)
    for dim, sd, s in sweeps:
        u = round_storage(sweep(u, n, k, dim, sd, s), k, len(n), ndouble)
    return u


def _vp_dims(grid):
    if len(grid.n) == 2:
        for m in (0, 1):
            if grid.pair[m] == 1 - m and grid.pair[1 - m] < 0:
                return m, 1 - m
    raise ValueError("the self-consistent field needs one x and one v dimension")


def poisson_field(u: np.ndarray, grid, k: int) -> np.ndarray:
    """E at the x-cell centres for d_x E = rho - rho_bar on the periodic
    x-domain, int E dx = 0.  rho_i = h_v sum_j c_{i,j;0} is the x-cell average
    of int f dv; E is the field of that piecewise-constant density at the
    cell centres: sum_{j<i} q_j + q_i / 2 with q = (rho - rho_bar) h_x, minus
    its mean.  Sums run one after the other in index order."""
    x, v = _vp_dims(grid)
    nx, nv = grid.n[x], grid.n[v]
    hx = (grid.hi[x] - grid.lo[x]) / nx
    hv = (grid.hi[v] - grid.lo[v]) / nv
    c0 = u[:, 0].reshape(grid.n[1], grid.n[0])      # [index along dim 1][index along dim 0]
    rho = np.zeros(nx)
    for i in range(nx):
        s = 0.0
        for j in range(nv):
            s += c0[j, i] if x == 0 else c0[i, j]
        rho[i] = hv * s
    rho_bar = sum(rho) / nx
    q = (rho - rho_bar) * hx
    E = np.empty(nx)
    run = 0.0
    for i in range(nx):
        E[i] = run + 0.5 * q[i]
        run += q[i]
    return E - sum(E) / nx


def field_energy(E: np.ndarray, grid) -> float:
    """(1/2) sum_i E_i^2 h_x."""
    x, _ = _vp_dims(grid)
    return 0.5 * (grid.hi[x] - grid.lo[x]) / grid.n[x] * float(np.sum(np.asarray(E) ** 2))


def vp_step(u: np.ndarray, grid, k: int, splitting: str, dt: float, nsteps: int, energies=None) -> np.ndarray:
    """Split steps with the field recomputed from the state before every
    v-sweep; appends the field energy of the state after every step to
    `energies` if given."""
    x, v = _vp_dims(grid)
    for _ in range(nsteps):
        for dim, tau in ([(x, 0.5 * dt), (v, dt), (x, 0.5 * dt)] if splitting == "strang"
                         else [(x, dt), (v, dt)]):
            fields = [poisson_field(u, grid, k)] if dim == v else [np.zeros(grid.n[x])]
            sd, s = line_shifts(grid, dim, tau, fields)
            u = sweep(u, grid.n, k, dim, sd, s)
        if energies is not None:
            energies.append(field_energy(poisson_field(u, grid, k), grid))
    return u


def sample_after(grid, k: int, nq: int, weights, params, sweeps, cells) -> np.ndarray:
    """Coefficients of the flat cells `cells` after applying `sweeps`
    (a list of (dim, shift_dim, shifts), or ("nodal", dim, tau) for a nodal
    x-sweep, as schedule and schedule_nodal give them) to the projected
    initial condition.
    Each target cell depends on two source cells of the previous stage, so
    the work is 2^len(sweeps) cells per sample at most (shared cells are
    computed once)."""
    n = [int(x) for x in grid.n]
    ndim = len(n)
    strides = [1] * ndim
    for m in range(1, ndim):
        strides[m] = strides[m - 1] * n[m - 1]
    # per sweep: per class sigma and matrices; a nodal sweep ("nodal", dim, tau)
    # keeps the node sigmas of each v-cell
    prepared = []
    for sw in sweeps:
        if sw[0] == "nodal":
            _, dim, tau = sw
            vdim = grid.pair[dim]
            prepared.append(("nodal", dim, (vdim, float(tau),
                                            [node_sigma(grid, k, dim, tau, j) for j in range(n[vdim])])))
            continue
        dim, sd, s = sw
        s = np.atleast_1d(np.asarray(s, dtype=np.float64))
        cls = []
        for val in s:
            sg, al = shift_split(float(val))
            A, B = ab_matrices(k, al)
            cls.append((sg, A, B))
        prepared.append((dim, sd, cls))

    memo: List[Dict[int, np.ndarray]] = [dict() for _ in range(len(sweeps) + 1)]

    def coord(c, m):
        return (c // strides[m]) % n[m]

    # collect the needed cells stage by stage (backwards), then evaluate forward
    def sources(stage, c):
        """[(cell a, cell b)] per node (nodal) or the one pair of cell c."""
        if stage[0] == "nodal":
            _, dim, (vdim, tau, sigs) = stage
            sg_list = sigs[coord(c, vdim)]
        else:
            dim, sd, cls = stage
            sg_list = [cls[0 if sd < 0 else coord(c, sd)][0]]
        i = coord(c, dim)
        out = []
        for sg in sg_list:
            ia = (i - sg) % n[dim]
            ib = (ia - 1) % n[dim]
            out.append((c + (ia - i) * strides[dim], c + (ib - i) * strides[dim]))
        return out

    need = [set() for _ in range(len(sweeps) + 1)]
    need[len(sweeps)] = set(int(c) for c in cells)
    for st in range(len(sweeps), 0, -1):
        for c in need[st]:
            for ca, cb in sources(prepared[st - 1], c):
                need[st - 1].add(ca)
                need[st - 1].add(cb)
    base = sorted(need[0])
    vals = project_cells(grid, k, nq, weights, params, base)
    for c, v in zip(base, vals):
        memo[0][c] = v
    for st in range(1, len(sweeps) + 1):
        stage = prepared[st - 1]
        for c in need[st]:
            pairs = sources(stage, c)
            if stage[0] == "nodal":
                _, dim, (vdim, tau, _) = stage
                memo[st][c] = apply_cell_nodal(grid, k, dim, tau, coord(c, vdim),
                                               [memo[st - 1][a] for a, _ in pairs],
                                               [memo[st - 1][b] for _, b in pairs])
            else:
                dim, sd, cls = stage
                _, A, B = cls[0 if sd < 0 else coord(c, sd)]
                ca, cb = pairs[0]
                memo[st][c] = apply_cell(ndim, k, dim, A, B, memo[st - 1][ca], memo[st - 1][cb])
    return np.stack([memo[len(sweeps)][int(c)] for c in cells])


# --------------------------------------------------------------------------
# error measures (function-space L2 of the Legendre expansion)
# --------------------------------------------------------------------------

def l2_weights(k: int, ndim: int) -> np.ndarray:
    """||P_j||^2 on [-1,1] is 2/(2j+1); a tensor-product coefficient J gets the
    product over dimensions (the cell-volume factor cancels in relative norms)."""
    o = k + 1
    w = np.ones(o ** ndim)
    for J in range(o ** ndim):
        r = J
        for _ in range(ndim):
            j = r % o
            r //= o
            w[J] *= 2.0 / (2 * j + 1)
    return w


def l2_norm(u: np.ndarray, grid, k: int) -> float:
    """Function-space L2 norm of the expansion on the grid's box:
    int u^2 dx = sum over cells of prod_m (h_m / 2) sum_J c_J^2 prod_m 2 / (2 j_m + 1)
    (each cell maps to [-1, 1]^d with Jacobian prod_m h_m / 2)."""
    ndim = len(grid.n)
    jac = 1.0
    for m in range(ndim):
        jac *= 0.5 * (grid.hi[m] - grid.lo[m]) / grid.n[m]
    v = np.asarray(u, dtype=np.float64)
    return math.sqrt(jac * float(np.sum(v * v * l2_weights(k, ndim))))


def rel_l2(u: np.ndarray, ref: np.ndarray, k: int, ndim: int) -> float:
    w = l2_weights(k, ndim)
    d = np.asarray(u, dtype=np.float64) - np.asarray(ref, dtype=np.float64)
    num = math.sqrt(float(np.sum(d * d * w)))
    den = math.sqrt(float(np.sum(np.asarray(ref, dtype=np.float64) ** 2 * w)))
    return num / den if den > 0 else num


def rel_max(u: np.ndarray, ref: np.ndarray) -> float:
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.max(np.abs(ref))) if ref.size else 0.0
    num = float(np.max(np.abs(np.asarray(u, dtype=np.float64) - ref))) if ref.size else 0.0
    return num / den if den > 0 else num
