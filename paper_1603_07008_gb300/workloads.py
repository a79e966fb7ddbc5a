"""Seeded synthetic workloads for the sLdG projection sweep.

This module only *describes* problems: grids, degrees, storage modes, time
steps, initial conditions as lists of separable factors, and electric-field
samples.  It holds none of the method's arithmetic (no projection, no shift
decomposition, no sweep): the CUDA library and the CPU oracle each turn these
descriptions into coefficients and sweeps with their own code.

Workloads follow the paper's setting (Sec. II: the Vlasov equation reduced by
time splitting to one-dimensional advections; Sec. II-A: degree-p Legendre
modal basis per cell) at the sizes of the five configurations this library is
measured on.  Initial conditions are sums of separable products

    u0(x) = sum_t w_t prod_m g_{t,m}(x_m),   g(x) = exp(-gamma (x-mu)^2) cos(kappa x + phi),

so every factor is the parameter quadruple (gamma, mu, kappa, phi).  Random
numbers (mode amplitudes, wave numbers, phases, problem sizes) come from
SplitMix64, a published 64-bit generator (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), so every run is reproducible.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "SplitMix64", "Grid", "Problem", "config1", "config2", "config3", "config4",
    "config5", "maxwellian_factor", "CONFIGS", "Table2Protocol", "table2_protocol",
]

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64: state += 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive), by rejection-free modulo of 64 bits."""
        return lo + self.next_u64() % (hi - lo + 1)


@dataclass
class Grid:
    """Periodic box [lo_m, hi_m) split into n_m cells per dimension; dimension 0
    is innermost in memory.  pair[m] = v-dimension advected together with
    x-dimension m (the x-sweep along m uses the v-cell-centre velocity, the
    v-sweep along pair[m] uses the field E_m(x_m)); -1 for v-dimensions and
    for dimensions without a partner."""
    n: Tuple[int, ...]
    lo: Tuple[float, ...]
    hi: Tuple[float, ...]
    pair: Tuple[int, ...]

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def cells(self) -> int:
        return int(np.prod(self.n, dtype=np.int64))

    def x_dims(self) -> List[int]:
        return [m for m in range(self.ndim) if self.pair[m] >= 0]

    def v_dims(self) -> List[int]:
        return [self.pair[m] for m in self.x_dims()]


@dataclass
class Problem:
    name: str
    grid: Grid
    k: int                       # polynomial degree p; o = k+1 coefficients per dimension
    storage: str                 # "fp64" | "mix_fp32" | "mix_bf16" | "mix_fp16"
    dt: float
    steps: int
    splitting: str               # "strang" | "lie" | "advect" (single constant-velocity sweep per step)
    weights: np.ndarray          # [nterms] float64
    params: np.ndarray           # [nterms, ndim, 4] float64: gamma, mu, kappa, phi
    nq: int = 5                  # Gauss points per dimension for the initial projection
    fields: dict = field(default_factory=dict)   # x-dim -> E samples at that dim's cell centres
    velocity: Optional[float] = None             # constant velocity for splitting == "advect"

    @property
    def o(self) -> int:
        return self.k + 1

    @property
    def ncoef(self) -> int:
        return self.o ** self.grid.ndim

    @property
    def dof(self) -> int:
        return self.grid.cells * self.ncoef

    def field_list(self) -> List[np.ndarray]:
        """Fields ordered by x-dimension index (the order the libraries take them)."""
        return [np.ascontiguousarray(self.fields[m], dtype=np.float64) for m in self.grid.x_dims()]


def maxwellian_factor() -> Tuple[float, Tuple[float, float, float, float]]:
    """(2 pi)^(-1/2) exp(-v^2/2) as (weight, factor)."""
    return 1.0 / math.sqrt(2.0 * math.pi), (0.5, 0.0, 0.0, 0.0)


ONE = (0.0, 0.0, 0.0, 0.0)   # the constant factor 1


def _cell_centres(n: int, lo: float, hi: float) -> np.ndarray:
    h = (hi - lo) / n
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * h


def _field(n: int, lo: float, hi: float, amp: float = 0.1, kx: float = 0.5) -> np.ndarray:
    """E(x) = amp * sin(kx * x) sampled at the cell centres."""
    return amp * np.sin(kx * _cell_centres(n, lo, hi))


def _terms_maxwellian_modes(nx: int, nv: int, modes: Sequence[Tuple[float, Sequence[float], float]]):
    """Maxwellian in every v-dimension times (1 + sum_r a_r cos(kappa_r . x + phi_r)).

    Each mode cos(sum_m kappa_m x_m + phi) is expanded into separable products
    by the angle-addition formula, one cosine factor per x-dimension with phase
    shifts of -pi/2 standing for sines.  Returns (weights, params)."""
    mw, mf = maxwellian_factor()
    vpart = [mf] * nv
    weights = [mw ** nv]
    params = [[ONE] * nx + vpart]
    for amp, kap, phi in modes:
        # cos(theta_0 + ... + theta_{nx-1} + phi) as sums of products of one
        # cosine factor per x-dimension: carry C = cos(partial sum) and
        # S = sin(partial sum) and add one angle at a time with
        #   C' = C cos b - S sin b,  S' = S cos b + C sin b,  sin y = cos(y - pi/2).
        C = [(1.0, [(0.0, 0.0, kap[0], phi)])]
        S = [(1.0, [(0.0, 0.0, kap[0], phi - math.pi / 2)])]
        for m in range(1, nx):
            cb = (0.0, 0.0, kap[m], 0.0)
            sb = (0.0, 0.0, kap[m], -math.pi / 2)
            C, S = ([(sg, f + [cb]) for sg, f in C] + [(-sg, f + [sb]) for sg, f in S],
                    [(sg, f + [cb]) for sg, f in S] + [(sg, f + [sb]) for sg, f in C])
        for sgn, facs in C:
            weights.append(sgn * amp * mw ** nv)
            params.append(list(facs) + vpart)
    return np.array(weights, dtype=np.float64), np.array(params, dtype=np.float64)


def _random_modes(rng: SplitMix64, nx: int, nmodes: int, amp: float):
    modes = []
    for _ in range(nmodes):
        a = amp * (2.0 * rng.uniform() - 1.0)
        kap = [0.5 * rng.randint(1, 2) for _ in range(nx)]
        phi = 2.0 * math.pi * rng.uniform()
        modes.append((a, kap, phi))
    return modes


FOUR_PI = 4.0 * math.pi


def config1() -> Problem:
    """1D advection u_t + u_x = 0 on periodic [0,1], N=1024, k=2, all FP64,
    dt = 0.37/N (fractional shift 0.37 cells), 100 steps,
    u0 = exp(-100 (x-1/2)^2) projected with 5-point Gauss."""
    n = 1024
    g = Grid(n=(n,), lo=(0.0,), hi=(1.0,), pair=(-1,))
    return Problem(name="1d_n1024_k2_fp64", grid=g, k=2, storage="fp64", dt=0.37 / n,
                   steps=100, splitting="advect",
                   weights=np.array([1.0]), params=np.array([[[100.0, 0.5, 0.0, 0.0]]]),
                   nq=5, velocity=1.0)


def _xv_grid(nx_cells: Sequence[int], nv_cells: Sequence[int]) -> Grid:
    nx, nv = len(nx_cells), len(nv_cells)
    n = tuple(nx_cells) + tuple(nv_cells)
    lo = (0.0,) * nx + (-6.0,) * nv
    hi = (FOUR_PI,) * nx + (6.0,) * nv
    pair = tuple(nx + m for m in range(nx)) + (-1,) * nv
    return Grid(n=n, lo=lo, hi=hi, pair=pair)


def _xv_fields(g: Grid) -> dict:
    return {m: _field(g.n[m], g.lo[m], g.hi[m]) for m in g.x_dims()}


def config2(n: int = 512, steps: int = 200, storage: str = "mix_fp32") -> Problem:
    """2D x-v split advection, n x n cells on [0,4pi) x [-6,6), k=2, Strang,
    dt = 0.1, E = 0.1 sin(x/2), u0 = Maxwellian(v) (1 + 0.01 cos(x/2))."""
    g = _xv_grid([n], [n])
    w, p = _terms_maxwellian_modes(1, 1, [(0.01, [0.5], 0.0)])
    return Problem(name=f"2d_xv_{n}x{n}_k2_{storage}", grid=g, k=2, storage=storage, dt=0.1,
                   steps=steps, splitting="strang", weights=w, params=p, nq=5,
                   fields=_xv_fields(g))


def config3(n: int = 64, steps: int = 20, storage: str = "mix_fp32", seed: int = 0) -> Problem:
    """4D (x1,x2,v1,v2) split advection, n^4 cells, k=2 tensor product, Strang,
    dt = 0.1, E_m = 0.1 sin(x_m/2), u0 = Maxwellian(v1) Maxwellian(v2) times
    (1 + four random modes of amplitude up to 1e-2)."""
    g = _xv_grid([n, n], [n, n])
    rng = SplitMix64(seed)
    w, p = _terms_maxwellian_modes(2, 2, _random_modes(rng, 2, 4, 1e-2))
    return Problem(name=f"4d_xxvv_{n}^4_k2_{storage}", grid=g, k=2, storage=storage, dt=0.1,
                   steps=steps, splitting="strang", weights=w, params=p, nq=5,
                   fields=_xv_fields(g))


def config4(nprob: int = 256, seed: int = 0, nmin: int = 64, nmax: int = 1024,
            steps: int = 10, storage: str = "mix_fp32") -> List[Problem]:
    """256 independent 2D x-v problems with N_x, N_v uniform in [64, 1024] and
    k uniform in {1, 2}, otherwise as the 2D workload."""
    rng = SplitMix64(seed)
    probs = []
    for b in range(nprob):
        nx = rng.randint(nmin, nmax)
        nv = rng.randint(nmin, nmax)
        k = rng.randint(1, 2)
        g = _xv_grid([nx], [nv])
        w, p = _terms_maxwellian_modes(1, 1, [(0.01, [0.5], 0.0)])
        probs.append(Problem(name=f"batch{b}_{nx}x{nv}_k{k}", grid=g, k=k, storage=storage,
                             dt=0.1, steps=steps, splitting="strang", weights=w, params=p,
                             nq=5, fields=_xv_fields(g)))
    return probs


def config5(n: int = 20, steps: int = 10, storage: str = "mix_bf16", seed: int = 0) -> Problem:
    """6D (x1,x2,x3,v1,v2,v3) split advection, n^6 cells, k=1 tensor product,
    Strang, dt = 0.1, E_m = 0.1 sin(x_m/2), u0 = Maxwellian^3 times
    (1 + four random low modes of amplitude up to 1e-2)."""
    g = _xv_grid([n] * 3, [n] * 3)
    rng = SplitMix64(seed)
    w, p = _terms_maxwellian_modes(3, 3, _random_modes(rng, 3, 4, 1e-2))
    return Problem(name=f"6d_xxxvvv_{n}^6_k1_{storage}", grid=g, k=1, storage=storage, dt=0.1,
                   steps=steps, splitting="strang", weights=w, params=p, nq=5,
                   fields=_xv_fields(g))


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}


@dataclass
class Table2Protocol:
    """The accuracy study of Table II (Sec. III-A): 10^4 steps of 1D periodic
    advection on [0, 1) with a constant shift per step, orders 2 and 4
    (k = 1, 3), a smooth and an oscillatory initial value.  The paper gives
    neither N nor the CFL number; n and shift are this library's choice."""
    n: int = 512
    steps: int = 10_000
    shift: float = 0.37
    nq: int = 8
    # profile -> (weights, params) of the separable form above
    initial: dict = field(default_factory=lambda: {
        # exp(-100 (x - 1/2)^2)
        "smooth": (np.array([1.0]), np.array([[[100.0, 0.5, 0.0, 0.0]]])),
        # 1 + cos(16 pi x + 0.3): eight periods on [0, 1), mass 1
        "oscillatory": (np.array([1.0, 1.0]),
                        np.array([[[0.0, 0.0, 0.0, 0.0]], [[0.0, 0.0, 2 * math.pi * 8, 0.3]]])),
    })

    def grid(self) -> "Grid":
        return Grid(n=(self.n,), lo=(0.0,), hi=(1.0,), pair=(-1,))


def table2_protocol(n: int = 512, steps: int = 10_000) -> Table2Protocol:
    return Table2Protocol(n=n, steps=steps)


def random_coefficients(cells: int, k: int, ndim: int, seed: int, decay: float = 0.1) -> np.ndarray:
    """Seeded random coefficient array [cells][(k+1)^ndim] with the c_j ~ h^j
    decay of smooth data (Sec. II-A): coefficient J gets the scale
    decay**(j_0 + ... + j_{d-1}).  Used for edge-case inputs where no smooth
    initial condition is wanted."""
    o = k + 1
    rng = np.random.default_rng(seed)
    deg = np.zeros(o ** ndim, dtype=np.int64)
    for J in range(o ** ndim):
        r = J
        for _ in range(ndim):
            deg[J] += r % o
            r //= o
    return rng.standard_normal((cells, o ** ndim)) * decay ** deg[None, :]
