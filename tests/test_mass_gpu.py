"""The FP64 mass M = (prod_m h_m) sum_i c_{i;0..0} (Sec. II-A, III-A: c_0 is
the cell mean) of every store that keeps the mean in FP64, and of a batch,
against the exact sum.

References: the correctly rounded sum of the means (math.fsum) times the cell
volume -- the exact mass to two roundings -- and the oracle's mass (a plain
left-to-right sum, whose rounding error is at most (n - 1) 2^-53 of the sum
for positive means).  The GPU reduction (fixed-shape tree) must lie within
1e-14 of the exact value; one case per store has more than 1024 x 256 x 8
cells, so the reduction runs at its cap of 1024 blocks with a grid-stride
loop.  A wrong cell-volume factor or a wrong plane fails these at once.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_1603_07008_gb300 as S
from paper_1603_07008_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BIG = (1536, 1400)   # 2 150 400 cells > 1024 * 256 * 8


def _grid(n):
    d = len(n)
    return W.Grid(n=tuple(n), lo=tuple(-1.3 + 0.1 * m for m in range(d)),
                  hi=tuple(2.9 + 0.7 * m for m in range(d)), pair=(-1,) * d)


def _state(n, k, seed):
    rng = np.random.default_rng(seed)
    u = W.random_coefficients(int(np.prod(n)), k, len(n), seed)
    u[:, 0] = rng.uniform(0.5, 1.5, u.shape[0])
    return u


def _exact(u, g):
    vol = 1.0
    for m in range(len(g.n)):
        vol *= (g.hi[m] - g.lo[m]) / g.n[m]
    return vol * math.fsum(u[:, 0].tolist())


def _check(got, u, g, k):
    exact = _exact(u, g)
    ref = O.mass(u, g, k)
    n = u.shape[0]
    assert abs(ref - exact) <= n * 2.0 ** -53 * abs(exact)          # the oracle's own bound
    assert abs(got - exact) <= 1e-14 * abs(exact), (got, exact)
    assert abs(got - ref) <= (1e-14 + n * 2.0 ** -53) * abs(ref), (got, ref)


@pytest.mark.parametrize("storage", ["fp64", "mix_fp32", "mix_bf16", "mix_fp16", "mix_fp32_d2"])
@pytest.mark.parametrize("n,k", [((7, 5), 2), ((33,), 1), ((6, 5, 4), 1), (BIG, 2)])
def test_mass_matches_the_exact_sum(storage, n, k):
    if storage == "mix_fp32_d2" and k < 2:
        pytest.skip("# double = 2 needs degree >= 2")
    g = _grid(n)
    u = _state(n, k, 21 + len(n))
    with S.Context(g, k, storage) as ctx:
        ctx.set_coeffs(u)
        held = ctx.get_coeffs()
        assert np.array_equal(held[:, 0], u[:, 0])   # the mean is stored exactly
        _check(ctx.mass(), u, g, k)
        # after sweeps the mass of the new state
        ctx.advect(0, -1, [0.37])
        ctx.advect(len(n) - 1, -1, [-1.61])
        _check(ctx.mass(), ctx.get_coeffs(), g, k)


def test_batch_mass_matches_the_exact_sum():
    grids = [_grid(BIG), _grid((100, 37)), _grid((64, 64)), _grid((5, 3))]
    for g in grids:
        object.__setattr__(g, "pair", (1, -1))
    degrees = [1, 2, 1, 2]
    with S.Batch(grids, degrees, "mix_fp32") as b:
        us = []
        for i, (g, k) in enumerate(zip(grids, degrees)):
            u = _state(g.n, k, 40 + i)
            b.set_coeffs(i, u)
            us.append(u)
        got = b.mass()
        for i, (g, k) in enumerate(zip(grids, degrees)):
            _check(got[i], us[i], g, k)
