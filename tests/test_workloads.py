"""The seeded workload descriptions: reproducible, and the separable
expansion of the random modes equals the modes themselves pointwise."""
import math

import numpy as np

from paper_1603_07008_gb300 import workloads as W


def _eval_terms(weights, params, x):
    """u0 at one point x (ndim,) from the separable description."""
    tot = 0.0
    for w, facs in zip(weights, params):
        prod = w
        for (g, mu, kap, phi), xm in zip(facs, x):
            prod *= math.exp(-g * (xm - mu) ** 2) * math.cos(kap * xm + phi)
        tot += prod
    return tot


def test_splitmix64_reference_values():
    # first outputs for seed 0 as published with the generator
    r = W.SplitMix64(0)
    assert r.next_u64() == 0xE220A8397B1DCDAF
    assert r.next_u64() == 0x6E789E6AA1B965F4
    assert r.next_u64() == 0x06C45D188009454F


def test_mode_expansion_is_pointwise_exact():
    p = W.config3(n=8)
    rng = W.SplitMix64(0)
    modes = W._random_modes(rng, 2, 4, 1e-2)
    pts = np.random.default_rng(0).uniform([0, 0, -6, -6], [4 * math.pi] * 2 + [6, 6], size=(20, 4))
    for x in pts:
        M = math.exp(-(x[2] ** 2 + x[3] ** 2) / 2) / (2 * math.pi)
        direct = M * (1 + sum(a * math.cos(k[0] * x[0] + k[1] * x[1] + ph) for a, k, ph in modes))
        assert abs(_eval_terms(p.weights, p.params, x) - direct) < 1e-15


def test_mode_expansion_6d():
    p = W.config5(n=4)
    rng = W.SplitMix64(0)
    modes = W._random_modes(rng, 3, 4, 1e-2)
    pts = np.random.default_rng(1).uniform([0] * 3 + [-6] * 3, [4 * math.pi] * 3 + [6] * 3, size=(10, 6))
    for x in pts:
        M = math.exp(-(x[3] ** 2 + x[4] ** 2 + x[5] ** 2) / 2) / (2 * math.pi) ** 1.5
        direct = M * (1 + sum(a * math.cos(sum(kk * xx for kk, xx in zip(k, x[:3])) + ph) for a, k, ph in modes))
        assert abs(_eval_terms(p.weights, p.params, x) - direct) < 1e-15


def test_batch_config_is_seeded():
    a = W.config4()
    b = W.config4()
    assert [(q.grid.n, q.k) for q in a] == [(q.grid.n, q.k) for q in b]
    assert len(a) == 256
    assert all(64 <= q.grid.n[0] <= 1024 and 64 <= q.grid.n[1] <= 1024 and q.k in (1, 2) for q in a)
