"""The device-side binary32 <-> binary64 conversions of the mean row (integer
pipe forms) against IEEE 754 round-to-nearest-even conversions on the host,
bit for bit outside the binary32 subnormal range, on random values and the
edge cases of both formats; inside it, the documented flush (to a signed zero,
or below 2^-126 for float to double)."""
import numpy as np
import pytest

import paper_1603_07008_gb300 as S

pytestmark = pytest.mark.gpu


def _bits32(x):
    return np.asarray(x, dtype=np.float32).view(np.uint32)


def _bits64(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def _doubles():
    rng = np.random.default_rng(7)
    f32 = np.finfo(np.float32)
    base = [0.0, -0.0, 1.0, -1.0, 1.5, np.pi, 1e-3, 0.37, 2.0 ** -126, 2.0 ** -127, 2.0 ** -149,
            2.0 ** -150, 1e-45, 1e-300, 5e-324, float(f32.max), -float(f32.max), 3.5e38, 1e300,
            np.inf, -np.inf, np.nan]
    # exact ties between two binary32 values: mantissa bit 28 of the 29 dropped bits set, rest zero
    ties = []
    for m in (0, 1, 2, 3, 0x7FFFFF):
        for e in (-100, -1, 0, 1, 60, 127):
            x = np.float64((1.0 + m * 2.0 ** -23 + 2.0 ** -24) * 2.0 ** e)
            ties += [x, -x, np.nextafter(x, np.inf), np.nextafter(x, -np.inf)]
    # largest finite double that rounds to FLT_MAX, and the one above (overflow to inf)
    ties += [float(f32.max) * (1 + 2.0 ** -25), float(f32.max) * (1 + 2.0 ** -24)]
    rnd = rng.standard_normal(20000) * np.exp2(rng.integers(-140, 130, 20000))
    bits = rng.integers(0, 2 ** 63, 20000, dtype=np.int64).astype(np.uint64).view(np.float64)
    return np.concatenate([base, ties, rnd, bits[np.isfinite(bits)]]).astype(np.float64)


def _floats(n):
    rng = np.random.default_rng(8)
    f32 = np.finfo(np.float32)
    base = np.array([0.0, -0.0, 1.0, -2.5, f32.max, -f32.max, f32.tiny, f32.tiny / 2, 1e-45, -1e-45,
                     np.inf, -np.inf, np.nan], dtype=np.float32)
    rnd = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32).view(np.float32)
    out = np.concatenate([base, rnd])[:n]
    return np.resize(out, n)


def test_conversions_match_ieee_round_to_nearest_even():
    d = _doubles()
    f = _floats(d.size)
    with np.errstate(over="ignore"):
        want_pos = d.astype(np.float32)
        want_neg = (-d).astype(np.float32)
    got_pos, got_neg, got_d, mism = S.sl_selftest_conversions(d, f)
    assert mism == 0     # the branching and branch-free forms agree bit for bit
    tiny = np.float64(np.finfo(np.float32).tiny)                 # 2^-126
    nan_p = np.isnan(want_pos)
    assert np.array_equal(np.isnan(got_pos), nan_p) and np.array_equal(np.isnan(got_neg), np.isnan(want_neg))
    sub = (np.abs(d) < tiny) & (d != 0)                           # results in the subnormal range
    keep = ~nan_p & ~sub
    assert np.array_equal(_bits32(got_pos[keep]), _bits32(want_pos[keep]))
    assert np.array_equal(_bits32(got_neg[keep]), _bits32(want_neg[keep]))
    assert np.all(got_pos[sub] == 0) and np.array_equal(np.signbit(got_pos[sub]), np.signbit(d[sub]))
    assert np.all(got_neg[sub] == 0) and np.array_equal(np.signbit(got_neg[sub]), ~np.signbit(d[sub]))
    want_d = f.astype(np.float64)
    nan_d = np.isnan(want_d)
    assert np.array_equal(np.isnan(got_d), nan_d)
    subf = (np.abs(f) < np.finfo(np.float32).tiny) & (f != 0)   # subnormal inputs
    keep = ~nan_d & ~subf
    assert np.array_equal(_bits64(got_d[keep]), _bits64(want_d[keep]))
    assert np.all(np.abs(got_d[subf]) < tiny) and np.array_equal(np.signbit(got_d[subf]), np.signbit(f[subf]))


def test_conversion_selftest_rejects_bad_sizes():
    with pytest.raises(ValueError):
        S.sl_selftest_conversions(np.zeros(3), np.zeros(2, np.float32))
    st = S.lib().sl_selftest_conversions(None, None, 0, None, None, None)
    assert st == S.SL_EINVAL


def test_widened_difference_is_the_fp64_subtraction():
    """The mean row's difference of two widened per-cell FP32 sums, formed on
    the integer pipe when exact: bit for bit the IEEE FP64 subtraction of the
    widened values (outside the binary32 subnormal range), on neighbour-like
    pairs (close values, every sign), pairs 0..40 binades apart, equal values,
    zeros, extremes, infinities and NaN."""
    rng = np.random.default_rng(9)
    n = 100000
    x = (rng.standard_normal(n) * np.exp2(rng.integers(-120, 120, n))).astype(np.float32)
    near = (x * (1 + rng.standard_normal(n) * np.exp2(rng.integers(-24, 0, n)))).astype(np.float32)
    far = (x * np.exp2(rng.integers(-40, 41, n)) * rng.choice([-1.0, 1.0], n)).astype(np.float32)
    f32 = np.finfo(np.float32)
    special = np.array([0.0, -0.0, 1.0, -1.0, f32.max, -f32.max, f32.tiny, -f32.tiny, np.inf, -np.inf, np.nan,
                        2.0 ** 100, 2.0 ** -100], dtype=np.float32)
    sa, sb = np.meshgrid(special, special)
    a = np.concatenate([x, x, x, sa.ravel()])
    b = np.concatenate([near, far, x, sb.ravel()])
    out, mism = S.sl_selftest_sub_widened(a, b)
    assert mism == 0
    want = a.astype(np.float64) - b.astype(np.float64)
    normal = (np.abs(a) >= f32.tiny) | (a == 0) | ~np.isfinite(a)
    normal &= (np.abs(b) >= f32.tiny) | (b == 0) | ~np.isfinite(b)
    ok = normal & ~np.isnan(want)
    assert np.array_equal(_bits64(out[ok]), _bits64(want[ok]))
    assert np.all(np.isnan(out[np.isnan(want) & normal]))
