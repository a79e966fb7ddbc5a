"""Host-side checks of the C-ABI library: it builds, loads and exports every
symbol include/sl.h declares; its host logic (argument validation, the byte
model, the exact A/B tables) is right.  No device work is done here."""
import math
import os
import re
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import paper_1603_07008_gb300 as S
from paper_1603_07008_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "sl.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sl_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = S.lib()
    syms = _declared_symbols()
    assert len(syms) >= 19
    for s in syms:
        assert hasattr(L, s), s


def test_binding_covers_every_symbol():
    for s in _declared_symbols():
        assert callable(getattr(S, s)), s


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_ab_tables_match_oracle(k):
    rng = np.random.default_rng(k)
    for a in list(rng.uniform(0, 1, 40)) + [0.0, 1e-12, 0.5, 1 - 1e-12, 0.375]:
        A, B = S.sl_ab_host(k, a)
        Ao, Bo = O.ab_matrices(k, a)
        assert np.max(np.abs(A - Ao)) < 2e-15
        assert np.max(np.abs(B - Bo)) < 2e-15


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_ab_tables_exact_at_zero(k):
    A, B = S.sl_ab_host(k, 0.0)
    assert np.array_equal(A, np.eye(k + 1)) and not B.any()


def test_ab_tables_match_symbolic():
    sp = pytest.importorskip("sympy")
    xi = sp.Symbol("xi")
    for k in (2, 3):
        for fr in (Fraction(3, 8), Fraction(37, 100), Fraction(1, 7)):
            a = sp.Rational(fr.numerator, fr.denominator)
            A, B = S.sl_ab_host(k, float(fr))
            for j in range(k + 1):
                for l in range(k + 1):
                    Aj = sp.Rational(2 * j + 1, 2) * sp.integrate(
                        sp.legendre(j, xi) * sp.legendre(l, xi - 2 * a), (xi, 2 * a - 1, 1))
                    Bj = sp.Rational(2 * j + 1, 2) * sp.integrate(
                        sp.legendre(j, xi) * sp.legendre(l, xi + 2 - 2 * a), (xi, -1, 2 * a - 1))
                    assert abs(A[j, l] - float(Aj)) < 2e-15
                    assert abs(B[j, l] - float(Bj)) < 2e-15


def _grid(n):
    return W.Grid(n=tuple(n), lo=(0.0,) * len(n), hi=(1.0,) * len(n), pair=(-1,) * len(n))


def test_state_bytes_model():
    g = _grid((10, 20))
    assert S.sl_state_bytes(g, 2, "fp64") == 200 * 9 * 8
    assert S.sl_state_bytes(g, 2, "mix_fp32") == 200 * (8 + 8 * 4)
    assert S.sl_state_bytes(g, 1, "mix_bf16") == 200 * (8 + 3 * 2 + 4)
    assert S.sl_state_bytes(g, 1, "mix_fp16") == 200 * (8 + 3 * 2 + 4)


def test_memory_reduction_matches_paper():
    """The paper's memorydown figures (Tables III-VI, Sec. III-A) follow from
    the byte model of every store: FP64 bytes over 8 n_lo + 4 n_hi, for
    "# double" = 0, 1, 2 (c_0 .. c_{q-1} in FP64 in one dimension)."""
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", "memory_reduction.txt")):
        if line.strip() and not line.startswith("#"):
            d, o, nd, red, _ = line.split()
            rows.append((int(d), int(o), int(nd), float(red)))
    checked = 0
    store = {0: "fp32", 1: "mix_fp32", 2: "mix_fp32_d2", 3: "mix_fp32_d3"}
    for d, o, nd, red in rows:
        g = _grid((8,) * d)
        if nd == o ** d:
            continue   # all-FP64 reference row
        assert d == 1 or nd == 1
        r = S.sl_state_bytes(g, o - 1, "fp64") / S.sl_state_bytes(g, o - 1, store[nd])
        digits = len(str(red).split(".")[1])
        # the paper truncates 2D (128/68 = 1.88) to 1.8; allow one unit in its last digit
        assert abs(r - red) <= 10 ** -digits * 1.0 + 1e-12, (d, o, r, red)
        checked += 1
    assert checked == 10


@pytest.mark.parametrize("bad,code", [
    (dict(n=(0,)), S.SL_EINVAL),
    (dict(n=(4,), lo=(1.0,), hi=(1.0,)), S.SL_EINVAL),
    (dict(n=(4, 4), pair=(1, 0)), S.SL_EINVAL),
    (dict(n=(4, 4), pair=(5, -1)), S.SL_EINVAL),
    (dict(n=(70000, 70000)), S.SL_ENOTSUP),
])
def test_create_rejects_bad_grids_before_device_work(bad, code):
    n = bad["n"]
    g = W.Grid(n=n, lo=bad.get("lo", (0.0,) * len(n)), hi=bad.get("hi", (1.0,) * len(n)),
               pair=bad.get("pair", (-1,) * len(n)))
    with pytest.raises(S.SlError) as e:
        S.sl_create(g, 1, "fp64")
    assert e.value.status == code
    assert S.sl_last_error()


def test_create_rejects_bad_degree_and_scaled_size():
    with pytest.raises(S.SlError) as e:
        S.sl_create(_grid((4,)), 4, "fp64")
    assert e.value.status == S.SL_EINVAL
    with pytest.raises(S.SlError) as e:
        S.sl_create(_grid((2, 2, 2, 2, 2)), 2, "mix_bf16")   # 3^5 = 243 > 128
    assert e.value.status == S.SL_ENOTSUP


def test_plane_layout_matches_state_bytes():
    for n, k, st in [((10, 7), 2, "mix_fp32"), ((3, 2, 2, 3, 2, 2), 1, "mix_bf16"), ((5, 3), 1, "fp64"),
                     ((4, 3, 5), 3, "mix_fp16")]:
        g = W.Grid(n=n, lo=(0.0,) * len(n), hi=(1.0,) * len(n), pair=(-1,) * len(n))
        lay = S.sl_plane_layout(g, k, st)
        cells = int(np.prod(n))
        assert lay["plane_stride"] == -(-cells // 64) * 64
        assert lay["mean_bytes"] == lay["plane_stride"] * 8
        if lay["record_slots"]:
            assert lay["hi_bytes"] == cells * lay["record_slots"] * 2
        else:
            elem = {"mix_fp32": 4, "fp64": 8, "mix_bf16": 2, "mix_fp16": 2}[st]
            assert lay["hi_bytes"] == lay["plane_stride"] * ((k + 1) ** len(n) - 1) * elem
        assert lay["scale_bytes"] == (lay["plane_stride"] * 4 if st in ("mix_bf16", "mix_fp16") else 0)
    with pytest.raises(S.SlError):
        S.sl_plane_layout(W.Grid(n=(0,), lo=(0.0,), hi=(1.0,), pair=(-1,)), 1, "fp64")


def test_create_external_rejects_bad_planes_before_device_work():
    g = W.Grid(n=(8,), lo=(0.0,), hi=(1.0,), pair=(-1,))
    with pytest.raises(S.SlError) as e:
        S.sl_create_external(g, 1, "fp64", [0, 0, 0, 0, 0, 0])
    assert e.value.status == S.SL_EINVAL
    with pytest.raises(S.SlError) as e:
        S.sl_create_external(g, 1, "fp64", [256, 512 + 8, 0, 1024, 2048, 0])   # misaligned hi_0
    assert e.value.status == S.SL_EINVAL


@pytest.mark.parametrize("ndim", [1, 2, 3, 4, 5, 6])
def test_split_store_layout_counts_the_fp64_block(ndim):
    """The stores of # double = q hold q^d FP64 planes and o^d - q^d FP32
    planes (host-side layout, no device work); invalid q for the degree is
    rejected."""
    g = _grid((3,) * ndim)
    cells = 3 ** ndim
    ps = (cells + 63) // 64 * 64
    for k in (1, 2, 3):
        o = k + 1
        if o ** ndim > 4096:
            continue
        for store, q in (("fp32", 0), ("mix_fp32", 1), ("mix_fp32_d2", 2), ("mix_fp32_d3", 3)):
            if q > k:
                with pytest.raises(S.SlError):
                    S.sl_plane_layout(g, k, store)
                continue
            lay = S.sl_plane_layout(g, k, store)
            assert lay["plane_stride"] == ps
            assert lay["mean_bytes"] == q ** ndim * ps * 8
            assert lay["hi_bytes"] == (o ** ndim - q ** ndim) * ps * 4
            assert S.sl_state_bytes(g, k, store) == cells * (8 * q ** ndim + 4 * (o ** ndim - q ** ndim))
            assert S.plane_counts(ndim, k, store) == (q ** ndim, o ** ndim - q ** ndim)


def test_fp64_rate_selftest_rejects_bad_arguments_without_device_work():
    for iters in (0, -1, (1 << 24) + 1):
        with pytest.raises(S.SlError) as e:
            S.sl_selftest_fp64_rate(iters)
        assert e.value.status == S.SL_EINVAL
