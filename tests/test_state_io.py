"""Host-side checks of the checkpoint format, the tune cache and the
allocation-failure hook (CPU only: no device work)."""
import json

import numpy as np
import pytest

import paper_1603_07008_gb300 as S
from paper_1603_07008_gb300 import state_io as IO
from paper_1603_07008_gb300 import workloads as W


def test_checkpoint_round_trip(tmp_path):
    g = W.Grid(n=(3, 4), lo=(0.0, -6.0), hi=(1.0, 6.0), pair=(1, -1))
    meta = IO.checkpoint_meta(g, 2, "mix_fp32_d2", step=17, time=1.7, extra={"note": "x"})
    rng = np.random.default_rng(1)
    mean = rng.standard_normal((4, 12))
    hi = rng.standard_normal((5, 12)).astype(np.float32)
    p = tmp_path / "a.npz"
    IO.write_checkpoint(p, meta, mean, hi, None)
    m2, mean2, hi2, scale2 = IO.read_checkpoint(p)
    assert m2 == json.loads(json.dumps(meta)) and m2["step"] == 17 and m2["grid"]["pair"] == [1, -1]
    assert np.array_equal(mean2, mean) and mean2.dtype == np.float64
    assert np.array_equal(hi2, hi) and hi2.dtype == np.float32
    assert scale2 is None
    # the all-FP32 store has no FP64 plane; the scaled stores keep 16-bit patterns and scales
    sc = rng.standard_normal(12).astype(np.float32)
    bits = rng.integers(0, 2 ** 16, size=(12, 16), dtype=np.uint16)
    IO.write_checkpoint(p, meta, None, bits, sc)
    _, mean3, hi3, scale3 = IO.read_checkpoint(p)
    assert mean3 is None and np.array_equal(hi3, bits) and hi3.dtype == np.uint16 and np.array_equal(scale3, sc)
    assert not list(tmp_path.glob("*.tmp"))


def test_checkpoint_version_is_checked(tmp_path):
    g = W.Grid(n=(2,), lo=(0.0,), hi=(1.0,), pair=(-1,))
    meta = IO.checkpoint_meta(g, 1, "fp64", 0, 0.0)
    meta["version"] = 99
    p = tmp_path / "b.npz"
    IO.write_checkpoint(p, meta, np.zeros(2), np.zeros((1, 2)), None)
    with pytest.raises(ValueError):
        IO.read_checkpoint(p)


class FakeCtx:
    """Duck-typed context: records the shapes set and counts autotunes."""

    def __init__(self, ok=lambda d, sh: True):
        self.grid = W.Grid(n=(8, 6), lo=(0.0, 0.0), hi=(1.0, 1.0), pair=(1, -1))
        self.degree, self.storage = 2, "mix_fp32"
        self.tunes = {0: {"block": 256, "fibres_per_thread": 1, "unroll": 4, "pipeline": 0, "chunk": 0,
                          "max_blocks_per_sm": 0},
                      1: {"block": 128, "fibres_per_thread": 2, "unroll": 2, "pipeline": 0, "chunk": 3,
                          "max_blocks_per_sm": 5}}
        self.autotuned = 0
        self.set_calls = []
        self.ok = ok

    def autotune(self, reps):
        self.autotuned += 1

    def get_tune(self, d):
        return dict(self.tunes[d])

    def set_tune(self, d, **sh):
        if not self.ok(d, sh):
            raise S.SlError(S.SL_EINVAL, "not built")
        self.set_calls.append((d, sh))


def test_tune_cache_miss_then_hit(tmp_path):
    p = tmp_path / "tunes.json"
    a = FakeCtx()
    assert IO.autotune_cached(a, p, device="GB300 test") is False
    assert a.autotuned == 1 and not a.set_calls
    b = FakeCtx()
    assert IO.autotune_cached(b, p, device="GB300 test") is True
    assert b.autotuned == 0 and b.set_calls == [(0, a.tunes[0]), (1, a.tunes[1])]
    # another device, degree or store is another key
    c = FakeCtx()
    c.degree = 1
    assert IO.autotune_cached(c, p, device="GB300 test") is False
    assert len(json.load(open(p))) == 2


def test_tune_cache_survives_bad_entries(tmp_path):
    p = tmp_path / "tunes.json"
    p.write_text("{not json")
    a = FakeCtx()
    assert IO.autotune_cached(a, p, device="d") is False       # unreadable file: tune and rewrite
    b = FakeCtx(ok=lambda d, sh: False)                         # cached shape no longer built
    assert IO.autotune_cached(b, p, device="d") is False and b.autotuned == 1


def test_fail_alloc_hook_is_host_side():
    with pytest.raises(S.SlError) as e:
        S.sl_debug_fail_alloc(-1)
    assert e.value.status == S.SL_EINVAL
    S.sl_debug_fail_alloc(0)
