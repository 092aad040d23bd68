"""Host logic of the shape autotuner: signatures, the staged search and the
JSON cache, driven by a fake timing function (no GPU)."""
import json

import pytest

from paper_2412_16750_gb300 import tune


def test_signature_buckets():
    a = tune.signature(100, 2_000_000, 1000, 1)
    assert a == tune.signature(128, 1_500_000, 600, 1)          # same power-of-two buckets
    assert a != tune.signature(129, 2_000_000, 1000, 1)
    assert a != tune.signature(100, 2_000_000, 1000, 10)
    assert tune.signature(1, 1, 1) == "loss_grad|lane<=1|N~1|K~1|s=1"


def test_candidate_pairs_hold_the_longest_lane():
    for lane in (1, 64, 65, 200, 2048):
        pairs = tune.candidates_pairs(lane)
        assert pairs and all(32 * v * g >= lane for v, g in pairs)
    assert tune.candidates_pairs(2048) == [(8, 8)]


def test_search_finds_the_minimum_of_a_separable_cost():
    # cost = f(vpt, warps) + h(ckpt) + k(wpb); (4, 2) best pair, ckpt 16, wpb 4
    def cost(shape):
        v, g, c, w = shape
        if (v, g) == (8, 8):
            return None                                          # rejected by the library
        return abs(v - 4) + abs(g - 2) + 0.1 * abs(c - 16) + 0.01 * abs(w - 4) + 1.0
    best, ms, timings = tune.search(cost, 100)
    assert best == (4, 2, 16, 4)
    assert ms == pytest.approx(1.0)
    assert all(32 * s[0] * s[1] >= 100 for s in timings)
    # every shape is timed at most once
    assert len(timings) == len(set(timings))


def test_search_skips_wpb_not_multiple_of_warps():
    seen = []

    def cost(shape):
        seen.append(shape)
        return 1.0 if shape[1] == 8 else 2.0
    best, _, _ = tune.search(cost, 2048)
    assert best[1] == 8 and best[3] % 8 == 0
    assert all(s[3] % s[1] == 0 for s in seen)


def test_search_raises_when_nothing_fits():
    with pytest.raises(RuntimeError):
        tune.search(lambda s: None, 100)


def test_cache_roundtrip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    sig = tune.signature(100, 10_000, 275, 10, kind="batch")
    assert tune.lookup("GB300", sig, path) is None
    tune.store("GB300", sig, (2, 8, 16, 8), 12.5, path)
    tune.store("GB300", "other", (4, 4, 8, 8), 3.0, path)
    assert tune.lookup("GB300", sig, path) == (2, 8, 16, 8)
    assert tune.lookup("B200", sig, path) is None
    d = json.load(open(path))
    assert d["GB300"][sig]["ms"] == 12.5


def test_corrupt_cache_is_ignored(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert tune.load_cache(str(path)) == {}
    tune.store("GB300", "s", (2, 1, 8, 8), 1.0, str(path))
    assert tune.lookup("GB300", "s", str(path)) == (2, 1, 8, 8)
