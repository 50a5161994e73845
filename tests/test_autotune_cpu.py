"""The autotuner's host side without a GPU: grid classes, the candidate launch shapes (every
one valid for cmcg_options.tile and for the ABI's range checks), and cache lookups."""
import json

import pytest

from paper_1903_12522_gb300 import autotune, cmcg


def test_size_class_rounds_to_the_nearest_power_of_two():
    assert autotune.size_class(3, 256, cmcg.MIXED) == "d3_n256_fp32"
    assert autotune.size_class(3, 200, cmcg.FP32) == "d3_n256_fp32"
    assert autotune.size_class(3, 180, cmcg.FP32) == "d3_n128_fp32"  # log2 180 = 7.49
    assert autotune.size_class(2, 1024, cmcg.FP64) == "d2_n1024_fp64"
    assert autotune.size_class(2, 1, cmcg.FP32) == "d2_n2_fp32"


@pytest.mark.parametrize("cands", [autotune.candidates_3d(), autotune.candidates_2d()])
def test_candidates_are_valid_tiles(cands):
    assert len(set(cands)) == len(cands)
    for t in cands:
        assert len(t) == 4
        # the ranges cmcg_create accepts
        assert 0 <= t[0] <= 512 and 0 <= t[1] <= 512 and 0 <= t[2] <= 60 and 0 <= t[3] <= 6, t


def test_3d_candidates_span_every_scheme_and_both_depths():
    schemes = {t[3] for t in autotune.candidates_3d()}
    assert schemes == {1, 2, 3, 4, 5, 6}
    # temporal-blocking depth: one step per launch (schemes 1, 3-6) and two (scheme 2), and the
    # staged kernels' planes staged ahead
    assert {t[0] for t in autotune.candidates_3d() if t[3] == 2} == {2, 3}
    assert {t[2] for t in autotune.candidates_3d() if t[3] == 6} == {2, 3}


def test_engine_candidates():
    cands = autotune.engine_candidates()
    assert (0, 8) in cands and len(set(cands)) == len(cands)
    assert all(b >= 0 and 0 < z <= 256 for b, z in cands)


def test_cache_lookups(tmp_path, monkeypatch):
    cache = tmp_path / "cache.json"
    cache.write_text(json.dumps({"d3_n256_fp32": {"tile": [16, 0, 0, 3]},
                                 "engine_batch2d": {"shape": [4, 16]}}))
    monkeypatch.setattr(autotune, "CACHE", str(cache))
    assert autotune.lookup(3, 256, cmcg.MIXED) == (16, 0, 0, 3)
    assert autotune.lookup(3, 512, cmcg.MIXED) is None
    assert autotune.lookup_engine("batch2d") == (4, 16)
    assert autotune.lookup_engine("mix") is None
    cache.write_text("not json")
    assert autotune.lookup(3, 256, cmcg.MIXED) is None  # a damaged cache means defaults


def test_committed_cache_entries_are_valid():
    data = json.load(open(autotune.CACHE))
    for key, entry in data.items():
        if key.startswith("engine_"):
            b, z = entry["shape"]
            assert b >= 0 and 0 <= z <= 256
        else:
            t = entry["tile"]
            assert len(t) == 4 and 0 <= t[3] <= 6
            assert entry["ms_per_adjoint_period"] <= entry["worst_ms"]
