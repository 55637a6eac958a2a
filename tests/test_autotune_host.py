"""Autotuner host logic (no GPU): the candidate space per key width, the
shape-class key, and the JSON cache round trip."""
import json

import pytest

from paper_0811_3448_gb300 import autotune


@pytest.mark.parametrize("kb,vb,cutoffs,tiles", [
    (4, 4, {2048, 4096, 8192}, {6144, 4096}), (4, 0, {2048, 4096, 8192}, {7168, 4096}),
    (8, 4, {2048, 4096}, {4096, 2048}), (16, 0, {2048}, {2048, 1024})])
def test_candidates_cover_the_accepted_space(kb, vb, cutoffs, tiles):
    cands = autotune.candidates(kb, vb)
    assert {c.small_cutoff for c in cands} == cutoffs
    assert {c.tile_keys for c in cands} == tiles
    assert {c.bits_per_pass for c in cands} == {6, 7, 8}
    assert len(cands) == len(tiles) * 3 * len(cutoffs)
    assert len({autotune.describe(c) for c in cands}) == len(cands)
    # CTAs per SM stay at each kernel's occupancy
    assert all(c.ctas_per_sm == 0 for c in cands)


def test_shape_key_classes():
    k = autotune.shape_key
    assert k(1 << 20, 4, 4, 0, "G") == k((1 << 21) - 1, 4, 4, 0, "G")      # same log2 class
    assert k(1 << 20, 4, 4, 0, "G") != k(1 << 21, 4, 4, 0, "G")
    assert k(1 << 20, 4, 4, 0, "G") != k(1 << 20, 8, 4, 0, "G")
    assert k(1 << 20, 4, 4, 0, "G") != k(1 << 20, 4, 0, 0, "G")
    assert k(1 << 20, 4, 4, 1, "G") == k(1 << 20, 4, 4, 0, "G")            # one segment = plain
    assert k(1 << 20, 4, 4, 20000, "G") != k(1 << 20, 4, 4, 100, "G")
    assert k(1 << 20, 4, 4, 0, "A") != k(1 << 20, 4, 4, 0, "B")


def test_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("BINAR_TUNE_CACHE", str(path))
    assert autotune.cache_path() == str(path)
    assert autotune._load_cache() == {}
    autotune._store_cache({"x": {"config": {"small_cutoff": 4096, "bits_per_pass": 7}}})
    assert json.loads(path.read_text())["x"]["config"]["small_cutoff"] == 4096
    assert autotune._load_cache()["x"]["config"]["bits_per_pass"] == 7
    path.write_text("not json")
    assert autotune._load_cache() == {}                                    # corrupt cache ignored
