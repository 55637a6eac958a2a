"""Autotuner host logic (no GPU): the candidate space per key width, the
shape-class key, and the JSON cache round trip."""
import json

import pytest

from paper_0811_3448_gb300 import autotune


@pytest.mark.parametrize("kb,cutoffs", [(4, {2048, 4096, 8192}), (8, {2048, 4096}), (16, {2048})])
def test_candidates_cover_the_accepted_space(kb, cutoffs):
    cands = autotune.candidates(kb)
    assert {c.small_cutoff for c in cands} == cutoffs
    assert {c.ctas_per_sm for c in cands} == {0, 1, 2}
    assert len(cands) == 3 * len(cutoffs)
    # every other knob is left at the library default
    assert all(c.tile_keys == 0 and c.bits_per_pass == 0 for c in cands)


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
    autotune._store_cache({"x": {"config": {"small_cutoff": 4096, "ctas_per_sm": 0}}})
    assert json.loads(path.read_text())["x"]["config"]["small_cutoff"] == 4096
    assert autotune._load_cache()["x"]["config"]["ctas_per_sm"] == 0
    path.write_text("not json")
    assert autotune._load_cache() == {}                                    # corrupt cache ignored
