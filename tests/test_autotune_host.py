"""Host logic of the batched autotuner, on the CPU: the candidate tiles, the
problem classes, the JSON cache (round trip, a corrupt file) and applying
cached choices to problems without timing anything."""
import json

import numpy as np
import pytest
import torch


@pytest.fixture(scope="module")
def at():
    from paper_2601_09477_gb300 import build
    build.build()
    from paper_2601_09477_gb300 import autotune
    return autotune


def test_candidates_within_library_limits(at):
    for L, k in [(15, 4096), (10, 100), (5, 3000), (18, 512)]:
        cands = at.candidates(L, k)
        assert cands
        for tile, tt in cands:
            assert 5 <= tile <= min(14, L)      # slices the batched kernel holds
            assert tt == 0 or tt < k            # 0: the library's default t-tile
    assert {t for t, _ in at.candidates(10, 100)} == {8, 9, 10}
    assert {tt for _, tt in at.candidates(10, 100)} == {0, 64}


def test_class_key_rounds_k_up_to_a_power_of_two(at):
    assert at.class_key(512, 3000, 700, 13, 5) == "L13_k4096_d5"
    assert at.class_key(4096, 4096, 4096, 13, 5) == "L13_k4096_d5"
    assert at.class_key(4096, 4097, 4096, 13, 5) == "L13_k8192_d5"
    assert at.class_key(10, 1, 10, 10, 3) == "L10_k1_d3"


def test_cache_round_trip_and_corrupt_file(at, tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    t = at.Tuner(path)
    assert t.table == {}
    t.table[at.class_key(600, 900, 700, 12, 5)] = [11, 256]
    t.save()
    with open(path) as f:
        assert json.load(f) == {"L12_k1024_d5": [11, 256]}
    again = at.Tuner(path)
    assert again.lookup(700, 1000, 500, 12, 5) == [11, 256]   # same class
    assert again.lookup(700, 1000, 500, 13, 5) is None
    with open(path, "w") as f:
        f.write("{not json")
    assert at.Tuner(path).table == {}


def test_apply_uses_cached_choices_only(at, tmp_path):
    cmm = at.cmm
    t = at.Tuner(str(tmp_path / "tune.json"))
    t.table["L12_k1024_d5"] = [10, 64]
    g = np.random.default_rng(0)
    hit = cmm.Problem(torch.from_numpy(g.standard_normal((1000, 300)).astype(np.float32)),
                      torch.zeros((1000, 200), dtype=torch.float32), cmm.make_hashes(1, 5, 12))
    miss = cmm.Problem(torch.zeros((1000, 300), dtype=torch.float32),
                       torch.zeros((1000, 200), dtype=torch.float32), cmm.make_hashes(2, 5, 14))
    t.apply([hit, miss], d=5, tune_missing=False)   # no timing: nothing touches a GPU
    assert (hit.tile_log2, hit.t_tile) == (10, 64)
    assert (miss.tile_log2, miss.t_tile) == (0, 0)
