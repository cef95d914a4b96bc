"""The batch autotuner's JSON cache (host logic, no GPU): keys group assets by render size and
triangle count rounded up to a power of two, entries round-trip, and a missing or unreadable
file reads as a miss."""
import json

from paper_2404_09758_gb300 import _abi, tuning_cache_load, tuning_cache_store, tuning_key


def test_key_buckets_triangle_counts_and_separates_the_rest():
    k = tuning_key("GB300", [(512, 512, 1000)], 8)
    assert k == tuning_key("GB300", [(512, 512, 1024)], 8)
    assert k != tuning_key("GB300", [(512, 512, 1025)], 8)
    assert k != tuning_key("GB300", [(512, 256, 1000)], 8)
    assert k != tuning_key("B200", [(512, 512, 1000)], 8)
    assert k != tuning_key("GB300", [(512, 512, 1000)], 16)
    # the batch's order is part of the key (assets are walked in that order)
    a, b = (512, 512, 1000), (1024, 1024, 200000)
    assert tuning_key("GB300", [a, b], 8) != tuning_key("GB300", [b, a], 8)


def test_entries_round_trip_and_keep_each_other(tmp_path):
    path = str(tmp_path / "tune.json")
    assert tuning_cache_load(path, "k1") is None
    tuning_cache_store(path, "k1", _abi.BatchTuning(8, 2, 256), 95.25)
    tuning_cache_store(path, "k2", _abi.BatchTuning(4, 1, 128), 12.5)
    t, ms = tuning_cache_load(path, "k1")
    assert (t.pairs_per_item, t.blocks_per_sm, t.light_bin, ms) == (8, 2, 256, 95.25)
    t, ms = tuning_cache_load(path, "k2")
    assert (t.pairs_per_item, t.blocks_per_sm, t.light_bin, ms) == (4, 1, 128, 12.5)
    assert tuning_cache_load(path, "k3") is None
    assert sorted(json.load(open(path))) == ["k1", "k2"]


def test_unreadable_files_read_as_a_miss_and_are_replaced(tmp_path):
    path = str(tmp_path / "tune.json")
    open(path, "w").write("{not json")
    assert tuning_cache_load(path, "k1") is None
    tuning_cache_store(path, "k1", _abi.BatchTuning(2, 2, 64), 1.0)
    assert tuning_cache_load(path, "k1")[0].light_bin == 64
    json.dump({"k1": {"pairs_per_item": 8}}, open(path, "w"))  # an entry missing fields
    assert tuning_cache_load(path, "k1") is None
