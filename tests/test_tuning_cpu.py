"""Host logic of the launch-configuration cache (no GPU): keys separate what the autotuner's
choice depends on and nothing else, and the JSON file survives round trips, bad entries and
bad files."""
import json

import pytest

import paper_1803_11036_gb300 as ssd
from paper_1803_11036_gb300 import tuning
from paper_1803_11036_gb300._abi import TUNING_FIELDS

P = dict(log2_eta=11, q=18, r=5, delta=5, k=60, theta=1024)
T = dict(touch_chunk_bytes=32 << 20, stream_blocks_per_sm=0, scan_blocks_per_sm=8, scan_unroll=4, merge_group=8,
         combine_touches=0, collect_touches=0, pair_level=0)


def test_key_separates_device_params_routers_and_size():
    base = tuning.cache_key("GB300", ssd.make_params(P), 1, 6_250_000)
    assert base == tuning.cache_key("GB300", ssd.make_params(P), 1, 6_250_000)
    assert base == tuning.cache_key("GB300 ", ssd.make_params(P), 1, 6_000_000)   # same size class
    others = {
        tuning.cache_key("B200", ssd.make_params(P), 1, 6_250_000),
        tuning.cache_key("GB300", ssd.make_params(dict(P, q=17)), 1, 6_250_000),
        tuning.cache_key("GB300", ssd.make_params(P, ssd.SSD_VERIFY_H0), 1, 6_250_000),
        tuning.cache_key("GB300", ssd.make_params(P), 16, 6_250_000),
        tuning.cache_key("GB300", ssd.make_params(P), 1, 1_500_000),
    }
    assert base not in others and len(others) == 5
    # capacities and the touch chunk size are not part of the key: the tuner sets the latter
    assert base == tuning.cache_key("GB300", ssd.make_params(P, touch_chunk_bytes=8 << 20, ctb_capacity=1 << 20),
                                    1, 6_250_000)


def test_size_class():
    assert tuning.size_class(0) == 0
    assert tuning.size_class(1 << 20) == 20
    assert tuning.size_class(int(1.3 * (1 << 20))) == 20
    assert tuning.size_class(int(1.5 * (1 << 20))) == 21


def test_store_load_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "t.json")
    assert tuning.load(path) == {}
    tuning.store(path, "a", T)
    tuning.store(path, "b", dict(T, scan_unroll=8))
    tuning.store(path, "a", dict(T, merge_group=4))
    got = tuning.load(path)
    assert got == {"a": dict(T, merge_group=4), "b": dict(T, scan_unroll=8)}
    with pytest.raises(ValueError):
        tuning.store(path, "c", {"scan_unroll": 4})


def test_bad_files_and_entries_are_ignored(tmp_path):
    path = tmp_path / "t.json"
    path.write_text("{not json")
    assert tuning.load(str(path)) == {}
    path.write_text(json.dumps([1, 2]))
    assert tuning.load(str(path)) == {}
    path.write_text(json.dumps({"ok": T, "short": {"scan_unroll": 4}, "text": dict(T, scan_unroll="4")}))
    assert tuning.load(str(path)) == {"ok": T}
    assert set(TUNING_FIELDS) == set(T)
