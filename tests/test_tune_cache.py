"""The autotuner's JSON cache (host logic, no GPU): keys separate devices, library
builds and workloads; entries round-trip; a missing, corrupt or non-object file
reads as empty; a store replaces the file whole (no temporary file left behind)
and keeps the other entries."""
import json
import os

import paper_2105_09688_gb300 as S


def test_keys_separate_device_build_and_workload():
    base = ("NVIDIA GB300", 152, "0123456789abcdef", 3, 1 << 18, S.SSM_COEF_COUPLED3D, S.SSM_FP32C_LEARNED)
    k0 = S.tune_cache_key(*base)
    for i, other in enumerate(["NVIDIA B200", 148, "fedcba9876543210", 1, 1 << 16, S.SSM_COEF_CUBIC1D_GAUSS,
                               S.SSM_FP32C]):
        changed = list(base)
        changed[i] = other
        assert S.tune_cache_key(*changed) != k0
    assert S.tune_cache_key(*base) == k0


def test_round_trip_and_other_entries_kept(tmp_path):
    path = str(tmp_path / "tune.json")
    assert S.tune_cache_load(path) == {}
    plan = {"form": 2, "threads": 128, "targets_per_thread": 8, "chunks": 17, "chunk_len": 15872}
    S.tune_cache_store(path, "a", {"plans": [plan, None], "best_ms": [19.6, 17.7]})
    S.tune_cache_store(path, "b", {"plans": [None, plan], "best_ms": [0.0, 3.0]})
    got = S.tune_cache_load(path)
    assert got["a"]["plans"][0] == plan and got["a"]["plans"][1] is None
    assert got["b"]["best_ms"] == [0.0, 3.0]
    S.tune_cache_store(path, "a", {"plans": [None, None], "best_ms": [1.0, 2.0]})
    got = S.tune_cache_load(path)
    assert got["a"]["best_ms"] == [1.0, 2.0] and "b" in got
    assert sorted(os.listdir(tmp_path)) == ["tune.json"]


def test_unreadable_files_read_as_empty(tmp_path):
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    assert S.tune_cache_load(str(bad)) == {}
    arr = tmp_path / "list.json"
    arr.write_text(json.dumps([1, 2, 3]))
    assert S.tune_cache_load(str(arr)) == {}
    S.tune_cache_store(str(bad), "k", {"plans": [None, None], "best_ms": [0.0, 0.0]})
    assert list(S.tune_cache_load(str(bad))) == ["k"]
