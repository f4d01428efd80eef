"""The JSON cache of tuned settings (paper_1912_05508_gb300/tuning.py): keys, round trips,
per-GPU filtering, atomic replacement and corrupted files, all on the CPU."""
import json
import os

from paper_1912_05508_gb300 import tuning

OPTS = {"gemm_prec": 0, "target": 1, "krylov": 0, "reorth": 0, "panel_leaf": 0}
T1 = {"panel_width": 16, "node_mode": 0, "gemm_kernel": 0, "batched_ctas_per_sm": 0, "krylov_ctas": 0, "ms": 21.5}
T2 = {"panel_width": 8, "node_mode": 1, "gemm_kernel": 1, "batched_ctas_per_sm": 2, "krylov_ctas": 64, "ms": 3.25}


def test_key_round_trip():
    k = tuning.make_key("NVIDIA GB300", 152, 0, 32768, 4096, OPTS)
    assert tuning.parse_key(k) == ("NVIDIA GB300", 152, 0, 32768, 4096, OPTS)
    # a '|' in a device name cannot break the key apart
    k2 = tuning.make_key("odd|name", 8, 1, 4096, 512, OPTS)
    assert tuning.parse_key(k2)[0] == "odd/name"
    assert tuning.parse_key("garbage") is None
    assert tuning.parse_key("a|smx|kind0|1x2|gemm_prec=0|target=1|krylov=0|reorth=0|panel_leaf=0") is None


def test_record_load_and_device_filter(tmp_path):
    path = str(tmp_path / "sub" / "tuning.json")
    assert tuning.load(path) == {}
    k1 = tuning.make_key("NVIDIA GB300", 152, 0, 32768, 4096, OPTS)
    k2 = tuning.make_key("NVIDIA GB300", 152, 1, 4096, 512, OPTS)
    k3 = tuning.make_key("Other GPU", 100, 0, 32768, 4096, OPTS)
    tuning.record(k1, T1, path)
    tuning.record(k2, T2, path)
    tuning.record(k3, T2, path)
    entries = tuning.load(path)
    assert entries[k1] == T1 and entries[k2] == T2 and len(entries) == 3
    mine = tuning.entries_for_device(entries, "NVIDIA GB300", 152)
    assert sorted((kind, m, n) for kind, m, n, _, _ in mine) == [(0, 32768, 4096), (1, 4096, 512)]
    assert tuning.entries_for_device(entries, "NVIDIA GB300", 148) == []
    # replacing an entry keeps the others
    tuning.record(k1, T2, path)
    assert tuning.load(path)[k1] == T2 and tuning.load(path)[k2] == T2
    # no temporary files are left behind
    assert os.listdir(os.path.dirname(path)) == ["tuning.json"]


def test_corrupted_or_foreign_files_count_as_empty(tmp_path):
    path = str(tmp_path / "tuning.json")
    with open(path, "w") as fh:
        fh.write("{not json")
    assert tuning.load(path) == {}
    with open(path, "w") as fh:
        json.dump([1, 2, 3], fh)
    assert tuning.load(path) == {}
    # entries with a malformed key or missing fields are dropped, the rest kept
    good = tuning.make_key("NVIDIA GB300", 152, 0, 1024, 128, OPTS)
    with open(path, "w") as fh:
        json.dump({good: T1, "bad key": T1, tuning.make_key("x", 1, 0, 1, 1, OPTS): {"ms": 1.0}}, fh)
    assert tuning.load(path) == {good: T1}
    tuning.record(good, T2, path)
    assert tuning.load(path) == {good: T2}


def test_cache_path_from_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("LLS_TUNE_CACHE", str(tmp_path / "t.json"))
    assert tuning.cache_path() == str(tmp_path / "t.json")
    monkeypatch.delenv("LLS_TUNE_CACHE")
    assert tuning.cache_path().endswith(os.path.join("lls_gb300", "tuning.json"))
