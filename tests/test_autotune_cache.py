"""Host logic of the autotuner's result cache (no GPU): the JSON store keyed by
device name and problem shape survives a round trip, and a corrupt or
unwritable cache degrades to tuning without memory instead of failing."""
import json
import os

from paper_1511_03703_gb300 import autotune as A


def test_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("ENS_AUTOTUNE_CACHE", str(path))
    assert A.cache_path() == str(path)
    assert A._load() == {}
    db = {"GB300|spmv|64|32": "dfv", "GB300|check_every|x": 8}
    A._store(db)
    assert json.loads(path.read_text()) == db
    assert A._load() == db
    assert not [p for p in os.listdir(path.parent) if ".tmp" in p]  # written by rename


def test_corrupt_cache_reads_as_empty(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    monkeypatch.setenv("ENS_AUTOTUNE_CACHE", str(path))
    assert A._load() == {}


def test_unwritable_cache_is_ignored(tmp_path, monkeypatch):
    blocker = tmp_path / "file"
    blocker.write_text("x")  # a file where the cache directory would go
    monkeypatch.setenv("ENS_AUTOTUNE_CACHE", str(blocker / "tune.json"))
    A._store({"k": 1})       # must not raise
    assert A._load() == {}
