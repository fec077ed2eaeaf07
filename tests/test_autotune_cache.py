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


def test_mapping_choices_and_flags():
    """The tuned mapping's knobs: the chunks per SpMV CTA that fit 1024 threads
    at each width, and the ens_cg flags a cached mapping turns into."""
    import paper_1511_03703_gb300 as E
    assert A.k1_chunk_choices(1) == (1, 2, 4, 8)
    assert A.k1_chunk_choices(4) == (1, 2, 4, 8)
    assert A.k1_chunk_choices(8) == (1, 2, 4, 8)
    assert A.k1_chunk_choices(16) == (1, 2, 4)
    assert A.k1_chunk_choices(32) == (1, 2)
    assert A.mapping_flags({"form": "dfv", "k1_chunks": 1}) == 1 << 16
    assert A.mapping_flags({"form": "split", "k1_chunks": 8}) == E.CG_SPLIT64 | (4 << 16)
    assert A.mapping_flags({"form": "f64"}) == 0          # no chunks field: the library default
    assert E.cg_k1_chunks(0) == 0 and E.cg_k1_chunks(2) == 2 << 16
    assert A.k1_mapping_choices(32) == (1, 2, "defer")
    assert A.mapping_flags({"form": "dfv", "k1_chunks": "defer"}) == E.CG_K1_DEFER == 1 << 20


def test_cached_mapping_is_returned_without_tuning(tmp_path, monkeypatch):
    """A cached (form, chunks) entry is served from the JSON store: the timing
    routine must not run (it needs a GPU)."""
    monkeypatch.setenv("ENS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(A, "_key", lambda *parts: "|".join(["GPU"] + [str(p) for p in parts]))

    class Mesh:
        N, M = 64, 10

    entry = {"form": "dfv", "k1_chunks": 2, "spmv_ms": 0.35, "candidates_ms": {"dfv,1": 0.36, "dfv,2": 0.35}}
    A._store({A._key("mapping", 64, 10, 32, ",".join(A.FORMS)): entry})

    def no_gpu(*a, **k):
        raise AssertionError("tuning ran although the mapping is cached")
    monkeypatch.setattr(A, "time_spmv_mappings", no_gpu)
    assert A.best_mapping(Mesh(), 32) == entry
    assert A.best_form(Mesh(), 32) == "dfv"
