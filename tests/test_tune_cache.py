"""The autotuner's on-disk cache (host-only calls, no GPU): entries are written,
read back, replaced, and never confused with keys that only share a prefix."""
import pytest

from paper_1902_00176_gb300 import gfc


@pytest.fixture(autouse=True)
def _lib(gfc_lib):
    yield


def test_missing_file_and_missing_key(tmp_path):
    path = str(tmp_path / "tune.txt")
    assert gfc.tune_cache_get(path, "k") is None
    gfc.tune_cache_put(path, "k", "column_solver=0 chunk=0 streams=1")
    assert gfc.tune_cache_get(path, "other") is None


def test_write_reload_replace(tmp_path):
    path = str(tmp_path / "tune.txt")
    gfc.tune_cache_put(path, "gfc-tune v1 a", "rag_streams=4")
    gfc.tune_cache_put(path, "gfc-tune v1 b", "rag_streams=2")
    assert gfc.tune_cache_get(path, "gfc-tune v1 a") == "rag_streams=4"
    gfc.tune_cache_put(path, "gfc-tune v1 a", "rag_streams=8")  # replaced, b kept
    assert gfc.tune_cache_get(path, "gfc-tune v1 a") == "rag_streams=8"
    assert gfc.tune_cache_get(path, "gfc-tune v1 b") == "rag_streams=2"
    lines = open(path).read().splitlines()
    assert len(lines) == 2 and all("\t" in ln for ln in lines)


def test_key_mismatch_is_a_miss(tmp_path):
    """A key that is a prefix of a stored key (or the other way round) is not a hit:
    a build or device change yields a different key and a fresh tuning."""
    path = str(tmp_path / "tune.txt")
    gfc.tune_cache_put(path, "gfc-tune v1 build=abc dev=X kind=uniform H=8", "column_solver=1 chunk=0 streams=1")
    assert gfc.tune_cache_get(path, "gfc-tune v1 build=abc dev=X kind=uniform H=8") is not None
    assert gfc.tune_cache_get(path, "gfc-tune v1 build=abc dev=X kind=uniform H=80") is None
    assert gfc.tune_cache_get(path, "gfc-tune v1 build=abc dev=X kind=uniform H=") is None
    assert gfc.tune_cache_get(path, "gfc-tune v1 build=abd dev=X kind=uniform H=8") is None


def test_bad_entries_are_rejected(tmp_path):
    path = str(tmp_path / "tune.txt")
    with pytest.raises(gfc.GFCError):
        gfc.tune_cache_put(path, "a\tb", "v")
    with pytest.raises(gfc.GFCError):
        gfc.tune_cache_put(path, "a", "v\nw")
    with pytest.raises(gfc.GFCError):
        gfc.tune_cache_put(str(tmp_path / "no" / "such" / "dir" / "t.txt"), "a", "v")
