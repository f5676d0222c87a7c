"""The batch autotuner's cache file (CPU; no GPU call): entries written by
mhc_tune_cache_put are JSON lines that mhc_tune_cache_get reads back, the last entry of a
key wins, and an empty MHC_TUNE_CACHE turns the cache off."""
import json

import pytest


@pytest.fixture(scope="module")
def M():
    from paper_1411_3691_gb300 import build as B
    B.build()
    from paper_1411_3691_gb300 import mhc
    return mhc


def test_put_get_round_trip(M, tmp_path, monkeypatch):
    path = tmp_path / "tune.jsonl"
    monkeypatch.setenv("MHC_TUNE_CACHE", str(path))
    key = "gpu=X sm152;build=b;nc=18;shapes=18/96,18/96"
    assert M.mhc_tune_cache_get(key) == 0
    M.mhc_tune_cache_put(key, 64)
    M.mhc_tune_cache_put("gpu=X sm152;build=b;nc=8;shapes=6/48,6/48", 128)
    assert M.mhc_tune_cache_get(key) == 64
    M.mhc_tune_cache_put(key, 32)                       # a later entry replaces it
    assert M.mhc_tune_cache_get(key) == 32
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert [d["tile"] for d in lines] == [64, 128, 32]
    assert all(set(d) == {"key", "tile", "ms"} and len(d["ms"]) == 3 for d in lines)


def test_bad_entries_rejected(M, tmp_path, monkeypatch):
    monkeypatch.setenv("MHC_TUNE_CACHE", str(tmp_path / "t.jsonl"))
    for key, tile in (("a\"b", 64), ("", 64), ("ok", 48)):
        with pytest.raises(M.MHCError) as e:
            M.mhc_tune_cache_put(key, tile)
        assert e.value.status == M.MHC_EINVAL


def test_cache_disabled(M, monkeypatch):
    monkeypatch.setenv("MHC_TUNE_CACHE", "")
    assert M.mhc_tune_cache_get("k") == 0
    with pytest.raises(M.MHCError):
        M.mhc_tune_cache_put("k", 64)
