"""The autotuner's JSON cache (host code, no GPU): lookup of a missing file
or key, store / replace round trip, the file stays valid JSON, and invalid
entries are refused."""
import json

import numpy as np
import pytest

from paper_2510_27117_b300 import gfors as G


def test_cache_round_trip(tmp_path):
    path = tmp_path / "tune.json"
    assert G.tune_cache_lookup(path, "dev|N20") is None           # no file yet
    a = np.array([1, 2, 4, 8, 16, 1, 1, 4, 32, 32], np.int32)
    b = np.array([2, 2, 2, 2, 2, 4, 4, 4, 4, 4], np.int32)
    G.tune_cache_store(path, "dev|N20", a)
    G.tune_cache_store(path, "dev|N21|r3.-1", b)
    assert np.array_equal(G.tune_cache_lookup(path, "dev|N20"), a)
    assert np.array_equal(G.tune_cache_lookup(path, "dev|N21|r3.-1"), b)
    assert G.tune_cache_lookup(path, "dev|N22") is None
    d = json.loads(path.read_text())
    assert d["dev|N20"] == {"rows": [1, 2, 4, 8, 16], "cols": [1, 1, 4, 32, 32]}
    G.tune_cache_store(path, "dev|N20", b)                         # replace, not append
    assert np.array_equal(G.tune_cache_lookup(path, "dev|N20"), b)
    assert len(json.loads(path.read_text())) == 2


def test_cache_refuses_invalid_entries(tmp_path):
    path = tmp_path / "tune.json"
    with pytest.raises(G.GforsError):
        G.tune_cache_store(path, "k", np.array([3] * 10, np.int32))     # not a lane count
    with pytest.raises(G.GforsError):
        G.tune_cache_store(path, 'bad"key', np.ones(10, np.int32))
    with pytest.raises(G.GforsError):
        G.tune_cache_store(tmp_path / "no_dir" / "t.json", "k", np.ones(10, np.int32))
    assert not path.exists()
