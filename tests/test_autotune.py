"""Host logic of the batched-form autotuner: job-set classes and the JSON
cache (no GPU)."""
import json

from paper_1802_09488_gb300 import autotune


class FakeIndex:
    def __init__(self, nodes, mode):
        self._s = {"n_nodes": nodes, "mode": mode}

    def stats(self):
        return self._s


def test_key_classes():
    a, e = FakeIndex(1000, 0), FakeIndex(50, 1)
    k1 = autotune.key([a, e], [1 << 20, 1 << 20])
    assert k1 == "p21-n5-e5-m1"          # log4(1050 nodes) = 5.0
    # shared indexes count once; points, exact share and job count set the class
    assert autotune.key([a, a, e], [1 << 19, 1 << 19, 1 << 20]) == "p21-n5-e5-m1"
    assert autotune.key([a], [1 << 20]) == "p20-n4-e0-m0"
    assert autotune.key([e], [5]) == "p2-n2-e10-m0"


def test_cache_roundtrip(tmp_path, monkeypatch):
    p = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("AGJ_AUTOTUNE_CACHE", str(p))
    assert autotune.cache_path() == str(p)
    assert autotune._load() == {}
    autotune._store({"k": {"points_per_lane": 4, "ctas_per_sm": 0, "ms": 1.5}})
    assert json.loads(p.read_text())["k"]["points_per_lane"] == 4
    assert autotune._load()["k"]["ctas_per_sm"] == 0
