"""Host logic of the plan cache (paper_1404_3458_gb300/tuning.py), on the CPU
with a stand-in context: plans come from lch_autotune only when the cache has
none for the shape, are installed with lch_tune_set otherwise, and a cache
written under another GPU or library build is ignored."""
import json

from paper_1404_3458_gb300 import tuning


class FakeCtx:
    def __init__(self):
        self.tuned, self.installed = [], []

    def autotune(self, field, h, S, stream=None):
        self.tuned.append((field, h, S))
        return {"split": (h.bit_length() - 1 + 1) // 2, "lg_tile_low": 8, "lg_tile_high": 8, "ms": 1.0}

    def tune_set(self, field, h, S, plan):
        self.installed.append((field, h, S, plan["split"]))


def test_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setattr(tuning, "_device_key", lambda: "GB300|sm_103|1")
    path = str(tmp_path / "plans.json")
    shapes = [(16, 65536, 4096), (16, 32768, 4096), (8, 1, 64)]  # h = 1 has no transform to tune
    c1 = FakeCtx()
    plans = tuning.tune(c1, shapes, path)
    assert c1.tuned == [(16, 65536, 4096), (16, 32768, 4096)] and c1.installed == []
    assert set(plans) == {"16/65536/4096", "16/32768/4096"}
    with open(path) as f:
        data = json.load(f)
    assert data["device"] == "GB300|sm_103|1" and set(data["plans"]) == set(plans)
    # a second run installs the cached plans and times nothing
    c2 = FakeCtx()
    assert tuning.tune(c2, shapes, path) == plans
    assert c2.tuned == [] and sorted(c2.installed) == [(16, 32768, 4096, 8), (16, 65536, 4096, 8)]


def test_cache_of_another_device_or_build_is_ignored(tmp_path, monkeypatch):
    path = str(tmp_path / "plans.json")
    monkeypatch.setattr(tuning, "_device_key", lambda: "GB300|sm_103|1")
    tuning.tune(FakeCtx(), [(16, 1024, 512)], path)
    monkeypatch.setattr(tuning, "_device_key", lambda: "GB300|sm_103|2")  # rebuilt library
    assert tuning.load(path) == {}
    c = FakeCtx()
    tuning.tune(c, [(16, 1024, 512)], path)
    assert c.tuned == [(16, 1024, 512)]
    assert json.load(open(path))["device"] == "GB300|sm_103|2"


def test_unreadable_cache_is_empty(tmp_path, monkeypatch):
    monkeypatch.setattr(tuning, "_device_key", lambda: "k")
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    assert tuning.load(str(bad)) == {}
    assert tuning.load(str(tmp_path / "missing.json")) == {}
    assert tuning.tune(FakeCtx(), [], None) == {}
