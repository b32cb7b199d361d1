"""The autotuner's ranking on the CPU, against a fake lattice and scripted timings: each shape
runs three times and is ranked by its slowest run, so a shape whose launches fall into a slow
schedule part of the time loses to a steady one; the choice is applied and cached."""
import json

import pytest

from paper_1002_3028_gb300 import autotune


class FakeLattice:
    storage = "f32"
    pattern = "ab"
    nx, nr = 4096, 1024

    def __init__(self):
        self.shape = None
        self.steps = 0
        self.applied = []

    def set_strip_width(self, cols):
        self.cols = cols

    def set_launch(self, band, warps):
        self.shape = (self.cols, band, warps)
        self.applied.append(self.shape)

    def step(self, n):
        self.steps += n


@pytest.fixture
def tuner(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "fake GPU")
    return autotune


def test_a_shape_with_slow_runs_loses_to_a_steady_one(tuner, monkeypatch):
    lat = FakeLattice()
    # (64, 6, 1) runs fast, slow, fast; (64, 5, 1) steadily between the two
    script = {(64, 6, 1): iter([0.0780, 0.0860, 0.0781]), (64, 5, 1): iter([0.0800, 0.0801, 0.0799])}
    monkeypatch.setattr(tuner, "_time", lambda run, steps, warmup: next(script[lat.shape]))
    shape = tuner.tune(lat, candidates=[(64, 6, 1), (64, 5, 1)], steps=10, warmup=2)
    assert shape == (64, 5, 1) and lat.shape == (64, 5, 1)
    # three runs each, in alternating orders
    assert lat.applied[:6] == [(64, 6, 1), (64, 5, 1), (64, 5, 1), (64, 6, 1), (64, 6, 1), (64, 5, 1)]
    (entry,) = json.load(open(tuner.CACHE)).values()
    assert (entry["strip"], entry["band"], entry["warps"]) == (64, 5, 1)
    assert entry["ms_per_step"] == pytest.approx(0.0801)
    assert [t[:3] for t in entry["timings"]] == [[64, 5, 1], [64, 6, 1]]
    assert entry["timings"][1][3] == pytest.approx(0.0860)


def test_the_cached_shape_is_applied_without_timing(tuner, monkeypatch):
    lat = FakeLattice()
    monkeypatch.setattr(tuner, "_time", lambda run, steps, warmup: 0.05 if lat.shape[1] == 4 else 0.06)
    assert tuner.tune(lat, candidates=[(64, 4, 1), (32, 8, 1)], steps=10, warmup=2) == (64, 4, 1)
    other = FakeLattice()
    monkeypatch.setattr(tuner, "_time", lambda run, steps, warmup: pytest.fail("timed a cached shape"))
    assert tuner.tune(other, candidates=[(64, 4, 1), (32, 8, 1)]) == (64, 4, 1)
    assert other.shape == (64, 4, 1) and other.steps == 0


def test_fp64_takes_only_32_column_strips(tuner, monkeypatch):
    lat = FakeLattice()
    lat.storage = "f64"
    monkeypatch.setattr(tuner, "_time", lambda run, steps, warmup: 0.1)
    assert tuner.tune(lat, candidates=[(64, 4, 1), (32, 2, 1)], steps=10, warmup=2) == (32, 2, 1)
    other = FakeLattice()
    other.storage = "f64"
    with pytest.raises(ValueError):  # no candidate of a width FP64 accepts
        tuner.tune(other, candidates=[(64, 4, 1)], use_cache=False)


def test_the_cache_keeps_the_two_memory_patterns_apart(tuner, monkeypatch):
    ab = FakeLattice()
    monkeypatch.setattr(tuner, "_time", lambda run, steps, warmup: 0.05 if ab.shape[0] == 32 else 0.06)
    assert tuner.tune(ab, candidates=[(64, 4, 1), (32, 8, 1)], steps=10, warmup=2) == (32, 8, 1)
    aa = FakeLattice()  # same storage and shape, one buffer updated in place: 64-column strips only
    aa.pattern = "aa"
    monkeypatch.setattr(tuner, "_time", lambda run, steps, warmup: 0.07)
    assert tuner.tune(aa, candidates=[(64, 4, 1), (32, 8, 1)], steps=10, warmup=2) == (64, 4, 1)
    assert len(json.load(open(tuner.CACHE))) == 2
