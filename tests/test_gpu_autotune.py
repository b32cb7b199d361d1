"""The launch-shape autotuner on the GPU: it applies and caches the fastest candidate."""
import json

import pytest

from paper_1002_3028_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_3028_gb300 import lbm as L

    L.lib()
    return L


def test_tune_applies_and_caches_a_candidate(lbm, tmp_path, monkeypatch):
    from paper_1002_3028_gb300 import autotune

    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    w = I.jet_workload(nx=512, nr=128)
    cands = [(2, 1), (4, 1)]
    lat = lbm.Lattice.from_workload(w, "f32")
    band, warps = autotune.tune(lat, candidates=cands, steps=60, warmup=5)
    assert (band, warps) in cands
    assert lat.launch()[:2] == (band, warps)
    assert lat.step_count == 60 + 2 * 2 * 65  # tuning steps the lattice: a warm-up, then each candidate twice
    data = json.load(open(autotune.CACHE))
    (entry,) = data.values()
    assert (entry["band"], entry["warps"]) == (band, warps) and len(entry["timings"]) == 2
    # a second lattice of the same kind takes the cached shape without being stepped
    other = lbm.Lattice.from_workload(w, "f32")
    assert autotune.tune(other, candidates=cands) == (band, warps)
    assert other.launch()[:2] == (band, warps) and other.step_count == 0


def test_tune_a_batch(lbm, tmp_path, monkeypatch):
    from paper_1002_3028_gb300 import autotune

    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    b = lbm.Batch("f16")
    for nx, nr in ((256, 64), (320, 96), (192, 32)):
        b.add(lbm.Lattice.from_workload(I.jet_workload(nx=nx, nr=nr), "f16"))
    cands = [(4, 1), (8, 1)]
    shape = autotune.tune(b, candidates=cands, steps=40, warmup=4)
    assert shape in cands
    b.step(1, graph=False)  # a batch reports the shape of the tables its last step used
    assert b.launch()[:2] == shape
