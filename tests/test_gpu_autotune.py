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
    cands = [(64, 2, 1), (32, 4, 1)]
    lat = lbm.Lattice.from_workload(w, "f32")
    shape = autotune.tune(lat, candidates=cands, steps=60, warmup=5)
    assert shape in cands
    assert (lat.strip_width, *lat.launch()[:2]) == shape
    assert lat.step_count == 60 + 3 * 2 * 65  # tuning steps the lattice: a warm-up, then each candidate three times
    data = json.load(open(autotune.CACHE))
    (entry,) = data.values()
    assert (entry["strip"], entry["band"], entry["warps"]) == shape and len(entry["timings"]) == 2
    # a second lattice of the same kind takes the cached shape without being stepped
    other = lbm.Lattice.from_workload(w, "f32")
    assert autotune.tune(other, candidates=cands) == shape
    assert (other.strip_width, *other.launch()[:2]) == shape and other.step_count == 0


def test_tune_picks_a_non_default_tile_and_results_do_not_change(lbm, tmp_path, monkeypatch):
    """The tuner sets a 32-column tile (one node per lane) when it is the candidate it finds
    fastest; the tuned lattice then advances exactly like one at the default 64-column tile."""
    from paper_1002_3028_gb300 import autotune

    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    w = I.jet_workload(nx=300, nr=70)
    tuned = lbm.Lattice.from_workload(w, "f16s")
    shape = autotune.tune(tuned, candidates=[(32, 3, 1)], steps=20, warmup=2)
    assert shape == (32, 3, 1) and tuned.strip_width == 32
    ref = lbm.Lattice.from_workload(w, "f16s")
    assert ref.strip_width == 64
    ref.step(tuned.step_count)
    tuned.step(30)
    ref.step(30)
    assert torch.equal(tuned.save()[0], ref.save()[0])


def test_strip_widths_a_storage_type_accepts(lbm):
    w = I.jet_workload(nx=100, nr=20)
    lat = lbm.Lattice.from_workload(w, "f64")
    assert lat.strip_width == 32
    with pytest.raises(lbm.LbmError):
        lat.set_strip_width(64)  # FP64 has no paired form
    with pytest.raises(lbm.LbmError):
        lbm.Lattice.from_workload(w, "f32").set_strip_width(48)
    aa = lbm.Lattice.from_workload(w, "f32", pattern="aa")
    with pytest.raises(lbm.LbmError):
        aa.set_strip_width(32)


def test_tune_a_batch(lbm, tmp_path, monkeypatch):
    from paper_1002_3028_gb300 import autotune

    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    b = lbm.Batch("f16")
    for nx, nr in ((256, 64), (320, 96), (192, 32)):
        b.add(lbm.Lattice.from_workload(I.jet_workload(nx=nx, nr=nr), "f16"))
    cands = [(64, 4, 1), (64, 8, 1), (32, 8, 1)]
    shape = autotune.tune(b, candidates=cands, steps=40, warmup=4)
    assert shape in cands
    b.step(1, graph=False)  # a batch reports the shape of the tables its last step used
    assert (b.strip_width, *b.launch()[:2]) == shape
