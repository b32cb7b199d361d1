"""The GPU service: each request's result is the same alone and in the mix."""
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


@pytest.mark.parametrize("storage", ["f16", "f32", "f16s"])
def test_results_alone_equal_results_in_the_mix(lbm, storage):
    from paper_1002_3028_gb300.serve import GpuBatchEngine, serve

    reqs = I.request_stream(count=14, rate_per_s=400.0, seed=5, min_steps=20, max_steps=300)
    eng = GpuBatchEngine(storage)
    budget = 3.5 * max(eng.bytes_needed(r) for r in reqs)  # forces queueing and joins
    stats = serve(reqs, eng, budget, chunk=48, keep_fields=True)
    assert len(stats.results) == len(reqs)
    for res in stats.results:
        w = reqs[res.rid].workload
        alone = lbm.Lattice.from_workload(w, storage)
        alone.step(w.steps)
        ref = alone.fields(dtype=torch.float32).cpu()
        assert torch.equal(res.fields, ref), res.rid
        alone.close()
    assert stats.mlups > 0 and stats.percentile(99) >= stats.percentile(50)
