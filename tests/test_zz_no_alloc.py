"""lbm_diagnostics_noalloc, the diagnostics entry point that allocates nothing.

It serves callers that cannot allocate device memory (their device memory
is owned by another allocator or must stay fixed after set-up): its partial
sums live in a fixed array inside the library instead of the lattice's
scratch area.  These tests call it through the C ABI and check it against
lbm_diagnostics on two calls in a row, and that it refuses lattices larger
than its array.  This file is collected last on purpose.
"""
import ctypes as C
import math

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


def call(lbm, fn, lat):
    d = lbm.Diag()
    rc = fn(lat.handle, C.byref(d), C.c_void_p(int(torch.cuda.current_stream().cuda_stream)))
    return rc, d.as_dict()


def same(a, b, rel=1e-11):
    for k, va in a.items():
        vb = b[k]
        if k == "nonfinite":
            assert va == vb, k
        elif math.isnan(va) or math.isnan(vb):
            assert math.isnan(va) and math.isnan(vb), k
        else:
            assert va == pytest.approx(vb, rel=rel, abs=1e-300), k


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_noalloc_equals_diagnostics_on_two_calls(lbm, storage):
    w = I.jet_workload(nx=300, nr=70, R=20.0, ntab=64)
    lat = lbm.Lattice.from_workload(w, storage)
    L = lbm.lib()
    for n in range(2):
        lat.step(25 + 7 * n)
        rc_a, a = call(lbm, L.lbm_diagnostics, lat)
        rc_b, b = call(lbm, L.lbm_diagnostics_noalloc, lat)
        assert rc_a == rc_b == 0
        same(b, a)
        assert b["mass"] > 0 and not math.isnan(b["residual_max"])
    lat.close()


def test_noalloc_refuses_more_rows_than_its_array(lbm):
    cfg = I.LatticeConfig(nx=1, nr=16385, bc_in="periodic", bc_out="periodic", bc_top="wall", T_top=1.0)
    lat = lbm.Lattice(cfg, "f32")
    rc, _ = call(lbm, lbm.lib().lbm_diagnostics_noalloc, lat)
    assert rc == -1
    assert "16384" in lbm.lib().lbm_last_error().decode()
    lat.close()
