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


@pytest.mark.parametrize("storage,pattern", [("f64", "ab"), ("f32", "ab"), ("f16", "ab"), ("bf16", "ab"),
                                             ("f16s", "ab"), ("bf16s", "ab"), ("f32", "aa"), ("bf16", "aa")])
def test_noalloc_equals_diagnostics_on_two_calls(lbm, storage, pattern):
    """Two calls in a row, at an odd and an even step count (the AA pattern's two
    representations), equal lbm_diagnostics; an AA lattice keeps no previous state, so both
    entry points report no residual for it."""
    w = I.jet_workload(nx=300, nr=70, R=20.0, ntab=64)
    lat = lbm.Lattice.from_workload(w, storage, pattern=pattern)
    L = lbm.lib()
    for n in range(2):
        lat.step(25 + 8 * n)  # 25, then 58 steps
        rc_a, a = call(lbm, L.lbm_diagnostics, lat)
        rc_b, b = call(lbm, L.lbm_diagnostics_noalloc, lat)
        assert rc_a == rc_b == 0
        same(b, a)
        assert b["mass"] > 0 and math.isnan(b["residual_max"]) == (pattern == "aa")
    lat.close()


def test_noalloc_allocates_nothing_and_leaves_the_lattice_memory_alone(lbm):
    """After a first call, further calls change neither the free device memory nor the
    caching allocator's reserved bytes, and no byte of the lattice's own device block
    (its populations, tables, counters and scratch area) is written."""
    w = I.jet_workload(nx=300, nr=70, R=20.0, ntab=64)
    lat = lbm.Lattice.from_workload(w, "f32")
    lat.step(30)
    L = lbm.lib()
    assert call(lbm, L.lbm_diagnostics_noalloc, lat)[0] == 0
    block0 = lat._mem.clone()  # the lattice's whole device block, as the library laid it out
    torch.cuda.synchronize()
    free, reserved = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for _ in range(3):
        rc, d = call(lbm, L.lbm_diagnostics_noalloc, lat)
        assert rc == 0 and d["mass"] > 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free
    assert torch.cuda.memory_reserved() == reserved
    assert torch.equal(lat._mem, block0)
    lat.close()


def test_noalloc_takes_the_largest_lattice_its_array_holds(lbm):
    cfg = I.LatticeConfig(nx=2, nr=16384, bc_in="periodic", bc_out="periodic", bc_top="wall", T_top=1.0)
    lat = lbm.Lattice(cfg, "f32")
    f0, g0 = I.random_state(2, 16384, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, [0.25] * 4, 0.02, 5)
    lat.set_state(f0, g0, 0)
    lat.step(3)
    L = lbm.lib()
    rc_a, a = call(lbm, L.lbm_diagnostics, lat)
    rc_b, b = call(lbm, L.lbm_diagnostics_noalloc, lat)
    assert rc_a == rc_b == 0
    same(b, a)
    lat.close()


def test_noalloc_refuses_more_rows_than_its_array(lbm):
    cfg = I.LatticeConfig(nx=1, nr=16385, bc_in="periodic", bc_out="periodic", bc_top="wall", T_top=1.0)
    lat = lbm.Lattice(cfg, "f32")
    rc, _ = call(lbm, lbm.lib().lbm_diagnostics_noalloc, lat)
    assert rc == -1
    assert "16384" in lbm.lib().lbm_last_error().decode()
    lat.close()
