"""The AA pattern (one population buffer updated in place) against the two-buffer path and the oracle.

Both patterns apply the same arithmetic to the same stored values in the same
order; only where a value is kept differs.  Every result of an AA lattice must
therefore equal the two-buffer lattice's bit for bit: stored populations,
fields, checkpoints, and the diagnostics except the steady residual, which an
AA lattice cannot form since it keeps no previous state.  This must hold
after odd and even step counts (the two representations of the AA state),
for every boundary kind, storage type, launch shape and item group, alone and
in batches.  FP64 AA steps are also compared with the oracle directly, at its
1e-12 bar.
"""
import math
import os

import numpy as np
import pytest

from paper_1002_3028_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NTHREADS = max(1, min(8, os.cpu_count() or 1))

BOUNDARIES = {
    "jet": dict(bc_in="inlet", bc_out="outflow", bc_top="open", bc_bottom="axis"),
    "pipe": dict(bc_in="inlet", bc_out="outflow", bc_top="wall", bc_bottom="axis"),
    "periodic_axis": dict(bc_in="periodic", bc_out="periodic", bc_top="wall", bc_bottom="axis"),
    "annulus": dict(bc_in="periodic", bc_out="periodic", bc_top="wall", bc_bottom="wall", r0=5.0),
    "substrate": dict(bc_in="inlet", bc_out="wall", bc_top="open", bc_bottom="axis"),
    "inner_wall_pipe": dict(bc_in="inlet", bc_out="outflow", bc_top="wall", bc_bottom="wall", r0=3.0),
    "open_periodic": dict(bc_in="periodic", bc_out="periodic", bc_top="open", bc_bottom="axis"),
}


@pytest.fixture(scope="module")
def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_3028_gb300 import lbm as L

    L.lib()
    return L


def workload(nx, nr, bc_in="inlet", bc_out="outflow", bc_top="open", bc_bottom="axis", r0=0.0):
    R = max(1.0, nr / 3.0)
    cfg = I.LatticeConfig(nx=nx, nr=nr, bc_in=bc_in, bc_out=bc_out, bc_top=bc_top, bc_bottom=bc_bottom, r0=r0,
                          Cs=0.17, Pr_t=0.3, T_top=1.2, T_bottom=1.5, T_out=0.8, noise_amp=1e-3, seed=99)
    u_in, T_in = I.jet_profiles(nr, R, 0.06, 1.0, 4.0)
    nu, al = I.power_law_tables(64, 0.8, 4.0, nu_max=0.2)
    return I.Workload("case", cfg, u_in, T_in, nu, al, 0.8, 4.0)


def twins(lbm, orc, w, storage, seed=21, step=3):
    ab = lbm.Lattice.from_workload(w, storage)
    aa = lbm.Lattice.from_workload(w, storage, pattern="aa")
    f0, g0 = I.random_state(w.cfg.nx, w.cfg.nr, orc.feq(1.0, 0.02, 0.0), orc.geq(1.2, 0.02, 0.0), 0.05, seed)
    for lat in (ab, aa):
        lat.set_state(f0, g0, step)
    return ab, aa


def assert_same(ab, aa):
    a, sa = ab.save()
    b, sb = aa.save()
    assert sa == sb
    assert torch.equal(a, b)
    assert torch.equal(ab.fields(), aa.fields())
    for x, y in zip(ab.get_state(), aa.get_state()):
        assert torch.equal(x, y)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("bname", sorted(BOUNDARIES))
def test_aa_equals_two_buffers(lbm, orc, bname, storage):
    """150 x 45: several strips (a ragged last one) and bands; chunks of 1, 2, 7 and 24
    steps leave the AA state in both representations."""
    ab, aa = twins(lbm, orc, workload(150, 45, **BOUNDARIES[bname]), storage)
    for n in (1, 2, 7, 24):
        ab.step(n)
        aa.step(n)
        assert_same(ab, aa)
    assert ab.check() == 0 and aa.check() == 0


@pytest.mark.parametrize("band,warps,group", [
    (1, 1, 1), (4, 1, 1), (5, 2, 1), (0, 1, 2), (7, 4, 3), (0, 8, 1), (61, 2, 2), (1000, 1, 5),
])
@pytest.mark.parametrize("bname", ["jet", "open_periodic"])
def test_aa_launch_shape_does_not_change_results(lbm, orc, bname, band, warps, group):
    """Bands (below the 4-row floor, one band for the whole lattice), warps per CTA and
    items of several strips give the two-buffer result exactly."""
    w = workload(300, 61, **BOUNDARIES[bname])
    ab, aa = twins(lbm, orc, w, "f32", seed=5)
    aa.set_launch(band, warps)
    aa.set_item_group(group)
    b, _, _ = aa.launch()
    assert b >= 4 and (band < 4 or b == min(band, 61) or band == 1000)
    for n in (3, 10):
        ab.step(n)
        aa.step(n)
        assert_same(ab, aa)
    assert aa.check() == 0


@pytest.mark.parametrize("size", [(1, 1), (2, 1), (1, 2), (3, 3), (33, 5), (64, 32), (70, 19)],
                         ids=lambda s: f"{s[0]}x{s[1]}")
@pytest.mark.parametrize("bname", ["jet", "pipe", "periodic_axis", "annulus"])
def test_aa_f64_matches_oracle(lbm, orc, bname, size):
    """FP64 AA steps against the oracle, including lattices too small for the
    multi-step schedule (one step per launch)."""
    w = workload(*size, **BOUNDARIES[bname])
    o = orc.Oracle.from_workload(w, NTHREADS)
    g = lbm.Lattice.from_workload(w, "f64", pattern="aa")
    f0, g0 = I.random_state(*size, orc.feq(1.0, 0.02, 0.0), orc.geq(1.3, 0.02, 0.0), 0.05, 1)
    o.set_state(f0, g0, 5)
    g.set_state(f0, g0, 5)
    for n in (1, 1, 2):
        o.step(n)
        g.step(n)
        f, gg = g.get_state()
        fo, go = o.get_state()
        for a, b in ((f, fo), (gg, go)):
            a = a.cpu().numpy()
            for q in range(b.shape[0]):
                scale = max(float(np.max(np.abs(b[q]))), 1.0)
                assert float(np.max(np.abs(a[q] - b[q]))) / scale < 1e-12
    assert g.step_count == o.step_count == 9


def test_aa_jet_1024x256_matches_oracle_per_step(lbm, orc):
    """The single-jet configuration (FP64, AA) one step at a time from a developed oracle state."""
    w = I.jet_workload(nx=1024, nr=256)
    o = orc.Oracle.from_workload(w, NTHREADS)
    o.step(300)
    f0, g0 = o.get_state()
    g = lbm.Lattice.from_workload(w, "f64", pattern="aa")
    g.set_state(f0, g0, o.step_count)
    for _ in range(2):
        o.step(1)
        g.step(1)
        f, gg = g.get_state()
        fo, go = o.get_state()
        for a, b in ((f, fo), (gg, go)):
            a = a.cpu().numpy()
            for q in range(b.shape[0]):
                assert float(np.max(np.abs(a[q] - b[q]))) / float(np.max(np.abs(b[q]))) < 1e-12


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_aa_diagnostics_equal_two_buffers(lbm, orc, storage):
    """Mass, heat and speed equal the two-buffer lattice's exactly; an AA lattice keeps no
    previous state, so its residual is NaN."""
    ab, aa = twins(lbm, orc, workload(97, 40), storage, seed=8)
    for n in (1, 4, 3):
        ab.step(n)
        aa.step(n)
        da, db = ab.diagnostics(), aa.diagnostics()
        for key in ("mass", "mass_axi", "heat", "heat_axi", "max_speed", "nonfinite", "diverged"):
            assert da[key] == db[key]
        assert not math.isnan(da["residual_l2"])
        assert math.isnan(db["residual_l2"]) and math.isnan(db["residual_max"])
    from paper_1002_3028_gb300.lbm import Diag, _stream_ptr
    import ctypes as C

    out = Diag()
    assert aa._L.lbm_diagnostics_noalloc(aa.handle, C.byref(out), _stream_ptr(None)) == 0
    assert math.isnan(out.residual_l2)
    assert out.mass == pytest.approx(da["mass"], rel=1e-14)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_aa_checkpoints_cross_patterns(lbm, orc, storage):
    """A checkpoint has the same layout for both patterns: one taken from either, at an odd
    or even step, resumes exactly on the other."""
    ab, aa = twins(lbm, orc, workload(150, 45), storage, seed=12)
    ab.step(5)
    aa.step(5)  # odd: the AA state is in its second representation
    cka, step = ab.save()
    ckb, _ = aa.save()
    assert torch.equal(cka, ckb)
    ab2 = lbm.Lattice.from_workload(workload(150, 45), storage)
    aa2 = lbm.Lattice.from_workload(workload(150, 45), storage, pattern="aa")
    aa2.restore(cka, step)  # two-buffer checkpoint into AA
    ab2.restore(ckb, step)  # AA checkpoint into two buffers
    for lat in (ab, aa, ab2, aa2):
        lat.step(8)
    ref, _ = ab.save()
    for lat in (aa, ab2, aa2):
        assert torch.equal(lat.save()[0], ref)


def test_aa_inlet_change_in_either_representation(lbm, orc):
    """A new inlet profile set after an odd or an even number of steps rewrites the
    boundary values of the AA state wherever that representation keeps them."""
    w = workload(150, 45)
    ab, aa = twins(lbm, orc, w, "f32", seed=4)
    for n, scale in ((3, 1.5), (4, 0.5)):
        ab.step(n)
        aa.step(n)
        for lat in (ab, aa):
            lat.set_inlet(w.u_in * scale, w.T_in * (0.5 + scale / 2))
        ab.step(6)
        aa.step(6)
        assert_same(ab, aa)


@pytest.mark.parametrize("storage", ["f32", "f16", "f64"])
def test_aa_bounded_waits_time_out_and_leave_the_lattice_usable(lbm, orc, storage):
    ab, aa = twins(lbm, orc, workload(150, 45), storage, seed=31)
    ab.step(3)
    aa.step(3)
    before, _ = aa.save()
    assert aa.selftest_wait_timeout() == 1  # LBM_STATUS_TIMEOUT
    after, step = aa.save()
    assert step == 6 and torch.equal(before, after)
    assert aa.check() == 0
    ab.step(5)
    aa.step(5)
    assert_same(ab, aa)


def test_aa_memory_and_batches(lbm):
    cfg = I.jet_workload(nx=4096, nr=1024).cfg
    per_node = {}
    for storage in ("f64", "f32", "f16"):
        b_ab = lbm.required_bytes(cfg, storage)
        b_aa = lbm.required_bytes(cfg, storage, "aa")
        per_node[storage] = (b_ab / (4096 * 1024), b_aa / (4096 * 1024))
    # padded planes: about 3% above 26 (or 13) values per node; AA adds about 1.5 edge moments
    assert per_node["f32"][0] == pytest.approx(104, rel=0.05) and per_node["f32"][1] == pytest.approx(58, rel=0.05)
    assert per_node["f16"][0] == pytest.approx(52, rel=0.05) and per_node["f16"][1] == pytest.approx(32, rel=0.05)
    assert per_node["f64"][1] == pytest.approx(116, rel=0.05)
    aa = lbm.Lattice(I.LatticeConfig(nx=64, nr=16), "f16", pattern="aa")
    ab = lbm.Lattice(I.LatticeConfig(nx=64, nr=16), "f16")
    batch = lbm.Batch("f16")
    batch.add(aa)
    with pytest.raises(lbm.LbmError):  # the members of a batch share one pattern
        batch.add(ab)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_aa_full_size_4096x1024(lbm, orc, storage):
    """The 4096 x 1024 jet in the AA layout: 5 steps of one launch equal the two-buffer lattice's."""
    w = I.jet_workload(nx=4096, nr=1024)
    ab = lbm.Lattice.from_workload(w, storage)
    aa = lbm.Lattice.from_workload(w, storage, pattern="aa")
    for lat in (ab, aa):
        lat.step(5)
    assert torch.equal(ab.save()[0], aa.save()[0])
    assert torch.equal(ab.fields(), aa.fields())
    assert aa.check() == 0


@pytest.mark.parametrize("storage", ["f32", "f16", "f64"])
def test_aa_batch_members_equal_two_buffer_lattices_alone(lbm, orc, storage):
    """A batch of ragged AA lattices (every boundary set, one of them a single tile)
    advances every member exactly as a two-buffer lattice stepped alone: through graph
    replays of 64 steps and a remainder launch, and after members leave and join."""
    sizes = [(150, 45), (64, 16), (33, 5), (200, 70), (97, 40), (40, 9), (300, 61)]
    names = sorted(BOUNDARIES)
    pairs = []
    batch = lbm.Batch(storage)
    for m, ((nx, nr), bname) in enumerate(zip(sizes, names)):
        ab, aa = twins(lbm, orc, workload(nx, nr, **BOUNDARIES[bname]), storage, seed=40 + m)
        pairs.append((ab, aa))
        batch.add(aa)
    for n in (1, 64 + 37):
        batch.step(n, graph=True)
        for ab, _ in pairs:
            ab.step(n)
        for ab, aa in pairs:
            assert_same(ab, aa)
    batch.remove(pairs[2][1])
    pairs[2][0].close()
    batch.step(7, graph=False)
    for k, (ab, aa) in enumerate(pairs):
        if k != 2:
            ab.step(7)
            assert_same(ab, aa)
        assert aa.check() == 0


def test_aa_serving_engine_admits_by_aa_size(lbm):
    """The serving engine with AA lattices counts their smaller footprint for admission."""
    from paper_1002_3028_gb300.serve import GpuBatchEngine

    w = I.ensemble_workloads(1, seed=7)[0]
    req = I.Request(0, 0.0, w)
    ab, aa = GpuBatchEngine("f16"), GpuBatchEngine("f16", pattern="aa")
    assert aa.bytes_needed(req) < 0.75 * ab.bytes_needed(req)
    lat = aa.admit(req)
    aa.step(10)
    assert lat.step_count == 10 and lat.check() == 0


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_aa_lattice_joins_and_leaves_a_batch_in_either_representation(lbm, orc, storage):
    """Members join after odd and even step counts of their own (so in either representation),
    run in the batch, then leave and step alone again: all equal two-buffer lattices alone."""
    pairs = []
    batch = lbm.Batch(storage)
    for m, (bname, alone) in enumerate([("jet", 3), ("periodic_axis", 4), ("substrate", 5)]):
        ab, aa = twins(lbm, orc, workload(150, 45, **BOUNDARIES[bname]), storage, seed=60 + m)
        ab.step(alone)
        aa.step(alone)
        batch.add(aa)
        pairs.append((ab, aa))
    batch.step(67, graph=True)
    for ab, _ in pairs:
        ab.step(67)
    for ab, aa in pairs:
        assert_same(ab, aa)
    batch.remove(pairs[0][1])
    pairs[0][1].step(9)
    pairs[0][0].step(9)
    batch.step(2)
    for ab, _ in pairs[1:]:
        ab.step(2)
    for ab, aa in pairs:
        assert_same(ab, aa)
