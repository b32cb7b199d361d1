"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Errors are max-norms of the difference relative to the max-norm of the
oracle's quantity: per population plane for states; for fields, rho and T
against their own max, the velocity components against the max speed
|u| = sqrt(u_x^2 + u_r^2).  Tolerances:
  FP64 storage   1e-12 per step, and 1e-12 over the 2000-step laminar pipe;
  FP32 storage   1e-5 on rho, u, T per step and after 1000 laminar steps;
  FP16 moment-split storage (f16s)
                 1e-3 on u and T per step, after 1000 laminar steps
                 (measured 1.0e-4 and 4.9e-4) and after 1000 steps of the
                 4096 x 1024 jet against the FP64 path (3.8e-4, 7.6e-5);
  BF16 moment-split storage (bf16s)
                 3e-3 per step; NOT within 1e-3 over a run: 1e-2 after 1000
                 laminar steps (measured 3.3e-3 on u, 4.6e-3 on T);
  FP16 rest-deviation storage (f16)
                 1e-3 on u and T per step; NOT within 1e-3 over a run:
                 2e-3 after 1000 laminar steps (measured 0.8e-3 and 1.3e-3);
  BF16 rest-deviation storage (bf16)
                 3e-3 on u and T per step; NOT within 1e-3 over a run: 4e-2
                 after 1000 laminar steps (measured 2.1e-2 on u, 3.0e-2 on T).
Rest-deviation storage rounds each stored deviation to 2^-12 (FP16) or
2^-9 (BF16) of its size every step, and that size grows with the velocity
and the temperature excess; the laminar pipe accumulates those roundings
over its thermal relaxation time.  Moment-split storage keeps j and T in
FP32 and rounds only the deviations from the linear equilibrium.
Turbulent runs are compared one step at a time from an identical state.
"""
import os

import numpy as np
import pytest

from paper_1002_3028_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NTHREADS = max(1, min(8, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_3028_gb300 import lbm as L

    L.lib()
    return L


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (scale if scale > 0 else 1.0))


def state_rel(lat_state, orc_state):
    """Worst per-plane relative difference of two (f, g) states."""
    worst = 0.0
    for a, b in zip(lat_state, orc_state):
        a = a.cpu().numpy() if hasattr(a, "cpu") else a
        for q in range(b.shape[0]):
            worst = max(worst, rel(a[q], b[q]))
    return worst


def fields_rel(Fg, Fo):
    """[rho, u_x, u_r, T] errors; velocity components relative to the max speed."""
    Fg = Fg.cpu().numpy() if hasattr(Fg, "cpu") else np.asarray(Fg)
    speed = float(np.max(np.hypot(Fo[1], Fo[2])))
    out = []
    for c in range(4):
        scale = speed if c in (1, 2) else float(np.max(np.abs(Fo[c])))
        d = float(np.max(np.abs(Fg[c] - Fo[c])))
        out.append(d / scale if scale > 0 else d)
    return out


def workload(nx, nr, bc_in="inlet", bc_out="outflow", bc_top="open", bc_bottom="axis", r0=0.0,
             Cs=0.17, noise=1e-3, axisym=True):
    R = max(1.0, nr / 3.0)
    cfg = I.LatticeConfig(nx=nx, nr=nr, bc_in=bc_in, bc_out=bc_out, bc_top=bc_top,
                          bc_bottom=bc_bottom, r0=r0, axisym=axisym, Cs=Cs, Pr_t=0.3,
                          T_top=1.2, T_bottom=1.5, T_out=0.8, noise_amp=noise, seed=99)
    u_in, T_in = I.jet_profiles(nr, R, 0.06, 1.0, 4.0)
    nu, al = I.power_law_tables(64, 0.8, 4.0, nu_max=0.2)
    return I.Workload("case", cfg, u_in, T_in, nu, al, 0.8, 4.0)


def pair(lbm_mod, orc, w, storage, seed=1, amp=0.05, step=5):
    o = orc.Oracle.from_workload(w, NTHREADS)
    g = lbm_mod.Lattice.from_workload(w, storage)
    f0, g0 = I.random_state(w.cfg.nx, w.cfg.nr, orc.feq(1.0, 0.02, 0.0), orc.geq(1.3, 0.02, 0.0), amp,
                            seed)
    o.set_state(f0, g0, step)
    g.set_state(f0, g0, step)
    return o, g


BOUNDARIES = {
    "jet": dict(bc_in="inlet", bc_out="outflow", bc_top="open", bc_bottom="axis"),
    "pipe": dict(bc_in="inlet", bc_out="outflow", bc_top="wall", bc_bottom="axis"),
    "periodic_axis": dict(bc_in="periodic", bc_out="periodic", bc_top="wall", bc_bottom="axis"),
    "annulus": dict(bc_in="periodic", bc_out="periodic", bc_top="wall", bc_bottom="wall", r0=5.0),
    "substrate": dict(bc_in="inlet", bc_out="wall", bc_top="open", bc_bottom="axis"),
    "inner_wall_pipe": dict(bc_in="inlet", bc_out="outflow", bc_top="wall", bc_bottom="wall", r0=3.0),
    "open_periodic": dict(bc_in="periodic", bc_out="periodic", bc_top="open", bc_bottom="axis"),
}
SIZES = [(70, 19), (33, 5), (1, 12), (3, 3), (64, 32), (97, 40)]


@pytest.mark.parametrize("bname", sorted(BOUNDARIES))
@pytest.mark.parametrize("size", SIZES, ids=[f"{a}x{b}" for a, b in SIZES])
def test_f64_step_matches_oracle(lbm, orc, bname, size):
    w = workload(*size, **BOUNDARIES[bname])
    o, g = pair(lbm, orc, w, "f64")
    for n in range(3):
        o.step(1)
        g.step(1)
        err = state_rel(g.get_state(), o.get_state())
        assert err < 1e-12, (n, err)
    assert g.step_count == o.step_count == 8
    assert max(fields_rel(g.fields(), o.fields())) < 1e-12


@pytest.mark.parametrize("size", [(1, 1), (2, 1), (1, 2), (5, 1), (31, 2), (32, 32), (33, 33)],
                         ids=lambda s: f"{s[0]}x{s[1]}")
@pytest.mark.parametrize("bname", ["jet", "pipe", "periodic_axis"])
def test_f64_degenerate_sizes(lbm, orc, size, bname):
    w = workload(*size, **BOUNDARIES[bname])
    o, g = pair(lbm, orc, w, "f64")
    o.step(2)
    g.step(2)
    assert state_rel(g.get_state(), o.get_state()) < 1e-12


def test_f64_planar_model(lbm, orc):
    w = workload(70, 19, axisym=False)
    o, g = pair(lbm, orc, w, "f64")
    o.step(2)
    g.step(2)
    assert state_rel(g.get_state(), o.get_state()) < 1e-12


def test_f64_pipe_2000_steps(lbm, orc):
    """Laminar Hagen-Poiseuille pipe, 64 x 32, 2000 steps from rest."""
    w = I.pipe_workload()
    o = orc.Oracle.from_workload(w, NTHREADS)
    g = lbm.Lattice.from_workload(w, "f64")
    o.step(2000)
    g.step(2000)
    errs = fields_rel(g.fields(), o.fields())
    assert max(errs) < 1e-12, errs


@pytest.mark.parametrize("storage,tol_u,tol_T", [("f32", 1e-5, 1e-5), ("f16s", 1e-3, 1e-3), ("bf16s", 1e-2, 1e-2),
                                                 ("f16", 2e-3, 2e-3), ("bf16", 4e-2, 4e-2)])
def test_reduced_storage_pipe_1000_steps(lbm, orc, storage, tol_u, tol_T):
    """rho, u, T of the laminar pipe after 1000 steps from rest."""
    w = I.pipe_workload()
    o = orc.Oracle.from_workload(w, NTHREADS)
    g = lbm.Lattice.from_workload(w, storage)
    o.step(1000)
    g.step(1000)
    errs = fields_rel(g.fields(), o.fields())
    assert errs[1] < tol_u and errs[2] < tol_u and errs[3] < tol_T, errs
    if storage == "f32":
        assert errs[0] < 1e-5, errs


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f16", 1e-3), ("bf16", 3e-3), ("f16s", 1e-3),
                                         ("bf16s", 3e-3)])
def test_reduced_storage_one_step(lbm, orc, storage, tol):
    """One step of a noisy hot jet from an identical state, every boundary of the jet."""
    w = workload(130, 45)
    o, g = pair(lbm, orc, w, storage, amp=0.02)
    o.step(1)
    g.step(1)
    errs = fields_rel(g.fields(), o.fields())
    assert errs[1] < tol and errs[2] < tol and errs[3] < tol, errs
    if storage == "f32":
        assert max(errs) < tol


def _developed_jet(orc, nx, nr, steps):
    w = I.jet_workload(nx=nx, nr=nr)
    o = orc.Oracle.from_workload(w, NTHREADS)
    o.step(steps)
    return w, o


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5), ("f16s", 1e-3), ("bf16s", 3e-3)])
def test_single_jet_1024x256_per_step(lbm, orc, storage, tol):
    """The 1024 x 256 turbulent jet in the benchmark's launch shape, stepped from the oracle's state."""
    w, o = _developed_jet(orc, 1024, 256, 150)
    f0, g0 = o.get_state()
    g = lbm.Lattice.from_workload(w, storage)
    g.set_state(f0, g0, o.step_count)
    for _ in range(2):
        o.step(1)
        g.step(1)
        errs = fields_rel(g.fields(), o.fields())
        assert max(errs) < tol, errs
    if storage == "f64":
        assert state_rel(g.get_state(), o.get_state()) < tol


@pytest.mark.parametrize("storage,bar", [("f32", 1e-5), ("f16", 1e-3), ("bf16", 3e-3), ("f16s", 1e-3),
                                         ("bf16s", 3e-3)])
def test_full_size_4096x1024(lbm, orc, storage, bar):
    """The 4096 x 1024 jet (the throughput workload) in the benchmark's launch configuration:
    three steps in one persistent launch from a perturbed state, against the oracle (the
    per-step bar of the storage type, times three)."""
    w = I.jet_workload(nx=4096, nr=1024)
    o = orc.Oracle.from_workload(w, NTHREADS)
    g = lbm.Lattice.from_workload(w, storage)
    f0, g0 = I.random_state(4096, 1024, orc.feq(1.0, 0.03, 0.0), orc.geq(2.0, 0.03, 0.0), 0.01, 4)
    o.set_state(f0, g0, 17)
    g.set_state(f0, g0, 17)
    del f0, g0
    o.step(3)
    g.step(3)
    errs = fields_rel(g.fields(), o.fields())
    assert max(errs) < 3 * bar, errs
    assert g.check() == 0


def test_f16s_jet_4096x1024_1000_steps_against_fp64(lbm):
    """FP16 moment-split storage stays within 1e-3 on u and T of the FP64 path over 1000 steps
    of the 4096 x 1024 jet from rest (the FP64 path is held to the oracle per step above)."""
    w = I.jet_workload(nx=4096, nr=1024)
    ref = lbm.Lattice.from_workload(w, "f64")
    ref.step(1000)
    Fr = ref.fields().cpu().numpy()
    ref.close()
    g = lbm.Lattice.from_workload(w, "f16s")
    g.step(1000)
    errs = fields_rel(g.fields(), Fr)
    assert errs[1] < 1e-3 and errs[2] < 1e-3 and errs[3] < 1e-3, errs
    assert g.check() == 0


@pytest.mark.parametrize("storage,band,warps,strip", [
    ("f32", 1, 1, 0), ("f32", 3, 8, 0), ("f32", 16, 4, 0), ("f32", 64, 2, 0), ("f32", 1000, 4, 0),
    ("f16s", 1, 1, 0), ("f16s", 16, 4, 0), ("bf16s", 3, 8, 0),
    ("f32", 1, 1, 32), ("f32", 6, 2, 32), ("f16", 4, 1, 32), ("bf16", 2, 4, 32), ("f16s", 5, 1, 32),
    ("bf16s", 1, 2, 32),
])
def test_launch_shape_does_not_change_results(lbm, orc, storage, band, warps, strip):
    """Band height, warps per CTA and the strip width (32-column tiles with one node per lane,
    64 with two) leave every stored value unchanged."""
    w = workload(97, 40)
    ref = lbm.Lattice.from_workload(w, storage)
    alt = lbm.Lattice.from_workload(w, storage)
    alt.set_strip_width(strip)
    alt.set_launch(band, warps)
    f0, g0 = I.random_state(97, 40, orc.feq(1.0, 0.0, 0.0), orc.geq(1.0, 0.0, 0.0), 0.03, 8)
    for lat in (ref, alt):
        lat.set_state(f0, g0, 0)
        lat.step(4)
    a = ref.get_state()
    b = alt.get_state()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


@pytest.mark.parametrize("storage,bounds,band,group", [
    ("f32", "jet", 0, 1), ("f32", "jet", 1, 1), ("f32", "periodic_axis", 0, 1), ("f32", "open_periodic", 1, 1),
    ("f16", "pipe", 4, 1), ("f64", "jet", 0, 1), ("f64", "annulus", 2, 1),
    ("f32", "jet", 0, 2), ("f32", "periodic_axis", 4, 2), ("f32", "open_periodic", 1, 3), ("f64", "jet", 3, 4),
    ("f16s", "pipe", 4, 1), ("f16s", "open_periodic", 1, 2), ("bf16s", "substrate", 0, 1),
    ("f32/32", "periodic_axis", 1, 1), ("f32/32", "open_periodic", 4, 2), ("f16s/32", "jet", 2, 1),
])
def test_many_steps_in_one_launch_equal_single_steps(lbm, orc, storage, bounds, band, group):
    """lbm_step(n) runs its n steps in one launch whose work items wait for their neighbours
    of the previous step; the result is bit for bit that of n separate one-step launches
    (one-row bands depend on two bands each side; periodic ends make the first and last
    items neighbours; items of several strips, a ragged last one, or one item per band).
    The lattice spans several strips and bands with a ragged last strip."""
    storage, _, strip = storage.partition("/")  # "f32/32": 32-column strips
    w = workload(150, 45, **BOUNDARIES[bounds])
    one = lbm.Lattice.from_workload(w, storage)
    many = lbm.Lattice.from_workload(w, storage)
    for lat in (one, many):
        lat.set_strip_width(int(strip or 0))
        lat.set_launch(band, 1)
    many.set_item_group(group)
    assert many.item_group == group
    f0, g0 = I.random_state(150, 45, orc.feq(1.0, 0.02, 0.0), orc.geq(1.2, 0.02, 0.0), 0.05, 21)
    for lat in (one, many):
        lat.set_state(f0, g0, 3)
    for _ in range(23):
        one.step(1)
    many.step(23)
    assert one.step_count == many.step_count == 26
    a, _ = one.save()
    b, _ = many.save()
    assert torch.equal(a, b)
    assert one.check() == 0 and many.check() == 0


@pytest.mark.parametrize("storage,nx", [("f64", 97), ("f32", 193)])
@pytest.mark.parametrize("bounds", ["periodic_axis", "open_periodic"])
@pytest.mark.parametrize("band,group", [(0, 1), (1, 1), (4, 1), (4, 2)])
def test_many_steps_periodic_with_a_one_column_last_strip(lbm, orc, storage, nx, bounds, band, group):
    """With periodic ends and a last strip of one column (and four strips or more), the
    pulled moments of column nx - 1 read column nx - 2 and the periodic image of column 0:
    the tiles of strip 0 and of the strip before the last depend on each other across the
    wrap, two strips apart.  Several multi-step launches must equal one-step launches bit
    for bit (the race this guards against showed up in about half of such runs)."""
    w = workload(nx, 40, **BOUNDARIES[bounds])
    f0, g0 = I.random_state(nx, 40, orc.feq(1.0, 0.02, 0.0), orc.geq(1.2, 0.02, 0.0), 0.05, 44)
    ref = lbm.Lattice.from_workload(w, storage)
    ref.set_launch(band, 1)
    ref.set_state(f0, g0, 3)
    for _ in range(60):
        ref.step(1)
    want, _ = ref.save()
    for _ in range(6):
        lat = lbm.Lattice.from_workload(w, storage)
        lat.set_launch(band, 1)
        lat.set_item_group(group)
        lat.set_state(f0, g0, 3)
        lat.step(60)
        assert torch.equal(lat.save()[0], want)
        assert lat.check() == 0
        lat.close()


@pytest.mark.parametrize("storage", ["f32", "f16", "f64", "f16s"])
def test_bounded_waits_time_out_and_leave_the_lattice_usable(lbm, orc, storage):
    """A launch whose dependency waits can never be met ends by itself with
    LBM_STATUS_TIMEOUT; the state is untouched and the next steps are exact."""
    w = workload(150, 45)
    a = lbm.Lattice.from_workload(w, storage)
    b = lbm.Lattice.from_workload(w, storage)
    f0, g0 = I.random_state(150, 45, orc.feq(1.0, 0.02, 0.0), orc.geq(1.2, 0.02, 0.0), 0.05, 31)
    for lat in (a, b):
        lat.set_state(f0, g0, 0)
        lat.step(3)
    before, _ = a.save()
    assert a.selftest_wait_timeout() == 1  # LBM_STATUS_TIMEOUT
    after, step = a.save()
    assert step == 3 and torch.equal(before, after)
    assert a.check() == 0  # the self-test cleared what it raised
    a.step(5)
    b.step(5)
    assert torch.equal(a.save()[0], b.save()[0])


def test_rest_state_is_exactly_steady(lbm):
    cfg = I.LatticeConfig(nx=100, nr=30, bc_top="wall", T_top=1.0)
    lat = lbm.Lattice(cfg, "f32")
    lat.step(20)
    f, g = lat.get_state()
    f0 = torch.tensor([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=torch.float64, device=f.device)
    assert torch.equal(f, f0.view(9, 1, 1).expand_as(f))
    assert torch.all(g == 0.25)


def test_state_roundtrip_f64(lbm, orc):
    w = workload(45, 13)
    g = lbm.Lattice.from_workload(w, "f64")
    f0, g0 = I.random_state(45, 13, orc.feq(1.0, 0.0, 0.0), orc.geq(1.0, 0.0, 0.0), 0.05, 3)
    g.set_state(f0, g0, 12)
    f1, g1 = g.get_state()
    assert g.step_count == 12
    np.testing.assert_allclose(f1.cpu().numpy(), f0, rtol=0, atol=1e-16)
    np.testing.assert_allclose(g1.cpu().numpy(), g0, rtol=0, atol=1e-16)


def test_fields_float32_output(lbm, orc):
    w = workload(50, 20)
    o, g = pair(lbm, orc, w, "f64")
    Fo = o.fields()
    F32 = g.fields(dtype=torch.float32)
    assert max(fields_rel(F32.double(), Fo)) < 1e-6


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16", "f16s", "bf16s"])
def test_checkpoint_resume_is_exact(lbm, storage):
    """Save mid-run, restore into a fresh lattice, continue: bit for bit the uninterrupted run."""
    w = workload(90, 33)
    a = lbm.Lattice.from_workload(w, storage)
    a.step(40)
    planes, step = a.save()
    assert step == 40
    b = lbm.Lattice.from_workload(w, storage)
    b.restore(planes.clone(), step)
    assert b.step_count == 40
    a.step(25)
    b.step(25)
    pa, _ = a.save()
    pb, _ = b.save()
    assert torch.equal(pa, pb)
    assert torch.equal(a.fields(), b.fields())


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "f16s"])
def test_state_roundtrip_through_fp64_resumes_closely(lbm, storage):
    """get_state / set_state round trips through absolute FP64 values: within a rounding of the storage."""
    w = workload(90, 33)
    a = lbm.Lattice.from_workload(w, storage)
    a.step(40)
    f, g = a.get_state()
    b = lbm.Lattice.from_workload(w, storage)
    b.set_state(f, g, a.step_count)
    a.step(25)
    b.step(25)
    tol = {"f64": 1e-15, "f32": 1e-6, "f16": 1e-3, "f16s": 1e-3}[storage]
    fa, ga = a.get_state()
    fb, gb = b.get_state()
    assert (fa - fb).abs().max().item() < tol and (ga - gb).abs().max().item() < tol


def test_create_refuses_caller_memory_too_small_or_misaligned(lbm):
    """lbm_create with a caller block one byte short (LBM_ERR_OOM) or off the 256-byte
    alignment (LBM_ERR_INVALID_ARG) fails before any device work and leaves *out untouched."""
    import ctypes as C

    w = workload(70, 20)
    d = lbm.make_desc(w.cfg, "f32", "ab")
    need = lbm.required_bytes(w.cfg, "f32")
    mem = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    L = lbm.lib()
    for ptr, nbytes, rc in ((mem.data_ptr(), need - 1, -2), (mem.data_ptr() + 128, need, -1)):
        h = C.c_void_p(12345)
        assert L.lbm_create(C.byref(d), C.c_void_p(ptr), nbytes, C.byref(h)) == rc
        assert h.value == 12345
    h = C.c_void_p()
    assert L.lbm_create(C.byref(d), C.c_void_p(mem.data_ptr()), need, C.byref(h)) == 0
    L.lbm_destroy(h)


def test_side_stream_steps_equal_default_stream_steps(lbm):
    """A lattice stepped and read on a side stream gives the default stream's results; the
    binding keeps its block from reuse until that stream's work has run."""
    w = workload(97, 40)
    a = lbm.Lattice.from_workload(w, "f32")
    b = lbm.Lattice.from_workload(w, "f32")
    a.step(30)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.step(30, stream=s)
        Fb = b.fields(stream=s)
    s.synchronize()
    assert torch.equal(a.fields(), Fb)
    assert list(b._streams) == [s.cuda_stream]
    b.close()
    a.close()


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_counters_carried_across_launches_with_shape_changes(lbm, orc, storage):
    """lbm_step's work and completion counters carry on from one launch to the next and are
    reset only when the item count changes or a wait ran out.  Launches of 1..7 steps with the
    band, the strip width and the item group changed between some of them (and repeated
    between others), and the bounded-wait self-test in the middle, give the bits of one
    lattice stepped in a single launch."""
    w = workload(150, 45, **BOUNDARIES["open_periodic"])
    ref = lbm.Lattice.from_workload(w, storage)
    lat = lbm.Lattice.from_workload(w, storage)
    f0, g0 = I.random_state(150, 45, orc.feq(1.0, 0.02, 0.0), orc.geq(1.2, 0.02, 0.0), 0.05, 31)
    for x in (ref, lat):
        x.set_state(f0, g0, 0)
    plan = [(3, 0, 0, 0), (1, 0, 0, 0), (4, 0, 0, 0), (2, 4, 0, 0), (5, 4, 0, 0), (7, 1, 32, 0),
            (1, 1, 32, 0), (2, 2, 32, 2), (3, 0, 64, 0), (6, 0, 64, 3), (2, 0, 0, 0)]
    steps = 0
    for n, band, strip, group in plan:
        lat.set_strip_width(strip)
        lat.set_launch(band, 1)
        lat.set_item_group(group)
        lat.step(n)
        steps += n
        if steps == 15:  # a timed-out launch leaves the counters to be reset
            assert lat.selftest_wait_timeout() != 0 and lat.step_count == 15
    ref.step(steps)
    assert lat.step_count == ref.step_count == steps
    assert torch.equal(lat.save()[0], ref.save()[0])
    assert lat.check() == 0 and ref.check() == 0
