"""Batched stepping: every member of a ragged batch advances exactly as it would alone."""
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


def ragged_jets(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nx = int(rng.integers(1, 12)) * 37 + int(rng.integers(0, 3))
        nr = int(rng.integers(1, 8)) * 11 + int(rng.integers(0, 2))
        w = I.jet_workload(nx=nx, nr=nr, u_max=0.05 + 0.01 * k, T_ratio=2.0 + k, seed=seed * 31 + k,
                           ntab=64)
        if k % 3 == 1:
            w.cfg.bc_top = "wall"
        if k % 3 == 2:
            w.cfg.bc_out = "wall"
        out.append(w)
    return out


def states_equal(a, b):
    fa, ga = a.get_state()
    fb, gb = b.get_state()
    return torch.equal(fa, fb) and torch.equal(ga, gb)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16", "f16s", "bf16s"])
def test_batch_members_match_standalone(lbm, storage):
    ws = ragged_jets(5, 3)
    alone = [lbm.Lattice.from_workload(w, storage) for w in ws]
    mixed = [lbm.Lattice.from_workload(w, storage) for w in ws]
    b = lbm.Batch(storage)
    for m in mixed:
        b.add(m)
    for a in alone:
        a.step(23)
    b.step(23, graph=False)
    for a, m in zip(alone, mixed):
        assert m.step_count == a.step_count == 23
        assert states_equal(a, m)


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_batch_with_32_column_strips_matches_standalone(lbm, storage):
    """A batch stepped with 32-column tiles (one node per lane) advances every member exactly as
    the member alone at the default tile."""
    ws = ragged_jets(5, 9)
    alone = [lbm.Lattice.from_workload(w, storage) for w in ws]
    mixed = [lbm.Lattice.from_workload(w, storage) for w in ws]
    b = lbm.Batch(storage)
    b.set_strip_width(32)
    for m in mixed:
        b.add(m)
    for a in alone:
        a.step(23)
    b.step(23, graph=True)
    assert b.strip_width == 32
    for a, m in zip(alone, mixed):
        assert states_equal(a, m)


def test_graph_replay_matches_eager(lbm):
    ws = ragged_jets(4, 5)
    eager = [lbm.Lattice.from_workload(w, "f16") for w in ws]
    graphed = [lbm.Lattice.from_workload(w, "f16") for w in ws]
    be, bg = lbm.Batch("f16"), lbm.Batch("f16")
    for x in eager:
        be.add(x)
    for x in graphed:
        bg.add(x)
    be.step(37, graph=False)
    bg.step(37, graph=True)  # two 16-step graph replays and 5 single steps
    for x, y in zip(eager, graphed):
        assert states_equal(x, y)


def test_membership_changes_mid_run(lbm):
    ws = ragged_jets(4, 7)
    alone = [lbm.Lattice.from_workload(w, "f32") for w in ws]
    mixed = [lbm.Lattice.from_workload(w, "f32") for w in ws]
    b = lbm.Batch("f32")
    b.add(mixed[0])
    b.add(mixed[1])
    b.step(10)
    b.add(mixed[2])
    b.step(20)
    b.remove(mixed[0])
    b.add(mixed[3])
    mixed[3].set_inlet(ws[3].u_in * 0.5, ws[3].T_in)
    alone[3].set_inlet(ws[3].u_in * 0.5, ws[3].T_in)
    b.step(17)
    alone[0].step(30)
    alone[1].step(47)
    alone[2].step(37)
    alone[3].step(17)
    for a, m in zip(alone, mixed):
        assert a.step_count == m.step_count
        assert states_equal(a, m)


def test_member_cannot_step_alone(lbm):
    w = ragged_jets(1, 9)[0]
    lat = lbm.Lattice.from_workload(w, "f32")
    b = lbm.Batch("f32")
    b.add(lat)
    with pytest.raises(lbm.LbmError):
        lat.step(1)
    b.remove(lat)
    lat.step(1)
    other = lbm.Lattice.from_workload(w, "f16")
    with pytest.raises(lbm.LbmError):
        b.add(other)  # storage type differs


def test_batch_member_matches_oracle(lbm, orc):
    """An FP64 member of a batch against the oracle, per step from an identical state."""
    ws = ragged_jets(3, 11)
    lats = [lbm.Lattice.from_workload(w, "f64") for w in ws]
    b = lbm.Batch("f64")
    for x in lats:
        b.add(x)
    w = ws[1]
    o = orc.Oracle.from_workload(w, NTHREADS)
    f0, g0 = I.random_state(w.cfg.nx, w.cfg.nr, orc.feq(1.0, 0.02, 0.0), orc.geq(1.5, 0.0, 0.0), 0.03, 2)
    o.set_state(f0, g0, 4)
    lats[1].set_state(f0, g0, 4)
    for _ in range(3):
        o.step(1)
        b.step(1)
    fg, gg = lats[1].get_state()
    fo, go = o.get_state()
    for q in range(9):
        assert np.max(np.abs(fg[q].cpu().numpy() - fo[q])) <= 1e-12 * np.max(np.abs(fo[q]))
    for q in range(4):
        assert np.max(np.abs(gg[q].cpu().numpy() - go[q])) <= 1e-12 * np.max(np.abs(go[q]))


@pytest.mark.parametrize("storage,bar", [("f32", 2e-5), ("f16", 2e-3), ("f16s", 2e-3)])
def test_full_ensemble_batch_matches_oracle(lbm, orc, storage, bar):
    """The benchmark's ensemble (256 ragged jets, 23.2 M nodes) in its own launch
    configuration: two batched steps from random states on sampled members, against the
    oracle (per-step bars of the parity tests, times two steps)."""
    ws = I.ensemble_workloads(256, seed=7)
    lats = [lbm.Lattice.from_workload(w, storage) for w in ws]
    b = lbm.Batch(storage)
    for x in lats:
        b.add(x)
    picks = [0, 77, 154, 255]
    orcs = {}
    for k in picks:
        w = ws[k]
        f0, g0 = I.random_state(w.cfg.nx, w.cfg.nr, orc.feq(1.0, 0.02, 0.0), orc.geq(1.5, 0.0, 0.0), 0.03, 100 + k)
        o = orc.Oracle.from_workload(w, NTHREADS)
        o.set_state(f0, g0, 9)
        lats[k].set_state(f0, g0, 9)
        orcs[k] = o
    b.step(2, graph=False)
    for k, o in orcs.items():
        o.step(2)
        fg, gg = lats[k].get_state()
        fo, go = o.get_state()
        for q in range(9):
            assert np.max(np.abs(fg[q].cpu().numpy() - fo[q])) <= bar * np.max(np.abs(fo[q])), (k, q)
        for q in range(4):
            assert np.max(np.abs(gg[q].cpu().numpy() - go[q])) <= bar * np.max(np.abs(go[q])), (k, q)
    assert max(x.check() for x in lats) == 0
