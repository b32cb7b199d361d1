"""Randomised check of the persistent multi-step schedules (GPU).

A launch of n steps runs its work items with waits on neighbour items
instead of kernel boundaries.  Any dependency the waits miss shows up as a
difference from n one-step launches, which order everything.  Seeded random
lattices are compared bit for bit, in both memory patterns:
- random sizes, biased towards strips of one or a few columns and towards
  one-row or one-band lattices;
- every boundary set, and the four storage types;
- random bands, warps per CTA and item groups.
One lattice is also wide enough that the AA schedule must widen its items
to keep one band of items resident.  Batches of random members, in both
patterns, go through a graph replay and a remainder launch, and each member
must equal its own one-step launches.
"""
import random

import pytest

from paper_1002_3028_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUNDARIES = [
    dict(bc_in="inlet", bc_out="outflow", bc_top="open", bc_bottom="axis"),
    dict(bc_in="inlet", bc_out="outflow", bc_top="wall", bc_bottom="axis"),
    dict(bc_in="periodic", bc_out="periodic", bc_top="wall", bc_bottom="axis"),
    dict(bc_in="periodic", bc_out="periodic", bc_top="wall", bc_bottom="wall", r0=5.0),
    dict(bc_in="inlet", bc_out="wall", bc_top="open", bc_bottom="axis"),
    dict(bc_in="inlet", bc_out="outflow", bc_top="wall", bc_bottom="wall", r0=3.0),
    dict(bc_in="periodic", bc_out="periodic", bc_top="open", bc_bottom="axis"),
]


@pytest.fixture(scope="module")
def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_3028_gb300 import lbm as L

    L.lib()
    return L


def case(seed):
    rng = random.Random(seed)
    storage = rng.choice(["f64", "f32", "f32", "f16", "bf16"])
    strip = 32 if storage == "f64" else 64
    nx = rng.choice([rng.randint(1, 400), strip * rng.randint(1, 6) + 1, strip * rng.randint(1, 6) + rng.randint(2, 5),
                     strip * rng.randint(1, 6)])
    nr = rng.choice([rng.randint(1, 100), rng.randint(1, 8), rng.randint(30, 90)])
    bounds = dict(rng.choice(BOUNDARIES))
    band = rng.choice([0, 0, 1, 2, 3, 4, 5, 6, 8, 12, 1000])
    warps = rng.choice([1, 1, 2, 4])
    group = rng.choice([0, 0, 1, 2, 3])
    return storage, nx, nr, bounds, band, warps, group


def workload(nx, nr, bounds):
    R = max(1.0, nr / 3.0)
    cfg = I.LatticeConfig(nx=nx, nr=nr, Cs=0.17, Pr_t=0.3, T_top=1.2, T_bottom=1.5, T_out=0.8, noise_amp=1e-3,
                          seed=5, **bounds)
    u_in, T_in = I.jet_profiles(nr, R, 0.06, 1.0, 4.0)
    nu, al = I.power_law_tables(64, 0.8, 4.0, nu_max=0.2)
    return I.Workload("fuzz", cfg, u_in, T_in, nu, al, 0.8, 4.0)


def run(lbm, orc, w, storage, pattern, band, warps, group, chunks, seed):
    lat = lbm.Lattice.from_workload(w, storage, pattern=pattern)
    lat.set_launch(band, warps)
    lat.set_item_group(group)
    f0, g0 = I.random_state(w.cfg.nx, w.cfg.nr, orc.feq(1.0, 0.02, 0.0), orc.geq(1.2, 0.02, 0.0), 0.05, seed)
    lat.set_state(f0, g0, 2)
    for n in chunks:
        lat.step(n)
    assert lat.check() == 0
    out = lat.save()[0]
    lat.close()
    return out


@pytest.mark.parametrize("seed", range(48))
def test_multi_step_launches_equal_one_step_launches(lbm, orc, seed):
    storage, nx, nr, bounds, band, warps, group = case(seed)
    w = workload(nx, nr, bounds)
    want = run(lbm, orc, w, storage, "ab", band, warps, group, [1] * 40, seed)
    for pattern in ("ab", "aa"):
        got = run(lbm, orc, w, storage, pattern, band, warps, group, [40], seed)
        assert torch.equal(got, want), (pattern, storage, nx, nr, bounds, band, warps, group)


def test_aa_widens_items_on_a_lattice_wider_than_the_resident_warps(lbm, orc):
    """160 000 columns make 2500 strips of 64: more than the GPU holds warps, so the AA
    schedule takes two strips per item to keep one band of items resident."""
    w = workload(160000, 8, BOUNDARIES[0])
    want = run(lbm, orc, w, "f32", "ab", 0, 0, 0, [1] * 6, 3)
    got = run(lbm, orc, w, "f32", "aa", 0, 0, 0, [6], 3)
    assert torch.equal(got, want)


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_batch_members_equal_one_step_launches_alone(lbm, orc, seed, pattern):
    """A batch of 3-9 random members (one storage type) stepped through a graph replay of
    64 steps and a remainder launch: every member equals its own one-step launches."""
    rng = random.Random(1000 + seed)
    storage = rng.choice(["f64", "f32", "f16"])
    strip = 32 if storage == "f64" else 64
    batch = lbm.Batch(storage)
    members = []
    for m in range(rng.randint(3, 9)):
        nx = rng.choice([rng.randint(1, 300), strip * rng.randint(1, 5) + 1])
        nr = rng.choice([rng.randint(1, 80), rng.randint(1, 6)])
        w = workload(nx, nr, dict(rng.choice(BOUNDARIES)))
        want = run(lbm, orc, w, storage, "ab", 0, 0, 0, [1] * 70, 77 + m)
        lat = lbm.Lattice.from_workload(w, storage, pattern=pattern)
        f0, g0 = I.random_state(nx, nr, orc.feq(1.0, 0.02, 0.0), orc.geq(1.2, 0.02, 0.0), 0.05, 77 + m)
        lat.set_state(f0, g0, 2)
        batch.add(lat)
        members.append((lat, want))
    batch.step(70, graph=True)
    for lat, want in members:
        assert lat.check() == 0
        assert torch.equal(lat.save()[0], want), (pattern, storage, lat.nx, lat.nr)
