"""FP64 diagnostics (mass, heat, steady residual, divergence) against the oracle's fields."""
import math
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


def expected(F_now, F_prev, r0=0.0):
    rho, ux, ur, T = F_now
    r = I.radii(rho.shape[0], r0)[:, None]
    out = {"mass": rho.sum(), "mass_axi": (r * rho).sum(), "heat": T.sum(), "heat_axi": (r * T).sum()}
    sp = np.hypot(ux, ur)
    out["max_speed"] = sp.max()
    if F_prev is not None:
        d = np.hypot(ux - F_prev[1], ur - F_prev[2])
        out["residual_max"] = d.max() / sp.max()
        out["residual_l2"] = math.sqrt((d ** 2).sum() / (sp ** 2).sum())
    return out


@pytest.mark.parametrize("size", [(97, 40), (300, 70), (5, 3)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_diagnostics_match_oracle_fields(lbm, orc, size):
    w = I.jet_workload(nx=size[0], nr=size[1], R=max(1.0, size[1] / 3.0), ntab=64)
    o = orc.Oracle.from_workload(w, NTHREADS)
    g = lbm.Lattice.from_workload(w, "f64")
    o.step(29)
    F_prev = o.fields()
    o.step(1)
    F_now = o.fields()
    g.step(30)
    d = g.diagnostics()
    want = expected(F_now, F_prev)
    assert d["nonfinite"] == 0 and not d["diverged"]
    for k, v in want.items():
        assert d[k] == pytest.approx(v, rel=1e-11, abs=1e-300), k


def test_residual_undefined_after_set_state(lbm, orc):
    w = I.jet_workload(nx=64, nr=20, ntab=64)
    g = lbm.Lattice.from_workload(w, "f32")
    f0, g0 = I.random_state(64, 20, orc.feq(1.0, 0.0, 0.0), orc.geq(1.0, 0.0, 0.0), 0.01, 1)
    g.set_state(f0, g0, 0)
    d = g.diagnostics()
    assert math.isnan(d["residual_max"]) and math.isnan(d["residual_l2"])
    g.step(1)
    assert not math.isnan(g.diagnostics()["residual_max"])


def test_divergence_is_reported(lbm, orc):
    w = I.jet_workload(nx=64, nr=20, ntab=64)
    g = lbm.Lattice.from_workload(w, "f32")
    f0, g0 = I.random_state(64, 20, orc.feq(1.0, 0.0, 0.0), orc.geq(1.0, 0.0, 0.0), 0.01, 1)
    f0[:, 6:9, 29:32] = -0.2  # a patch whose streamed density is negative at its centre
    g.set_state(f0, g0, 0)
    d = g.diagnostics()
    assert d["diverged"] and d["nonfinite"] >= 1


@pytest.mark.parametrize("storage,tol", [("f64", 1e-13), ("f32", 1e-6)])
def test_closed_domain_conserves_mass_on_gpu(lbm, orc, storage, tol):
    """Planar model, periodic ends, axis and wall: total mass stays put."""
    cfg = I.LatticeConfig(nx=96, nr=40, bc_in="periodic", bc_out="periodic", bc_top="wall", axisym=False,
                          Cs=0.17, T_top=1.0)
    g = lbm.Lattice(cfg, storage)
    nu, al = I.power_law_tables(32, 0.9, 1.2, nu_max=0.05)
    g.set_properties(nu, al, 0.9, 1.2)
    f0, g0 = I.random_state(96, 40, orc.feq(1.0, 0.0, 0.0), orc.geq(1.0, 0.0, 0.0), 0.05, 9)
    g.set_state(f0, g0, 0)
    m0 = g.diagnostics()["mass"]
    g.step(1000)
    m1 = g.diagnostics()["mass"]
    assert abs(m1 - m0) < tol * m0
