"""Whole-jet checks of the paper's qualitative results on the GPU path (FP32 storage, and FP16
moment-split storage for the free jet).

Section 4 of the paper reports that the radial temperature distribution of
the jet is Gaussian at successive cross-sections (Fig. 6), with the jet
widening and its centreline temperature falling downstream.  These tests
develop the synthetic 1024 x 256 jet (nozzle radius 32, flat-top T profile
at the inlet) and check that shape at three stations, for the free jet and
for the substrate variant (outlet wall).
"""
import dataclasses

import numpy as np
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


def gaussian_fit(r, y):
    """Fit y = A exp(-r^2 / (2 s^2)) by least squares on ln y over the core (y > A / 10);
    return A, s and the coefficient of determination of the fit over r < 2.5 s."""
    core = y > 0.1 * y.max()
    slope, intercept = np.polyfit(r[core] ** 2, np.log(y[core]), 1)
    A, s = float(np.exp(intercept)), float(np.sqrt(-1.0 / (2.0 * slope)))
    m = r < 2.5 * s
    resid = y[m] - A * np.exp(-r[m] ** 2 / (2 * s * s))
    r2 = 1.0 - float((resid ** 2).sum() / ((y[m] - y[m].mean()) ** 2).sum())
    return A, s, r2


@pytest.mark.parametrize("bc_out,storage", [("outflow", "f32"), ("wall", "f32"), ("outflow", "f16s")])
def test_developed_jet_has_gaussian_radial_temperature(lbm, bc_out, storage):
    w = I.jet_workload(nx=1024, nr=256)
    w = dataclasses.replace(w, cfg=dataclasses.replace(w.cfg, bc_out=bc_out))
    lat = lbm.Lattice.from_workload(w, storage)
    lat.step(30000)
    assert lat.check() == 0
    F = lat.fields().cpu().numpy()
    assert np.isfinite(F).all()
    r = I.radii(256)
    fits = [gaussian_fit(r, F[3][:, i] - w.cfg.T0) for i in (64, 128, 256)]
    for A, s, r2 in fits:
        assert r2 > 0.95
    A, s = [f[0] for f in fits], [f[1] for f in fits]
    assert A[0] > A[1] > A[2] > 0  # the centreline temperature falls downstream
    assert s[0] < s[1] < s[2]  # and the jet widens
