"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than its own formulas:
published generator outputs, moment identities of the lattice, a direct
numerical solve of Eq. 3, closed-form flows of the axisymmetric equations
(Bessel-mode decay, radial conduction in an annulus, Hagen-Poiseuille
pressure drop), symmetry and conservation invariants, and hand-worked
boundary cases on tiny lattices.
"""
import math
import os

import numpy as np
import pytest

from paper_1002_3028_gb300 import inputs as I

J0_ZERO = 2.404825557695773  # first zero of the Bessel function J0

E9 = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
E4 = [(1, 0), (0, 1), (-1, 0), (0, -1)]


def _golden(name):
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    with open(path) as fh:
        return [ln.strip() for ln in fh if ln.strip() and not ln.startswith("#")]


# ---- inlet noise generator -------------------------------------------------

def test_splitmix64_published_outputs(orc):
    """SplitMix64 from state 0 (Steele, Lea, Flood 2014) gives the published sequence."""
    want = [int(v, 16) for v in _golden("splitmix64_seed0.txt")]
    gamma = 0x9E3779B97F4A7C15
    got = [orc.splitmix64((n * gamma) & 0xFFFFFFFFFFFFFFFF) for n in range(3)]
    assert got == want


def test_inlet_noise_uniform_in_range(orc):
    amp = 1e-3
    xs = np.array([orc.inlet_noise(1234, t, j, amp) for t in range(40) for j in range(100)])
    assert np.all(np.abs(xs) <= amp)
    assert abs(xs.mean()) < 0.05 * amp  # 4000 samples: sd of mean = amp / sqrt(3 * 4000)
    assert abs(xs.std() - amp / math.sqrt(3.0)) < 0.05 * amp
    assert orc.inlet_noise(1234, 7, 3, amp) == orc.inlet_noise(1234, 7, 3, amp)
    assert orc.inlet_noise(1234, 7, 3, amp) != orc.inlet_noise(1235, 7, 3, amp)


# ---- equilibria and moments (Eq. 2) -----------------------------------------

@pytest.mark.parametrize("rho,ux,ur", [(1.0, 0.0, 0.0), (1.07, 0.08, -0.03), (0.93, -0.05, 0.1)])
def test_feq_moments(orc, rho, ux, ur):
    """The D2Q9 equilibrium has moments rho, rho u and rho (delta/3 + u u)."""
    f = orc.feq(rho, ux, ur)
    e = np.array(E9, dtype=float)
    assert abs(f.sum() - rho) < 1e-15
    np.testing.assert_allclose(e.T @ f, [rho * ux, rho * ur], atol=1e-16)
    P = np.einsum("ka,kb,k->ab", e, e, f)
    want = rho * (np.eye(2) / 3.0 + np.outer([ux, ur], [ux, ur]))
    np.testing.assert_allclose(P, want, atol=1e-15)
    m = orc.moments(f, np.zeros(4))
    np.testing.assert_allclose(m[:3], [rho, rho * ux, rho * ur], atol=1e-15)


@pytest.mark.parametrize("T,ux,ur", [(1.0, 0.0, 0.0), (7.5, 0.06, 0.02)])
def test_geq_moments(orc, T, ux, ur):
    """The D2Q4 equilibrium has zeroth moment T and first moment T u."""
    g = orc.geq(T, ux, ur)
    e = np.array(E4, dtype=float)
    assert abs(g.sum() - T) < 1e-14
    np.testing.assert_allclose(e.T @ g, [T * ux, T * ur], atol=1e-15)
    assert orc.moments(np.zeros(9), g)[3] == pytest.approx(T, abs=1e-14)


def test_single_direction_moments(orc):
    """A lone population of direction k has rho = 1 and momentum e_k; all nine velocities occur."""
    seen = set()
    for k in range(9):
        f = np.zeros(9)
        f[k] = 1.0
        m = orc.moments(f, np.zeros(4))
        assert m[0] == 1.0
        seen.add((int(m[1]), int(m[2])))
    assert seen == {(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)}


# ---- Smagorinsky relaxation time (Eqs. 3-4) ----------------------------------

def _tau_by_bisection(tau_nu, Cs, f):
    """Solve Eq. 3, nu + Cs^2 |S(tau)| = (tau - 1/2)/3, for tau by bisection.

    The strain rate follows from the non-equilibrium stress of the populations
    relaxing with tau: S_ij = -3 Q_ij / (2 rho tau), |S| = sqrt(2 S_ij S_ij).
    Q is taken as the second moment minus its equilibrium value
    rho (delta/3 + u u), without the oracle's equilibrium function.
    """
    e = np.array(E9, dtype=float)
    rho = f.sum()
    u = e.T @ f / rho
    P = np.einsum("ka,kb,k->ab", e, e, f)
    Q = P - rho * (np.eye(2) / 3.0 + np.outer(u, u))
    Qn = math.sqrt(2.0 * float(np.sum(Q * Q)))
    nu = (tau_nu - 0.5) / 3.0

    def resid(tau):
        return nu + Cs * Cs * 3.0 * Qn / (2.0 * rho * tau) - (tau - 0.5) / 3.0

    lo, hi = tau_nu * 0.999, tau_nu + 10.0
    assert resid(lo) > 0 > resid(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if resid(mid) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("seed", range(6))
def test_tau_total_solves_eq3(orc, seed):
    rng = np.random.default_rng(seed)
    f = orc.feq(1.0 + 0.05 * rng.standard_normal(), 0.05 * rng.standard_normal(),
                0.05 * rng.standard_normal())
    f = f * (1.0 + 0.05 * rng.standard_normal(9))
    tau_nu = 0.505 + rng.random()
    Cs = 0.1 + 0.2 * rng.random()
    got = orc.tau_total(tau_nu, Cs, f)
    want = _tau_by_bisection(tau_nu, Cs, f)
    assert abs(got - want) < 1e-13 * want
    assert got > tau_nu


def test_tau_total_no_model_is_exact(orc):
    """Cs = 0 leaves the molecular relaxation time unchanged, bit for bit."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        f = orc.feq(1.0, 0.03, -0.02) * (1.0 + 0.1 * rng.standard_normal(9))
        tau = 0.5 + 1e-3 + rng.random()
        assert orc.tau_total(tau, 0.0, f) == tau


def test_tau_total_at_equilibrium(orc):
    f = orc.feq(1.02, 0.07, 0.01)
    assert orc.tau_total(0.6, 0.17, f) == pytest.approx(0.6, abs=1e-12)


# ---- property tables (Section 2.3) -------------------------------------------

def test_property_interpolation(orc):
    T_lo, T_hi, n = 1.0, 10.0, 7
    Tg = np.linspace(T_lo, T_hi, n)
    tab = 0.3 * Tg + 0.01  # linear in T: interpolation is exact
    for T in [1.0, 1.3, 4.0, 5.5, 9.99, 10.0]:
        assert orc.prop(tab, T_lo, T_hi, T) == pytest.approx(0.3 * T + 0.01, abs=1e-14)
    # clamped outside the range
    assert orc.prop(tab, T_lo, T_hi, 0.2) == pytest.approx(tab[0], abs=1e-15)
    assert orc.prop(tab, T_lo, T_hi, 50.0) == pytest.approx(tab[-1], abs=1e-15)
    # nodes are hit exactly; a one-entry table is a constant
    tab2 = np.array([0.1, 0.4, 0.2, 0.9, 0.3, 0.5, 0.7])
    for m in range(n):
        assert orc.prop(tab2, T_lo, T_hi, Tg[m]) == pytest.approx(tab2[m], abs=1e-15)
    assert orc.prop(np.array([0.25]), 0.0, 1.0, 123.0) == 0.25


# ---- collision and source terms (Eq. 1) --------------------------------------

def test_source_moments(orc):
    """At equilibrium the collision adds exactly F1 to mass, F2 to momentum and S to T."""
    rho, ux, ur, T = 1.03, 0.04, -0.02, 3.0
    fs = orc.feq(rho, ux, ur)
    gs = orc.geq(T, ux, ur)
    d = np.array([1e-3, -2e-3, 5e-4, 0.05])
    fo, go, diag = orc.collide_node(fs, gs, 4.5, d, 0.05, 0.07, 0.17, 0.3, True)
    e9 = np.array(E9, dtype=float)
    df = fo - fs
    assert abs(df.sum() - diag[2]) < 1e-15
    np.testing.assert_allclose(e9.T @ df, diag[3:5], atol=1e-15)
    assert abs((go - gs).sum() - diag[5]) < 1e-15
    # mass source of the axisymmetric continuity equation
    assert diag[2] == pytest.approx(-rho * ur / 4.5, rel=1e-14)


def test_sources_vanish_without_radial_flow_and_gradients(orc):
    fs = orc.feq(1.0, 0.05, 0.0)
    gs = orc.geq(2.0, 0.05, 0.0)
    fo, go, diag = orc.collide_node(fs, gs, 3.5, np.zeros(4), 0.05, 0.05, 0.17, 0.3, True)
    assert np.all(diag[2:] == 0.0)
    np.testing.assert_allclose(fo, fs, atol=1e-16)
    np.testing.assert_allclose(go, gs, atol=1e-16)


def test_planar_switch_turns_sources_off(orc):
    rng = np.random.default_rng(0)
    fs = orc.feq(1.0, 0.05, 0.03) * (1 + 0.01 * rng.standard_normal(9))
    gs = orc.geq(2.0, 0.05, 0.03)
    fo, go, diag = orc.collide_node(fs, gs, 2.5, rng.standard_normal(4), 0.05, 0.05, 0.17, 0.3, False)
    assert np.all(diag[2:] == 0.0)
    assert abs(fo.sum() - fs.sum()) < 1e-15  # BGK conserves mass
    assert abs(go.sum() - gs.sum()) < 1e-14  # and temperature


def test_collision_relaxes_by_one_over_tau(orc):
    """Without sources, f_post - f_eq = (1 - 1/tau)(f - f_eq) for every direction."""
    rng = np.random.default_rng(1)
    f = orc.feq(1.0, 0.02, 0.01) * (1 + 0.02 * rng.standard_normal(9))
    g = orc.geq(1.5, 0.02, 0.01) * (1 + 0.02 * rng.standard_normal(4))
    m = orc.moments(f, g)
    feq = orc.feq(m[0], m[1] / m[0], m[2] / m[0])
    geq = orc.geq(m[3], m[1] / m[0], m[2] / m[0])
    nu, alpha = 0.1, 0.2
    fo, go, diag = orc.collide_node(f, g, 2.5, np.zeros(4), nu, alpha, 0.0, 0.3, False)
    tau = 0.5 + 3 * nu
    tau_a = 0.5 + 2 * alpha
    assert diag[0] == tau and diag[1] == pytest.approx(tau_a, abs=1e-15)
    np.testing.assert_allclose(fo - feq, (1 - 1 / tau) * (f - feq), atol=1e-16)
    np.testing.assert_allclose(go - geq, (1 - 1 / tau_a) * (g - geq), atol=1e-16)


def test_turbulent_prandtl_coupling(orc):
    """Eq. 5: the thermal relaxation time grows by 2 nu_t / Pr_t."""
    rng = np.random.default_rng(2)
    f = orc.feq(1.0, 0.05, 0.0) * (1 + 0.05 * rng.standard_normal(9))
    g = orc.geq(1.0, 0.05, 0.0)
    nu, alpha = 0.02, 0.03
    _, _, diag = orc.collide_node(f, g, 2.5, np.zeros(4), nu, alpha, 0.17, 0.3, False)
    tau_nu = 0.5 + 3 * nu
    nu_t = (diag[0] - tau_nu) / 3
    assert nu_t > 0
    assert diag[1] == pytest.approx(0.5 + 2 * (alpha + nu_t / 0.3), rel=1e-14)


# ---- lattice derivatives feeding Eq. 1 ----------------------------------------

def _polynomial_state(orc, nx, nr, case):
    """Equilibrium populations whose streamed moments are polynomials of degree <= 2 in x and in r.

    Case "radial": rho = 1, u_x = U, u_r = a r (1 + b x), T = T0 + c x.
    Case "thermal": rho = 1 + e r^2, u_x = U (1 + b x), u_r = 0, T = T0 + c r^2.
    Both extend across the axis as mirror images (rho, u_x, T even in r, u_r
    odd), so the axis rows are polynomial too.
    """
    f = np.empty((9, nr, nx))
    g = np.empty((4, nr, nx))
    for j, r in enumerate(I.radii(nr)):
        for i in range(nx):
            if case == "radial":
                rho, ux, ur, T = 1.0, 0.04, 2e-3 * r * (1 + 0.05 * i), 1.0 + 0.02 * i
            else:
                rho, ux, ur, T = 1.0 + 4e-4 * r * r, 0.03 * (1 + 0.05 * i), 0.0, 1.0 + 2e-3 * r * r
            f[:, j, i] = orc.feq(rho, ux, ur)
            g[:, j, i] = orc.geq(T, ux, ur)
    return f, g


@pytest.mark.parametrize("case", ["radial", "thermal"])
def test_lattice_derivatives_are_exact_on_quadratics(orc, case):
    """The gradients entering F2 and S are exact derivatives of the streamed moments.

    A central difference is exact on a quadratic, so with streamed moments
    that are polynomials of degree <= 2 the collision of every node away from
    the wall and the periodic seam must equal the node collision given the
    analytic derivatives (taken from a least-squares polynomial fit of the
    streamed moments).  This pins the stencil, its 1/2, and the parities of
    the moments at the axis.
    """
    nx, nr, nu, alpha, Cs = 12, 10, 0.1, 0.12, 0.17
    cfg = I.LatticeConfig(nx=nx, nr=nr, bc_in="periodic", bc_out="periodic", bc_top="wall",
                          bc_bottom="axis", axisym=True, Cs=Cs, T_top=1.0)
    o = orc.Oracle(cfg)
    o.set_properties(np.array([nu]), np.array([alpha]), 0.0, 2.0)
    f, g = _polynomial_state(orc, nx, nr, case)
    o.set_state(f, g)
    fs, gs = o.streamed()
    o.step(1)
    f1, g1 = o.get_state()

    e9 = np.array(E9, dtype=float)
    mom = np.stack([fs.sum(0), np.einsum("k,kji->ji", e9[:, 0], fs), np.einsum("k,kji->ji", e9[:, 1], fs),
                    gs.sum(0)])
    P = np.polynomial.polynomial
    cols = np.arange(1, nx - 1)  # streamed from real columns only (no periodic seam)
    rows = np.arange(0, nr - 1)  # streamed from real rows or the axis mirror (no wall)
    X, R = np.meshgrid(cols.astype(float), I.radii(nr)[rows], indexing="xy")
    V = P.polyvander2d(X.ravel(), R.ravel(), [2, 2])
    coef = []
    for c in range(4):
        vals = mom[c][np.ix_(rows, cols)].ravel()
        cf, *_ = np.linalg.lstsq(V, vals, rcond=None)
        assert np.abs(V @ cf - vals).max() < 1e-14  # the streamed moments are that polynomial
        coef.append(cf.reshape(3, 3))
    checked = 0
    for j in range(0, nr - 2):
        r = I.radii(nr)[j]
        for i in range(2, nx - 2):
            d = [P.polyval2d(i, r, P.polyder(coef[1], axis=1)),
                 P.polyval2d(i, r, P.polyder(coef[2], axis=1)),
                 P.polyval2d(i, r, P.polyder(coef[2], axis=0)),
                 P.polyval2d(i, r, P.polyder(coef[3], axis=1))]
            fo, go, _ = orc.collide_node(fs[:, j, i], gs[:, j, i], r, np.array(d), nu, alpha, Cs, 0.3, True)
            np.testing.assert_allclose(f1[:, j, i], fo, rtol=0, atol=1e-14)
            np.testing.assert_allclose(g1[:, j, i], go, rtol=0, atol=1e-14)
            checked += 1
    assert checked == (nr - 2) * (nx - 4)


# ---- boundary rules on tiny lattices ----------------------------------------

def _tiny(orc, nx=3, nr=3, **kw):
    cfg = I.LatticeConfig(nx=nx, nr=nr, **kw)
    o = orc.Oracle(cfg)
    rng = np.random.default_rng(11)
    f = 0.05 + 0.1 * rng.random((9, nr, nx))
    g = 0.2 + 0.1 * rng.random((4, nr, nx))
    o.set_state(f, g, 0)
    return o, f, g


def test_interior_pull(orc):
    o, f, g = _tiny(orc, 4, 4, bc_in="periodic", bc_out="periodic", bc_top="wall")
    fs, gs = o.streamed()
    for k, (ex, ey) in enumerate(E9):
        assert fs[k, 1, 2] == f[k, 1 - ey, 2 - ex]
    for k, (ex, ey) in enumerate(E4):
        assert gs[k, 1, 2] == g[k, 1 - ey, 2 - ex]


def test_axis_is_a_mirror(orc):
    o, f, g = _tiny(orc, bc_in="periodic", bc_out="periodic", bc_top="wall")
    fs, gs = o.streamed()
    # upward populations at row 0 come from the mirror image of downward ones
    assert fs[2, 0, 1] == f[4, 0, 1]
    assert fs[5, 0, 1] == f[8, 0, 0]
    assert fs[6, 0, 1] == f[7, 0, 2]
    assert gs[1, 0, 1] == g[3, 0, 1]


def test_wall_bounce_back(orc):
    o, f, g = _tiny(orc, bc_in="periodic", bc_out="periodic", bc_top="wall", T_top=0.7)
    fs, gs = o.streamed()
    nr = 3
    assert fs[4, nr - 1, 1] == f[2, nr - 1, 1]
    assert fs[7, nr - 1, 1] == f[5, nr - 1, 1]
    assert fs[8, nr - 1, 1] == f[6, nr - 1, 1]
    # thermal anti-bounce-back holds the wall temperature: g_in + g_out = T_wall / 2
    assert gs[3, nr - 1, 1] == pytest.approx(-g[1, nr - 1, 1] + 0.35, abs=1e-16)


def test_inner_wall_and_periodic(orc):
    o, f, g = _tiny(orc, bc_in="periodic", bc_out="periodic", bc_top="wall", bc_bottom="wall",
                    r0=5.0, T_bottom=2.0)
    fs, gs = o.streamed()
    assert fs[2, 0, 1] == f[4, 0, 1]
    assert fs[5, 0, 1] == f[7, 0, 1]
    assert gs[1, 0, 1] == pytest.approx(-g[3, 0, 1] + 1.0, abs=1e-16)
    # periodic wrap in x
    assert fs[1, 1, 0] == f[1, 1, 2]
    assert fs[3, 1, 2] == f[3, 1, 0]


def test_inlet_ghost_is_equilibrium(orc):
    o, f, g = _tiny(orc, bc_in="inlet", bc_out="outflow", bc_top="wall")
    u_in = np.array([0.05, 0.03, 0.01])
    T_in = np.array([9.0, 5.0, 1.0])
    o.set_inlet(u_in, T_in)
    fs, gs = o.streamed()
    for j in range(3):
        rho_b = f[:, j, 0].sum()  # density of the first column's stored populations
        feq = orc.feq(rho_b, u_in[j], 0.0)
        assert fs[1, j, 0] == pytest.approx(feq[1], abs=1e-16)
        geq = orc.geq(T_in[j], u_in[j], 0.0)
        assert gs[0, j, 0] == pytest.approx(geq[0], abs=1e-16)
    # diagonal from row 1 into row 2 at the inlet uses row 1's profile
    rho_b = f[:, 1, 0].sum()
    assert fs[5, 2, 0] == pytest.approx(orc.feq(rho_b, u_in[1], 0.0)[5], abs=1e-16)


def test_inlet_noise_enters_flowing_rows_only(orc):
    """The inlet perturbation xi_{j,t} of the pull at step t is added on rows whose profile flows.

    Rows with zero inlet velocity (the coflow-free part of a nozzle) get no
    noise; the pull of step t uses the generator's value at counter (t, j).
    """
    nx, nr, seed, amp = 3, 3, 77, 1e-3
    cfg = I.LatticeConfig(nx=nx, nr=nr, bc_in="inlet", bc_out="outflow", bc_top="wall",
                          noise_amp=amp, seed=seed)
    o = orc.Oracle(cfg)
    u_in = np.array([0.05, 0.0, 0.02])
    T_in = np.array([3.0, 2.0, 1.0])
    o.set_inlet(u_in, T_in)
    rng = np.random.default_rng(12)
    f = 0.05 + 0.1 * rng.random((9, nr, nx))
    g = 0.2 + 0.1 * rng.random((4, nr, nx))
    for t in (9, 10):
        o.set_state(f, g, t)
        fs, gs = o.streamed()
        for j in range(nr):
            u = u_in[j] + (orc.inlet_noise(seed, t, j, amp) if u_in[j] != 0.0 else 0.0)
            assert fs[1, j, 0] == pytest.approx(orc.feq(f[:, j, 0].sum(), u, 0.0)[1], abs=1e-16)
            assert gs[0, j, 0] == pytest.approx(orc.geq(T_in[j], u, 0.0)[0], abs=1e-16)
        assert abs(fs[1, 0, 0] - orc.feq(f[:, 0, 0].sum(), u_in[0], 0.0)[1]) > 1e-6  # the noise is there


def test_outflow_holds_reference_density(orc):
    o, f, g = _tiny(orc, bc_in="inlet", bc_out="outflow", bc_top="wall")
    fs, gs = o.streamed()
    j, i = 1, 2
    node = f[:, j, i]
    rho = node.sum()
    e = np.array(E9, dtype=float)
    u = e.T @ node / rho
    # the ghost beyond the outlet is the last column shifted back to rho0 = 1
    ghost = node + (1.0 - rho) * orc.feq(1.0, u[0], u[1])
    assert fs[3, j, i] == pytest.approx(ghost[3], abs=1e-15)
    assert ghost.sum() == pytest.approx(1.0, abs=1e-14)
    assert gs[2, j, i] == g[2, j, i]  # temperature: zero gradient


def test_axis_mirror_equals_full_domain(orc):
    """A lattice with the axis evolves exactly like the lower half of its mirrored double.

    Planar model (sources off): the full domain has walls at both radial
    edges and a mirror-symmetric initial state.
    """
    nx, nr = 8, 5
    rng = np.random.default_rng(5)
    f_half = 0.05 + 0.1 * rng.random((9, nr, nx))
    g_half = 0.2 + 0.1 * rng.random((4, nr, nx))
    mir9 = [0, 1, 4, 3, 2, 8, 7, 6, 5]
    mir4 = [0, 3, 2, 1]
    f_full = np.concatenate([f_half[mir9, ::-1, :], f_half], axis=1)
    g_full = np.concatenate([g_half[mir4, ::-1, :], g_half], axis=1)
    common = dict(bc_in="periodic", bc_out="periodic", bc_top="wall", axisym=False, Cs=0.17,
                  T_top=0.3, T_bottom=0.3)
    half = orc.Oracle(I.LatticeConfig(nx=nx, nr=nr, **common))
    full = orc.Oracle(I.LatticeConfig(nx=nx, nr=2 * nr, bc_bottom="wall", r0=1.0, **common))
    nu, al = I.power_law_tables(16, 0.2, 0.6)
    for o in (half, full):
        o.set_properties(nu, al, 0.2, 0.6)
    half.set_state(f_half, g_half)
    full.set_state(f_full, g_full)
    half.step(60)
    full.step(60)
    fh, gh = half.get_state()
    ff, gf = full.get_state()
    np.testing.assert_allclose(ff[:, nr:, :], fh, rtol=0, atol=1e-14)
    np.testing.assert_allclose(gf[:, nr:, :], gh, rtol=0, atol=1e-14)


# ---- conservation -----------------------------------------------------------

def test_mass_conserved_in_closed_domain(orc):
    """Periodic axial ends, axis and wall: planar model conserves total mass to round-off."""
    nx, nr = 24, 12
    cfg = I.LatticeConfig(nx=nx, nr=nr, bc_in="periodic", bc_out="periodic", bc_top="wall",
                          axisym=False, Cs=0.17, T_top=1.0)
    o = orc.Oracle(cfg, nthreads=2)
    nu, al = I.power_law_tables(32, 0.9, 1.2, nu_max=0.05)
    o.set_properties(nu, al, 0.9, 1.2)
    f, g = I.random_state(nx, nr, orc.feq(1.0, 0.0, 0.0), orc.geq(1.0, 0.0, 0.0), 0.05, 9)
    o.set_state(f, g)
    m0 = f.sum()
    steps = 3000
    o.step(steps)
    f1, _ = o.get_state()
    # round-off only: well under one unit of 1e-15 relative per step (a wrong
    # weight or a leaking boundary drifts by 1e-6 or more)
    assert abs(f1.sum() - m0) < 1e-15 * steps * m0


def test_axisymmetric_mass_drift_is_small(orc):
    """With the axisymmetric sources the discrete sum of r rho is conserved only to O(dx^2)."""
    nx, nr = 24, 12
    cfg = I.LatticeConfig(nx=nx, nr=nr, bc_in="periodic", bc_out="periodic", bc_top="wall",
                          axisym=True, Cs=0.0, T_top=1.0)
    o = orc.Oracle(cfg, nthreads=2)
    o.set_properties(np.array([0.05]), np.array([0.05]), 0.0, 1.0)
    f, g = I.random_state(nx, nr, orc.feq(1.0, 0.0, 0.0), orc.geq(1.0, 0.0, 0.0), 0.01, 3)
    o.set_state(f, g)
    r = I.radii(nr)[None, :, None]
    m0 = (r * f).sum()
    o.step(2000)
    f1, _ = o.get_state()
    assert abs((r * f1).sum() - m0) < 1e-3 * m0


def test_rest_state_is_steady(orc):
    cfg = I.LatticeConfig(nx=10, nr=6, bc_in="periodic", bc_out="periodic", bc_top="wall",
                          T_top=1.0, Cs=0.17)
    o = orc.Oracle(cfg)
    f0, g0 = o.get_state()
    o.step(50)
    f1, g1 = o.get_state()
    np.testing.assert_allclose(f1, f0, atol=1e-15)
    np.testing.assert_allclose(g1, g0, atol=1e-15)


# ---- closed-form flows of the axisymmetric equations ------------------------

def _bessel_column(orc, nr, nu, alpha, amp_u, amp_T, axisym=True):
    cfg = I.LatticeConfig(nx=1, nr=nr, bc_in="periodic", bc_out="periodic", bc_top="wall",
                          bc_bottom="axis", axisym=axisym, Cs=0.0, T_top=1.0)
    o = orc.Oracle(cfg)
    o.set_properties(np.array([nu]), np.array([alpha]), 0.0, 2.0)
    from scipy.special import j0

    r = I.radii(nr)
    shape = j0(J0_ZERO * r / nr)
    f = np.zeros((9, nr, 1))
    g = np.zeros((4, nr, 1))
    for j in range(nr):
        f[:, j, 0] = orc.feq(1.0, amp_u * shape[j], 0.0)
        g[:, j, 0] = orc.geq(1.0 + amp_T * shape[j], 0.0, 0.0)
    o.set_state(f, g)
    return o, shape


def _amplitude(field, shape):
    return float(field @ shape / (shape @ shape))


def test_bessel_mode_decay_velocity(orc):
    """Axial velocity u(r) = J0(2.4048 r / R) decays as exp(-nu (2.4048/R)^2 t) keeping its shape."""
    nr, nu = 32, 0.1
    o, shape = _bessel_column(orc, nr, nu, 0.1, 1e-3, 0.0)
    o.step(300)
    a0 = _amplitude(o.fields()[1][:, 0], shape)
    o.step(2000)
    F = o.fields()[1][:, 0]
    a1 = _amplitude(F, shape)
    rate = -math.log(a1 / a0) / 2000
    want = nu * (J0_ZERO / nr) ** 2
    assert rate == pytest.approx(want, rel=0.02)
    resid = F - a1 * shape
    assert np.linalg.norm(resid) < 0.01 * np.linalg.norm(a1 * shape)


def test_bessel_mode_decay_needs_the_axisymmetric_terms(orc):
    """The planar model decays the same profile at a clearly different rate."""
    nr, nu = 32, 0.1
    o, shape = _bessel_column(orc, nr, nu, 0.1, 1e-3, 0.0, axisym=False)
    o.step(300)
    a0 = _amplitude(o.fields()[1][:, 0], shape)
    o.step(2000)
    a1 = _amplitude(o.fields()[1][:, 0], shape)
    rate = -math.log(a1 / a0) / 2000
    assert abs(rate / (nu * (J0_ZERO / nr) ** 2) - 1.0) > 0.2


def test_bessel_mode_decay_temperature(orc):
    """T(r) - T_wall = J0(2.4048 r / R) decays as exp(-alpha (2.4048/R)^2 t)."""
    nr, alpha = 32, 0.15
    o, shape = _bessel_column(orc, nr, 0.1, alpha, 0.0, 0.01)
    o.step(300)
    a0 = _amplitude(o.fields()[3][:, 0] - 1.0, shape)
    o.step(2000)
    T = o.fields()[3][:, 0] - 1.0
    a1 = _amplitude(T, shape)
    rate = -math.log(a1 / a0) / 2000
    assert rate == pytest.approx(alpha * (J0_ZERO / nr) ** 2, rel=0.02)
    assert np.linalg.norm(T - a1 * shape) < 0.01 * np.linalg.norm(a1 * shape)
    # no flow is generated
    assert np.abs(o.fields()[1]).max() == 0.0


def test_radial_conduction_in_annulus(orc):
    """Steady conduction between r1 and r2: T = T1 + (T2 - T1) ln(r/r1) / ln(r2/r1)."""
    r1, nr = 8.0, 24
    r2 = r1 + nr
    cfg = I.LatticeConfig(nx=1, nr=nr, bc_in="periodic", bc_out="periodic", bc_top="wall",
                          bc_bottom="wall", r0=r1, axisym=True, Cs=0.0, T_bottom=1.0, T_top=0.0)
    o = orc.Oracle(cfg)
    o.set_properties(np.array([0.1]), np.array([0.25]), 0.0, 2.0)
    o.step(40000)
    T = o.fields()[3][:, 0]
    r = I.radii(nr, r1)
    want = 1.0 - np.log(r / r1) / np.log(r2 / r1)
    assert np.max(np.abs(T - want)) < 2e-3
    # the planar (linear) profile is far off
    lin = 1.0 - (r - r1) / (r2 - r1)
    assert np.max(np.abs(T - lin)) > 0.03


def test_hagen_poiseuille(orc):
    """Developed pipe flow: parabolic profile and the axisymmetric pressure drop.

    Hagen-Poiseuille needs dp/dx = -4 rho nu u_max / R^2, i.e. a density
    gradient of -12 nu u_max / R^2 (c_s^2 = 1/3); the planar channel needs half.
    """
    w = I.pipe_workload()
    o = orc.Oracle.from_workload(w, nthreads=4)
    o.step(6000)
    F = o.fields()
    nr = w.cfg.nr
    r = I.radii(nr)
    ref = 0.05 * (1 - (r / nr) ** 2)
    for i in (16, 32, 48):
        u = F[1][:, i]
        assert np.linalg.norm(u - ref) < 1e-2 * np.linalg.norm(ref)
    slope = np.polyfit(np.arange(16, 49), F[0][:, 16:49].mean(axis=0), 1)[0]
    want = -12 * 0.1 * 0.05 / nr**2
    assert slope == pytest.approx(want, rel=0.03)
    assert np.abs(F[2]).max() < 1e-3 * 0.05 * 10


def test_developing_pipe_conserves_volume_flux(orc):
    """Plug inlet: at steady state the flux sum_j r_j rho u_x is the same at every section."""
    nx, nr = 48, 16
    cfg = I.LatticeConfig(nx=nx, nr=nr, bc_in="inlet", bc_out="outflow", bc_top="wall",
                          Cs=0.0, T_top=1.0)
    o = orc.Oracle(cfg, nthreads=4)
    o.set_inlet(np.full(nr, 0.04), np.ones(nr))
    o.set_properties(np.array([1.0 / 6.0]), np.array([0.1]), 0.0, 2.0)
    o.step(8000)
    F = o.fields()
    r = I.radii(nr)[:, None]
    flux = (r * F[0] * F[1]).sum(axis=0)
    sec = flux[4:nx - 4]
    assert (sec.max() - sec.min()) < 0.01 * sec.mean()
    # the profile develops: centreline speed rises well above the plug value
    assert F[1][0, nx - 8] > 1.3 * 0.04
    # a planar flux would not be constant along the developing pipe
    plain = (F[0] * F[1]).sum(axis=0)[4:nx - 4]
    assert (plain.max() - plain.min()) > 0.03 * plain.mean()


def test_thread_count_does_not_change_results(orc):
    w = I.jet_workload(nx=40, nr=16, steps=30)
    a = orc.Oracle.from_workload(w, nthreads=1)
    b = orc.Oracle.from_workload(w, nthreads=3)
    a.step(30)
    b.step(30)
    fa, ga = a.get_state()
    fb, gb = b.get_state()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
