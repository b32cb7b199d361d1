"""The oracle's pins catch plausible mistakes.

Each mutation below plants one mistake in a copy of oracle/lbm_oracle.c
(on the CPU), builds it, and runs the pin suite against it: every mutant
must make at least one pin fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm_oracle.c")

MUTATIONS = [
    ("mass source without its lattice weight", "W9[k] * F1 +", "F1 +"),
    ("axisymmetric viscous term with the wrong sign", "F2x = -jx * ur / r + nu_tot / r * (d[0] + d[2]);",
     "F2x = -jx * ur / r - nu_tot / r * (d[0] + d[2]);"),
    ("hoop-stress term dropped", " - 2.0 * nu_tot * jr / (r * r);", ";"),
    ("radial conduction term dropped", "S = -T * ur / r + alpha_tot / r * d[3];", "S = -T * ur / r;"),
    ("rows at integer radii", "double r = s->p.r0 + (double)j + 0.5;", "double r = s->p.r0 + (double)j + 1.0;"),
    ("equilibrium quadratic coefficient", "4.5 * eu * eu", "3.0 * eu * eu"),
    ("stress norm without its factor 2", "sqrt(2.0 * (Qxx * Qxx", "sqrt(1.0 * (Qxx * Qxx"),
    ("Eq. 4 with 9 instead of 18", "18.0 * Cs * Cs * Qn / rho", "9.0 * Cs * Cs * Qn / rho"),
    ("axis reflects diagonals through the origin", "static const int MIR9[9] = {0, 1, 4, 3, 2, 8, 7, 6, 5};",
     "static const int MIR9[9] = {0, 1, 4, 3, 2, 7, 8, 5, 6};"),
    ("wall temperature halved", "+ 0.5 * p->T_top;", "+ 0.25 * p->T_top;"),
    ("outflow density correction with the wrong sign", "v += (p->rho0 - rb) * feq[kk];",
     "v -= (p->rho0 - rb) * feq[kk];"),
    ("inlet at the reference density", "orc_feq(rb, inlet_velocity(s, js, t), 0.0, feq);",
     "orc_feq(p->rho0, inlet_velocity(s, js, t), 0.0, feq);"),
    ("thermal equilibrium without the factor 2", "0.25 * T * (1.0 + 2.0 * eu)", "0.25 * T * (1.0 + eu)"),
    ("turbulent Prandtl number multiplies", "alpha + nu_t / Pr_t", "alpha + nu_t * Pr_t"),
    ("table interpolation adds the neighbours", "fr * (tab[m + 1] - tab[m])", "fr * (tab[m + 1] + tab[m])"),
    ("radial momentum even across the axis", "return (c == 2) ? -v : v;", "return v;"),
    ("thermal relaxation with the momentum time", "gs[k] - (gs[k] - geq[k]) / tau_al_tot",
     "gs[k] - (gs[k] - geq[k]) / tau_tot"),
    ("central difference without the 1/2", "d[1] = 0.5 * (moment_at(s, 2, i, j + 1, t)",
     "d[1] = 1.0 * (moment_at(s, 2, i, j + 1, t)"),
    ("axial derivative reversed", "d[2] = 0.5 * (moment_at(s, 2, i + 1, j, t) - moment_at(s, 2, i - 1, j, t));",
     "d[2] = 0.5 * (moment_at(s, 2, i - 1, j, t) - moment_at(s, 2, i + 1, j, t));"),
    ("temperature odd across the axis", "return (c == 2) ? -v : v;", "return (c == 2 || c == 3) ? -v : v;"),
    ("inlet noise on every row", "if (u != 0.0 && s->p.noise_amp != 0.0)", "if (s->p.noise_amp != 0.0)"),
    ("inlet noise of the next step", "u += orc_inlet_noise(s->p.seed, t, j, s->p.noise_amp);",
     "u += orc_inlet_noise(s->p.seed, t + 1, j, s->p.noise_amp);"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_the_mutation(tmp_path, name, old, new):
    from oracle import oracle

    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = oracle.compile_source(str(mutant), str(tmp_path / "libmutant.so"))
    env = dict(os.environ, ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x",
                        "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, f"no pin caught: {name}"
