"""Seeded synthetic inputs for the axisymmetric thermal LBM-LES workloads.

This module only describes and generates inputs: lattice sizes and boundary
kinds, inlet profiles (the shape of Eq. 7), temperature-indexed property
tables (Section 2.3) and random initial states.  It holds none of the
method's arithmetic and is the one module that both the CUDA path and the
CPU oracle take their inputs from.

The paper simulates an Ar-N2 plasma jet on a 200 x 96 half-plane lattice
(Section 2.4) with N2-Ar property data that is not reproduced here; the
workloads below are synthetic jets of the same kind: a hot, fast axisymmetric
jet entering a cold quiescent gas through the lower part of the inlet edge,
with a strongly temperature-dependent viscosity.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

BC_IN = ("inlet", "periodic")
BC_OUT = ("outflow", "wall", "periodic")
BC_TOP = ("wall", "open")
BC_BOTTOM = ("axis", "wall")


@dataclass
class LatticeConfig:
    """Size, boundary kinds and constants of one lattice (lattice units).

    x (index i, ``nx`` nodes) is the axial direction, r (index j, ``nr``
    nodes) the radial one; node j sits at radius ``r0 + j + 1/2``.
    """

    nx: int
    nr: int
    bc_in: str = "inlet"
    bc_out: str = "outflow"
    bc_top: str = "open"
    bc_bottom: str = "axis"
    axisym: bool = True
    r0: float = 0.0
    rho0: float = 1.0
    T0: float = 1.0
    Cs: float = 0.17
    Pr_t: float = 0.3
    T_top: float = 1.0
    T_bottom: float = 1.0
    T_out: float = 1.0
    noise_amp: float = 0.0
    seed: int = 0

    def validate(self) -> None:
        if self.nx < 1 or self.nr < 1:
            raise ValueError("nx and nr must be positive")
        if self.bc_in not in BC_IN or self.bc_out not in BC_OUT:
            raise ValueError("unknown axial boundary kind")
        if self.bc_top not in BC_TOP or self.bc_bottom not in BC_BOTTOM:
            raise ValueError("unknown radial boundary kind")
        if (self.bc_in == "periodic") != (self.bc_out == "periodic"):
            raise ValueError("periodic must be set on both axial ends")
        if self.bc_bottom == "axis" and self.r0 != 0.0:
            raise ValueError("the axis requires r0 == 0")


@dataclass
class Workload:
    """One lattice with its inlet profiles and property tables."""

    name: str
    cfg: LatticeConfig
    u_in: np.ndarray  # (nr,) axial inlet velocity at each row
    T_in: np.ndarray  # (nr,) inlet temperature at each row
    nu_tab: np.ndarray  # (n,) lattice kinematic viscosity on a uniform T grid
    alpha_tab: np.ndarray  # (n,) lattice thermal diffusivity on the same grid
    T_lo: float
    T_hi: float
    steps: int = 0

    @property
    def nodes(self) -> int:
        return self.cfg.nx * self.cfg.nr


def radii(nr: int, r0: float = 0.0) -> np.ndarray:
    """Radius of each lattice row (rows sit half a cell off the bottom edge)."""
    return r0 + np.arange(nr, dtype=np.float64) + 0.5


def constant_tables(nu: float, alpha: float):
    """Temperature-independent properties (a one-entry table)."""
    return np.array([nu]), np.array([alpha])


def power_law_tables(n: int, T_lo: float, T_hi: float, nu_max: float = 1.0 / 3.0,
                     exponent: float = 1.7, prandtl: float = 2.0 / 3.0):
    """Synthetic property tables standing in for the N2-Ar data of Section 2.3.

    nu(T) = nu_max (T / T_hi)^exponent on n uniform points of [T_lo, T_hi];
    alpha = nu / prandtl.  With nu_max = 1/3 the viscosity at T_hi is one
    third in lattice units; at T_hi / T_lo = 10 the cold gas has
    nu = 0.0066.
    """
    T = np.linspace(T_lo, T_hi, n)
    nu = nu_max * (T / T_hi) ** exponent
    return nu, nu / prandtl


def pipe_workload(nx: int = 64, nr: int = 32, u_max: float = 0.05, nu: float = 0.1,
                  alpha: float = 0.15, steps: int = 2000) -> Workload:
    """Laminar Hagen-Poiseuille pipe: parabolic inlet, wall at r = nr, hot inlet, cold wall.

    nu = 0.1 and alpha = 0.15 put both relaxation times at 0.8.
    """
    cfg = LatticeConfig(nx=nx, nr=nr, bc_in="inlet", bc_out="outflow", bc_top="wall",
                        bc_bottom="axis", axisym=True, Cs=0.0, Pr_t=0.3,
                        T_top=0.0, T0=1.0)
    r = radii(nr)
    R = float(nr)
    u_in = u_max * (1.0 - (r / R) ** 2)
    T_in = np.ones(nr)
    nu_t, al_t = constant_tables(nu, alpha)
    return Workload("pipe", cfg, u_in, T_in, nu_t, al_t, 0.0, 1.0, steps)


def jet_profiles(nr: int, R: float, u_max: float, T0: float, T_ratio: float,
                 T_exponent: float = 4.0):
    """Inlet profiles of Eq. 7 for a nozzle of radius R on the lower inlet edge.

    u = u_max (1 - (r/R)^2) and T = T0 + (T_ratio T0 - T0)(1 - (r/R)^T_exponent)
    inside the nozzle; u = 0, T = T0 outside.  Eq. 7 prints the exponent 3 for
    T; the synthetic jets use 4.
    """
    r = radii(nr)
    inside = r < R
    u = np.where(inside, u_max * (1.0 - (r / R) ** 2), 0.0)
    T = np.where(inside, T0 + (T_ratio * T0 - T0) * (1.0 - (r / R) ** T_exponent), T0)
    return u, T


def jet_workload(nx: int = 1024, nr: int = 256, R: Optional[float] = None, u_max: float = 0.08,
                 T_ratio: float = 10.0, Cs: float = 0.17, Pr_t: float = 0.3,
                 noise_amp: float = 1e-3, seed: int = 1234, ntab: int = 256,
                 steps: int = 20000, name: str = "jet") -> Workload:
    """Turbulent hot jet: open top, zero-gradient outflow, Smagorinsky on.

    The default is the 1024 x 256 single jet with a 32-node nozzle; larger
    lattices keep the nozzle at nr / 8.
    """
    if R is None:
        R = nr / 8.0
    cfg = LatticeConfig(nx=nx, nr=nr, bc_in="inlet", bc_out="outflow", bc_top="open",
                        bc_bottom="axis", axisym=True, Cs=Cs, Pr_t=Pr_t, T0=1.0,
                        noise_amp=noise_amp, seed=seed)
    u_in, T_in = jet_profiles(nr, R, u_max, 1.0, T_ratio)
    T_hi = T_ratio
    nu_t, al_t = power_law_tables(ntab, 1.0, T_hi)
    return Workload(name, cfg, u_in, T_in, nu_t, al_t, 1.0, T_hi, steps)


def ensemble_workloads(count: int = 256, seed: int = 7, steps: int = 5000) -> List[Workload]:
    """Ragged ensemble of independent jets.

    nx uniform in {128, 192, ..., 1024}, nr uniform in {64, 96, ..., 256},
    u_max = min(0.1, 0.06 exp(0.2 N(0,1))), temperature ratio uniform in
    [3, 12], nozzle radius nr / 8.
    """
    rng = np.random.default_rng(seed)
    out = []
    for n in range(count):
        nx = int(rng.integers(0, 15)) * 64 + 128
        nr = int(rng.integers(0, 7)) * 32 + 64
        u_max = float(min(0.1, 0.06 * math.exp(0.2 * rng.standard_normal())))
        ratio = float(rng.uniform(3.0, 12.0))
        out.append(jet_workload(nx=nx, nr=nr, u_max=u_max, T_ratio=ratio,
                                seed=seed * 100003 + n, steps=steps, name=f"jet{n}"))
    return out


@dataclass
class Request:
    """One simulation request of a serving stream."""

    rid: int
    arrival_s: float
    workload: Workload


def request_stream(count: int = 2000, rate_per_s: float = 40.0, seed: int = 11,
                   min_steps: int = 1000, max_steps: int = 20000) -> List[Request]:
    """Poisson arrivals of jets drawn like the ensemble, steps uniform in [min, max]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    jets = ensemble_workloads(count, seed=seed + 1)
    for n in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        w = jets[n]
        w.steps = int(rng.integers(min_steps, max_steps + 1))
        out.append(Request(n, t, w))
    return out


def random_state(nx: int, nr: int, base_f, base_g, amp: float, seed: int):
    """Random populations around the given per-direction values.

    base_f (9,) and base_g (4,) are the populations each direction is centred
    on (typically a rest equilibrium); every value is multiplied by
    1 + amp (2U - 1) with U uniform in [0, 1).  Returns f (9, nr, nx) and
    g (4, nr, nx) in float64.
    """
    rng = np.random.default_rng(seed)
    bf = np.asarray(base_f, dtype=np.float64).reshape(9, 1, 1)
    bg = np.asarray(base_g, dtype=np.float64).reshape(4, 1, 1)
    f = bf * (1.0 + amp * (2.0 * rng.random((9, nr, nx)) - 1.0))
    g = bg * (1.0 + amp * (2.0 * rng.random((4, nr, nx)) - 1.0))
    return f, g

