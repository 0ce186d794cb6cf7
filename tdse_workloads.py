"""Seeded synthetic workloads for the finite-difference TDSE path.

This module only produces inputs: grid and pulse parameters of the
benchmark configurations, initial wavefunctions and seeded random states, and
the seeded instance specs of the batched configuration.  It holds none of the
propagation arithmetic, and both the CUDA library's tests and the oracle read
their inputs from here.

Configurations (atomic units throughout):
  * ``small``  - hydrogen, N=500, dr=0.2, lmax=4, 3-point stencil, sin^2 pulse
                 E0=0.0534, omega=0.057, 2 cycles, Taylor order 8, dt=0.05
                 (stated; explicit Taylor is unstable there, dt=0.01 is the
                 stable companion).
  * ``scale``  - N=8000, dr=0.05 (r_N=400), lmax=63, 5-point stencil, same
                 pulse over 4 cycles, cos^(1/8) mask over the last 50 a.u.,
                 Taylor-12, RK4 and Lanczos-12 at dt=0.02.
  * ``batched``- 256 instances drawn with seed 1308 (see ``batched_specs``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List

import numpy as np

# Intensity (W/cm^2) that corresponds to a peak field of 1 a.u.
ATOMIC_INTENSITY_W_CM2 = 3.50944506e16
# Photon energy (a.u.) times wavelength (nm)
HARTREE_NM = 45.5633525


@dataclass
class Config:
    name: str
    N: int
    dr: float
    lmax: int
    stencil: int
    E0: float
    omega: float
    ncycles: float
    methods: List[tuple]            # (method, order) pairs
    dt: float
    dt_stable: float
    absorber_width: float = 0.0     # mask over the last absorber_width a.u. (0 = none)
    offset: float = 0.0
    Z: float = 1.0
    extra: dict = field(default_factory=dict)

    @property
    def G(self) -> int:
        """grid points per state vector"""
        return self.N * (self.lmax + 1)

    @property
    def R(self) -> float:
        return self.N * self.dr + self.offset

    @property
    def duration(self) -> float:
        return 2.0 * math.pi * self.ncycles / self.omega

    def nsteps(self, dt: float | None = None) -> int:
        return int(math.ceil(self.duration / (dt or self.dt) - 1e-9))


SMALL = Config("small", N=500, dr=0.2, lmax=4, stencil=3, E0=0.0534, omega=0.057, ncycles=2,
               methods=[("taylor", 8)], dt=0.05, dt_stable=0.01)
SCALE = Config("scale", N=8000, dr=0.05, lmax=63, stencil=5, E0=0.0534, omega=0.057, ncycles=4,
               methods=[("taylor", 12), ("rk4", 4), ("lanczos", 12)], dt=0.02, dt_stable=4e-6,
               absorber_width=50.0)
CONFIGS = {"small": SMALL, "scale": SCALE}


def radial_grid(N: int, dr: float, offset: float = 0.0) -> np.ndarray:
    """r_j = j*dr + offset, j = 1..N (the first point sits one step from the origin)."""
    return np.arange(1, N + 1, dtype=np.float64) * dr + offset


def hydrogen_1s(N: int, dr: float, lmax: int, offset: float = 0.0) -> np.ndarray:
    """P(r) = 2 r exp(-r) in the l = 0 wave, scaled so that dr * sum |P|^2 = 1.

    Returns complex128 of shape (lmax + 1, N).
    """
    r = radial_grid(N, dr, offset)
    F = np.zeros((lmax + 1, N), dtype=np.complex128)
    p = 2.0 * r * np.exp(-r)
    F[0] = p / math.sqrt(dr * float(np.dot(p, p)))
    return F


def smooth_state(N: int, dr: float, lmax: int, seed: int, offset: float = 0.0,
                 lmax_populated: int | None = None) -> np.ndarray:
    """Seeded smooth state: every populated wave is a random complex mix of
    hydrogen-like radial shapes r^(l+1) exp(-r/a) for a few widths a, normalised
    to dr * sum |F|^2 = 1."""
    rng = np.random.default_rng(seed)
    r = radial_grid(N, dr, offset)
    F = np.zeros((lmax + 1, N), dtype=np.complex128)
    top = lmax if lmax_populated is None else min(lmax, lmax_populated)
    widths = (1.0, 2.0, 4.0)
    for l in range(top + 1):
        amp = 0.5 ** l
        for a in widths:
            c = complex(rng.standard_normal(), rng.standard_normal()) * amp
            shape = (r / a) ** (l + 1) * np.exp(-r / a)
            F[l] += c * shape / max(1e-300, float(np.max(np.abs(shape))))
    F /= math.sqrt(dr * float(np.vdot(F, F).real))
    return F


def random_state(N: int, lmax: int, seed: int) -> np.ndarray:
    """Seeded complex Gaussian noise of shape (lmax + 1, N), unit 2-norm."""
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((lmax + 1, N)) + 1j * rng.standard_normal((lmax + 1, N))
    F /= np.linalg.norm(F)
    return F


@dataclass
class InstanceSpec:
    N: int
    dr: float
    lmax: int
    intensity_w_cm2: float
    wavelength_nm: float
    ncycles: int
    krylov: int

    @property
    def E0(self) -> float:
        return math.sqrt(self.intensity_w_cm2 / ATOMIC_INTENSITY_W_CM2)

    @property
    def omega(self) -> float:
        return HARTREE_NM / self.wavelength_nm


def batched_specs(count: int = 256, seed: int = 1308) -> List[InstanceSpec]:
    """Instances of the batched configuration: N ~ U{2000..16000}, dr = 0.1,
    lmax ~ U{15..127}, intensity log-uniform in [1e13, 5e14] W/cm^2,
    wavelength ~ U[400, 1600] nm, cycles ~ U{2..6}, Krylov dimension ~ U{8..16}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        N = int(rng.integers(2000, 16001))
        lmax = int(rng.integers(15, 128))
        I = float(math.exp(rng.uniform(math.log(1e13), math.log(5e14))))
        lam = float(rng.uniform(400.0, 1600.0))
        nc = int(rng.integers(2, 7))
        m = int(rng.integers(8, 17))
        out.append(InstanceSpec(N, 0.1, lmax, I, lam, nc, m))
    return out


def converging_dt(N: int, dr: float, lmax: int, krylov: int, stencil: int = 5, E0: float = 0.0,
                  offset: float = 0.0) -> float:
    """A step at which a Krylov propagator of dimension `krylov` converges on
    this grid: rho dt = krylov / 2, with rho a Gershgorin bound on the
    spectral radius of the operator (the second-difference weights
    (30 + 32 + 2)/24 or 4/2 over dr^2, the largest centrifugal term at the
    first point, the Coulomb term there and the coupling r_N E0 (k + k)).
    This chooses an input (the step); it is not part of the propagation."""
    r1 = dr + offset
    lap = (64.0 / 24.0 if stencil == 5 else 2.0) / (dr * dr)
    rho = lap + lmax * (lmax + 1) / (2.0 * r1 * r1) + 1.0 / r1 + 2.0 * abs(E0) * (N * dr + offset)
    return 0.5 * krylov / rho


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of `count` requests of a Poisson process of the given
    mean rate (req/s): exponential gaps, the first request at t = 0."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, count)
    gaps[0] = 0.0
    return np.cumsum(gaps)
