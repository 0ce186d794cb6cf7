"""Python face of the serial CPU oracle (``tdse_oracle.c``).

TEST INFRASTRUCTURE ONLY: the slow, plain reference the CUDA path is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this package.  It never imports the CUDA library,
and the CUDA library never imports it.

Arrays are numpy ``complex128`` of shape ``(lmax + 1, N)`` (l-major, as the
vector F of Eq. (h_matrix)).  ``precision="fld"`` selects the long-double
build used to measure the rounding floor of the double build.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import build as _build

TAYLOR, RK4, LANCZOS = 0, 1, 2
METHODS = {"taylor": TAYLOR, "rk4": RK4, "lanczos": LANCZOS}


class _Grid(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_int), ("stencil", ctypes.c_int),
                ("ghost", ctypes.c_int), ("h", ctypes.c_double), ("offset", ctypes.c_double),
                ("Z", ctypes.c_double), ("vtable", ctypes.POINTER(ctypes.c_double)),
                ("gauge", ctypes.c_int)]


class _Pulse(ctypes.Structure):
    _fields_ = [("E0", ctypes.c_double), ("omega", ctypes.c_double),
                ("ncycles", ctypes.c_double), ("cep", ctypes.c_double), ("shape", ctypes.c_int)]


class _Mask(ctypes.Structure):
    _fields_ = [("on", ctypes.c_int), ("r_a", ctypes.c_double)]


@dataclass
class Grid:
    """Radial grid r_j = j*h + offset (j = 1..N) and partial waves l = 0..L."""
    N: int
    h: float
    L: int
    stencil: int = 5
    ghost: int = 0          # 0: zero beyond the box; 1: odd reflection at r = 0
    offset: float = 0.0
    Z: float = 1.0
    vtable: Optional[np.ndarray] = None
    gauge: int = 0          # 0: length gauge (r E coupling); 1: velocity gauge (A coupling)

    def r(self) -> np.ndarray:
        return np.arange(1, self.N + 1, dtype=np.float64) * self.h + self.offset

    def _c(self):
        g = _Grid(self.N, self.L, self.stencil, self.ghost, self.h, self.offset, self.Z, None, self.gauge)
        keep = None
        if self.vtable is not None:
            keep = np.ascontiguousarray(self.vtable, dtype=np.float64)
            assert keep.shape == (self.N,)
            g.vtable = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        return g, keep


@dataclass
class Pulse:
    """shape 0: E(t) = E0 sin^2(pi t / T) sin(omega t + cep), T = 2 pi ncycles / omega;
    shape 1 ("SineA"): A(t) = -(c E0 / omega) sin^2(pi t / T) sin(omega t + cep), E = -(1/c) dA/dt."""
    E0: float = 0.0
    omega: float = 0.057
    ncycles: float = 2.0
    cep: float = 0.0
    shape: int = 0

    def duration(self) -> float:
        return 2.0 * math.pi * self.ncycles / self.omega

    def _c(self):
        return _Pulse(self.E0, self.omega, self.ncycles, self.cep, self.shape)


@dataclass
class Mask:
    """cos^(1/8) absorbing mask for r > r_a."""
    r_a: float
    on: bool = True

    def _c(self):
        return _Mask(1 if self.on else 0, self.r_a)


_LIBS: dict = {}
_PATHS: dict = {}


def register_library(key: str, path: str) -> None:
    """Make another build of tdse_oracle.c (e.g. a planted-mistake copy made by
    a test) selectable through the ``precision`` argument."""
    _PATHS[key] = path
    _LIBS.pop(key, None)


def _lib(precision: str = "f64"):
    if precision not in _LIBS:
        if precision in _PATHS:
            path = _PATHS[precision]
        else:
            _build.build()
            path = _build.lib_path(precision)
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_apply_H.argtypes = [ctypes.POINTER(_Grid), ctypes.c_double, dp, dp]
        lib.orc_propagate.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Pulse),
                                      ctypes.POINTER(_Mask), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_long, dp,
                                      ctypes.POINTER(ctypes.c_int)]
        lib.orc_dipole_moments.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Pulse), ctypes.c_double,
                                           dp, dp]
        lib.orc_flux.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Pulse), ctypes.c_double, dp,
                                 ctypes.c_double, ctypes.c_int, dp, dp, dp]
        lib.orc_propagate_rk.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Pulse),
                                         ctypes.POINTER(_Mask), ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_long, dp, dp]
        lib.orc_propagate_imag.argtypes = [ctypes.POINTER(_Grid), ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_long, dp, dp]
        lib.orc_lanczos_coefficients.argtypes = [ctypes.POINTER(_Grid), ctypes.c_double,
                                                 ctypes.c_int, dp, dp, dp]
        lib.orc_observables.argtypes = [ctypes.POINTER(_Grid), dp, dp, ctypes.c_double, dp]
        lib.orc_field.argtypes = [ctypes.POINTER(_Pulse), ctypes.c_double]
        lib.orc_field.restype = ctypes.c_double
        lib.orc_vecpot.argtypes = [ctypes.POINTER(_Pulse), ctypes.c_double]
        lib.orc_vecpot.restype = ctypes.c_double
        lib.orc_mask_value.argtypes = [ctypes.POINTER(_Mask), ctypes.c_double, ctypes.c_double]
        lib.orc_mask_value.restype = ctypes.c_double
        _LIBS[precision] = lib
    return _LIBS[precision]


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _state(psi: np.ndarray, grid: Grid) -> np.ndarray:
    a = np.ascontiguousarray(psi, dtype=np.complex128).reshape(grid.L + 1, grid.N).copy()
    return a


def _check(rc: int, what: str) -> None:
    if rc < 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def apply_H(grid: Grid, E: float, x: np.ndarray, precision: str = "f64") -> np.ndarray:
    """H(E) x for the length-gauge finite-difference Hamiltonian."""
    xs = _state(x, grid)
    y = np.empty_like(xs)
    g, keep = grid._c()
    _check(_lib(precision).orc_apply_H(ctypes.byref(g), E, _dptr(xs.view(np.float64)),
                                        _dptr(y.view(np.float64))), "apply_H")
    return y


def propagate(grid: Grid, psi: np.ndarray, method: str, order: int, dt: float, nsteps: int,
              t0: float = 0.0, pulse: Optional[Pulse] = None, mask: Optional[Mask] = None,
              precision: str = "f64"):
    """Advance psi by nsteps steps; returns (psi_new, smallest Krylov dimension used)."""
    ps = _state(psi, grid)
    g, keep = grid._c()
    p = (pulse or Pulse())._c()
    m = (mask or Mask(0.0, on=False))._c()
    kmin = ctypes.c_int(0)
    rc = _lib(precision).orc_propagate(ctypes.byref(g), ctypes.byref(p), ctypes.byref(m),
                                       METHODS[method], int(order), float(dt), float(t0),
                                       int(nsteps), _dptr(ps.view(np.float64)),
                                       ctypes.byref(kmin))
    _check(rc, "propagate")
    return ps, kmin.value


RK_TABLEAUS = {"euler": 0, "classic": 1, "fehlberg": 2, "cash_karp": 3, "dormand_prince": 4, "merson": 5}


def propagate_rk(grid: Grid, psi: np.ndarray, tableau: str, dt: float, nsteps: int, t0: float = 0.0,
                 pulse: Optional[Pulse] = None, mask: Optional[Mask] = None, precision: str = "f64"):
    """Explicit RK steps with the named tableau (Sec. "Runge-Kutta"); returns
    (psi_new, sigma = sum over the steps of sqrt(|Delta|^2 / S))."""
    ps = _state(psi, grid)
    g, keep = grid._c()
    p = (pulse or Pulse())._c()
    m = (mask or Mask(0.0, on=False))._c()
    sig = ctypes.c_double(0.0)
    rc = _lib(precision).orc_propagate_rk(ctypes.byref(g), ctypes.byref(p), ctypes.byref(m),
                                          RK_TABLEAUS[tableau], float(dt), float(t0), int(nsteps),
                                          _dptr(ps.view(np.float64)), ctypes.byref(sig))
    _check(rc, "propagate_rk")
    return ps, sig.value


def propagate_imag(grid: Grid, psi: np.ndarray, method: str, order: int, dtau: float, nsteps: int,
                   precision: str = "f64"):
    """Imaginary-time steps (Sec. 3) with renormalisation after each; returns
    (psi_new, energy estimate of the last step)."""
    ps = _state(psi, grid)
    g, keep = grid._c()
    e = ctypes.c_double(0.0)
    rc = _lib(precision).orc_propagate_imag(ctypes.byref(g), METHODS[method], int(order), float(dtau),
                                            int(nsteps), _dptr(ps.view(np.float64)), ctypes.byref(e))
    _check(rc, "propagate_imag")
    return ps, e.value


def lanczos_coefficients(grid: Grid, E: float, m: int, psi: np.ndarray, precision: str = "f64"):
    """(alpha, beta) of the Lanczos recurrence started from psi (one step's worth)."""
    ps = _state(psi, grid)
    alpha = np.zeros(m)
    beta = np.zeros(max(m - 1, 1))
    g, keep = grid._c()
    k = _lib(precision).orc_lanczos_coefficients(ctypes.byref(g), E, m, _dptr(ps.view(np.float64)),
                                                 _dptr(alpha), _dptr(beta))
    _check(k, "lanczos_coefficients")
    return alpha[:k].copy(), beta[:max(k - 1, 0)].copy()


def observables(grid: Grid, psi: np.ndarray, ref0: Optional[np.ndarray] = None,
                r_b: float = float("inf"), precision: str = "f64") -> dict:
    """norm, dipole, yield, p_ground and l-populations (dict)."""
    ps = _state(psi, grid)
    out = np.zeros(4 + grid.L + 1)
    g, keep = grid._c()
    refp = None
    if ref0 is not None:
        r0 = np.ascontiguousarray(ref0, dtype=np.complex128).reshape(grid.N)
        refp = _dptr(r0.view(np.float64))
    _check(_lib(precision).orc_observables(ctypes.byref(g), _dptr(ps.view(np.float64)), refp,
                                           float(r_b), _dptr(out)), "observables")
    return {"norm": out[0], "dipole": out[1], "yield": out[2], "p_ground": out[3],
            "l_pop": out[4:].copy()}


def dipole_moments(grid: Grid, psi: np.ndarray, t: float = 0.0, pulse: Optional[Pulse] = None,
                   precision: str = "f64") -> np.ndarray:
    """[<z>, d<z>/dt, d^2<z>/dt^2] of psi at time t (Sec. 4)."""
    ps = _state(psi, grid)
    g, keep = grid._c()
    p = (pulse or Pulse())._c()
    out = np.zeros(3)
    _check(_lib(precision).orc_dipole_moments(ctypes.byref(g), ctypes.byref(p), float(t),
                                              _dptr(ps.view(np.float64)), _dptr(out)), "dipole_moments")
    return out


def flux(grid: Grid, psi: np.ndarray, r_b: float, cos_theta=None, t: float = 0.0,
         pulse: Optional[Pulse] = None, precision: str = "f64"):
    """(total, per_angle): r_b^2 times the radial current through the sphere
    r = r_b, integrated over the angles and at each cos(theta) (Sec. 4)."""
    ps = _state(psi, grid)
    g, keep = grid._c()
    p = (pulse or Pulse())._c()
    ct = np.ascontiguousarray(np.zeros(0) if cos_theta is None else cos_theta, dtype=np.float64)
    per = np.zeros(max(len(ct), 1))
    tot = np.zeros(1)
    _check(_lib(precision).orc_flux(ctypes.byref(g), ctypes.byref(p), float(t), _dptr(ps.view(np.float64)),
                                    float(r_b), len(ct), _dptr(ct) if len(ct) else None, _dptr(tot),
                                    _dptr(per) if len(ct) else None), "flux")
    return float(tot[0]), per[:len(ct)]


def field(pulse: Pulse, t: float, precision: str = "f64") -> float:
    return _lib(precision).orc_field(ctypes.byref(pulse._c()), float(t))


def vecpot(pulse: Pulse, t: float, precision: str = "f64") -> float:
    """A(t) = -c int_0^t E (composite 5-point Gauss, Sec. 3)."""
    p = pulse._c()
    return _lib(precision).orc_vecpot(ctypes.byref(p), float(t))


def mask_value(mask: Mask, r: float, R: float, precision: str = "f64") -> float:
    return _lib(precision).orc_mask_value(ctypes.byref(mask._c()), float(r), float(R))


def band_H(grid: Grid, E: float = 0.0, l: int = 0, precision: str = "f64") -> np.ndarray:
    """Upper band storage (scipy ``eig_banded`` layout) of the diagonal block h_l,
    read off the oracle's operator by applying it to comb vectors (any grid size)."""
    b = grid.stencil // 2
    N = grid.N
    band = np.zeros((b + 1, N))
    for c in range(b + 1 + b):
        x = np.zeros((grid.L + 1, N), dtype=np.complex128)
        cols = np.arange(c, N, 2 * b + 1)
        x[l, cols] = 1.0
        y = apply_H(grid, E, x, precision)[l].real
        for k in cols:
            for d in range(b + 1):          # entry (k - d, k) lives in band[b - d, k]
                if k - d >= 0:
                    band[b - d, k] = y[k - d]
    return band


def dense_H(grid: Grid, E: float, precision: str = "f64") -> np.ndarray:
    """Dense matrix of H(E) (H(A) in the velocity gauge, complex), assembled
    column by column from apply_H (tiny grids only)."""
    n = (grid.L + 1) * grid.N
    if n > 4096:
        raise ValueError("dense_H is for tiny grids")
    H = np.empty((n, n), dtype=np.complex128 if grid.gauge else np.float64)
    e = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        e[:] = 0
        e[k] = 1
        col = apply_H(grid, E, e.reshape(grid.L + 1, grid.N), precision).reshape(n)
        H[:, k] = col if grid.gauge else col.real
    return H
