"""The CPU oracle against what the paper and the mathematics fix (no GPU)."""
import math

import numpy as np
import pytest

import oracle
import oracle_pins
import tdse_workloads as W


@pytest.mark.parametrize("check", oracle_pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pin_double(check):
    check("f64")


@pytest.mark.parametrize("check", [oracle_pins.check_symmetric, oracle_pins.check_dense_expm,
                                   oracle_pins.check_field_free_eigenstate,
                                   oracle_pins.check_observables],
                         ids=lambda c: c.__name__)
def test_pin_long_double(check):
    """The long-double build (the rounding-floor instrument) obeys the same pins."""
    check("fld")


def test_long_double_is_wider():
    import ctypes
    lib = oracle._lib("fld")
    assert lib.orc_real_bytes() > 8 or np.finfo(np.longdouble).nmant <= 52


def test_initial_state_on_grid():
    """dr * sum (2 r e^{-r})^2 at dr = 0.2, N = 500 is the Riemann sum of
    int 4 r^2 e^{-2r} dr = 1 (Sec. 6, 1s radial probability); the generator
    rescales it to exactly 1."""
    r = W.radial_grid(500, 0.2)
    raw = 0.2 * float(np.sum((2 * r * np.exp(-r)) ** 2))
    assert abs(raw - 1.0) < 2e-4
    # Euler-Maclaurin: the sum equals the integral minus h^2/12 f'(0) + O(h^4), f'(0) = 0,
    # so the deficit is the h^4 term: tiny and negative
    assert 0 < 1.0 - raw < 2e-4
    F = W.hydrogen_1s(500, 0.2, 4)
    assert F.shape == (5, 500)
    assert abs(0.2 * float(np.sum(np.abs(F) ** 2)) - 1.0) < 1e-14
    assert np.all(F[1:] == 0)


def test_oracle_rejects_bad_arguments():
    g = oracle.Grid(N=10, h=0.1, L=1, stencil=4)
    with pytest.raises(ValueError):
        oracle.apply_H(g, 0.0, np.zeros((2, 10), complex))
    g = oracle.Grid(N=10, h=0.1, L=1, stencil=5)
    with pytest.raises(ValueError):
        oracle.propagate(g, np.zeros((2, 10), complex), "lanczos", 0, 0.1, 1)
    with pytest.raises(ValueError):
        oracle.propagate(g, np.zeros((2, 10), complex), "taylor", 4, -0.1, 1)


def test_lanczos_zero_state_and_single_point():
    """Degenerate inputs: a zero state stays zero; N = 1, lmax = 0 works."""
    g = oracle.Grid(N=1, h=0.2, L=0, stencil=5)
    psi = np.array([[1.0 + 0.5j]])
    out, k = oracle.propagate(g, psi, "lanczos", 4, 0.1, 2)
    Hs = oracle.dense_H(g, 0.0)[0, 0]
    assert k == 1
    assert abs(out[0, 0] - psi[0, 0] * np.exp(-2j * Hs * 0.1)) < 1e-14
    z, _ = oracle.propagate(oracle.Grid(N=7, h=0.2, L=2), np.zeros((3, 7), complex),
                            "lanczos", 4, 0.1, 1)
    assert np.all(z == 0)


def test_rk_and_observable_degenerate_inputs():
    """Zero steps leave the state and sigma at zero; a state in l = 0 alone
    has no dipole, no dipole velocity and only the field term -E ||psi||^2 in
    its acceleration (every pair sum over (l, l+1) vanishes); without angles
    the flux returns no density, and a real state carries no current."""
    g = oracle.Grid(N=50, h=0.2, L=3, stencil=5)
    psi = np.zeros((4, 50), complex)
    psi[0] = W.hydrogen_1s(50, 0.2, 3)[0]
    out, sig = oracle.propagate_rk(g, psi, "dormand_prince", 0.01, 0)
    assert np.array_equal(out, psi) and sig == 0.0
    pulse = oracle.Pulse(E0=0.05, omega=0.3, ncycles=2)
    t = 3.0
    z, zdot, zddot = oracle.dipole_moments(g, psi, t, pulse)
    norm = 0.2 * float(np.sum(np.abs(psi) ** 2))
    assert z == 0.0 and zdot == 0.0
    assert abs(zddot + oracle.field(pulse, t) * norm) <= 1e-15
    tot, per = oracle.flux(g, psi, 5.0)
    assert per.shape == (0,) and tot == 0.0      # a real state carries no current
