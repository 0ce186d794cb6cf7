"""Parity at the full size of the at-scale configuration (N=8000, dr=0.05,
lmax=63, 5-point stencil, cos^(1/8) mask over the last 50 a.u.), in the launch
configuration the benchmark times: one step of each method from a shared
input, compared element by element with the oracle."""
import numpy as np
import pytest

import oracle
import tdse_workloads as W
from gpu_helpers import grid_of, make, rel_l2

pytestmark = pytest.mark.gpu

C = W.SCALE


def _pulse():
    return oracle.Pulse(E0=C.E0, omega=C.omega, ncycles=C.ncycles)


def _start(seed):
    # smooth start populating the first 20 partial waves
    return W.smooth_state(C.N, C.dr, C.lmax, seed=seed, lmax_populated=20)


@pytest.mark.parametrize("method,order", C.methods)
def test_scale_one_step(method, order):
    psi = _start(31)
    t0 = 0.37 * C.duration
    t = make(C.N, C.dr, C.lmax, C.stencil, pulse=_pulse(), absorber_r=C.R - C.absorber_width)
    t.set_state(psi)
    t.time = t0
    t.propagate(method, order, C.dt, 1)
    got = t.get_state()
    t.close()
    want, _ = oracle.propagate(grid_of(C.N, C.dr, C.lmax, C.stencil), psi, method, order, C.dt, 1,
                               t0=t0, pulse=_pulse(), mask=oracle.Mask(C.R - C.absorber_width))
    assert rel_l2(got, want) <= 1e-12


def test_scale_observables_after_steps():
    psi = W.hydrogen_1s(C.N, C.dr, C.lmax)
    t = make(C.N, C.dr, C.lmax, C.stencil, pulse=_pulse(), absorber_r=C.R - C.absorber_width)
    t.time = 100.0
    t.propagate("lanczos", 12, C.dt, 3)
    got_state = t.get_state()
    got = t.observables()
    t.close()
    want_state, _ = oracle.propagate(grid_of(C.N, C.dr, C.lmax, C.stencil), psi, "lanczos", 12, C.dt,
                                     3, t0=100.0, pulse=_pulse(),
                                     mask=oracle.Mask(C.R - C.absorber_width))
    assert rel_l2(got_state, want_state) <= 1e-11
    want = oracle.observables(grid_of(C.N, C.dr, C.lmax, C.stencil), got_state, psi[0], r_b=10.0)
    for key in ("norm", "dipole", "yield", "p_ground"):
        assert abs(got[key] - want[key]) <= 1e-13 * max(1.0, abs(want[key])), key
