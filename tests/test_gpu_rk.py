"""Explicit Runge-Kutta methods and embedded pairs (appendix "Runge-Kutta") on
the GPU against the oracle: every tableau on ragged grids with field and
absorber, the velocity gauge, the at-scale grid, determinism, the classic
tableau against the dedicated RK4 path, and the argument checks.

Tolerances: the state within 1e-12 relative (both sides in FP64, the GPU
fusing each multiply-add of the stage sums, so they differ by a few unit
roundoffs per stage over three steps at dt rho(H) <= 1).  sigma within 1e-9
relative: Delta = dt sum (b_i - bhat_i) k_i cancels the slopes (|k_i| ~
rho(H) |psi|) down to the local error, >= ~1e-4 |psi| at these steps, so its
rounding is ~1e-12 relative; 1e-9 leaves room for the sqrt and the sums.
"""
import numpy as np
import pytest

import oracle
import tdse_workloads as W
from gpu_helpers import grid_of, make, rel_l2

pytestmark = pytest.mark.gpu

TABLEAUS = ["euler", "classic", "fehlberg", "cash_karp", "dormand_prince", "merson"]
NO_PAIR = ("euler", "classic")
GEOMS = [(1, 0.2, 0, 5), (7, 0.3, 2, 3), (257, 0.1, 6, 5), (517, 0.2, 13, 3), (1000, 0.05, 9, 5)]
PULSE = oracle.Pulse(E0=0.0534, omega=0.057, ncycles=2)


def _stable_dt(dr, L):
    # rho(H) bound: kinetic ~2.7/dr^2 plus the largest centrifugal term at r = dr
    return 1.0 / (2.7 / dr ** 2 + L * (L + 1) / (2 * dr ** 2))


def _run(N, dr, L, st, tableau, dt, nsteps, psi, *, gauge="length", absorber_r=None, t0=70.0):
    t = make(N, dr, L, st, pulse=PULSE, absorber_r=absorber_r, gauge=gauge)
    t.set_state(psi)
    t.time = t0
    sig = t.propagate_rk(tableau, dt, nsteps)
    out = t.get_state(), sig, t.time
    t.close()
    return out


def _oracle(N, dr, L, st, tableau, dt, nsteps, psi, *, gauge=0, absorber_r=None, t0=70.0):
    mask = oracle.Mask(absorber_r) if absorber_r is not None else None
    return oracle.propagate_rk(grid_of(N, dr, L, st, gauge=gauge), psi, tableau, dt, nsteps, t0=t0,
                               pulse=PULSE, mask=mask)


def _check(got, sig, want, wsig, tableau):
    assert rel_l2(got, want) <= 1e-12, rel_l2(got, want)
    if tableau in NO_PAIR:
        assert sig == 0.0 and wsig == 0.0, (sig, wsig)
    else:
        assert wsig > 0.0
        assert abs(sig - wsig) <= 1e-9 * wsig, (sig, wsig)


@pytest.mark.parametrize("tableau", TABLEAUS)
@pytest.mark.parametrize("N,dr,L,st", GEOMS)
def test_rk_steps_vs_oracle(tableau, N, dr, L, st):
    """Three steps with the field on and the absorber over the outer 30 %."""
    dt = _stable_dt(dr, L)
    psi = W.random_state(N, L, seed=N + 7 * L)
    absorber_r = 0.7 * N * dr
    got, sig, time = _run(N, dr, L, st, tableau, dt, 3, psi, absorber_r=absorber_r)
    want, wsig = _oracle(N, dr, L, st, tableau, dt, 3, psi, absorber_r=absorber_r)
    _check(got, sig, want, wsig, tableau)
    assert abs(time - (70.0 + 3 * dt)) <= 1e-12


@pytest.mark.parametrize("tableau", ["fehlberg", "dormand_prince", "merson"])
def test_rk_velocity_gauge(tableau):
    N, dr, L, st = 1000, 0.05, 9, 5
    dt = _stable_dt(dr, L)
    # a random state: a smooth one's local error (~1e-15 here) is the size of
    # Delta's own rounding, which would make sigma a rounding measurement
    psi = W.random_state(N, L, seed=5)
    got, sig, _ = _run(N, dr, L, st, tableau, dt, 3, psi, gauge="velocity")
    want, wsig = _oracle(N, dr, L, st, tableau, dt, 3, psi, gauge=1)
    _check(got, sig, want, wsig, tableau)


@pytest.mark.parametrize("tableau", ["cash_karp", "dormand_prince"])
def test_rk_at_scale(tableau):
    """The at-scale grid (N=8000, dr=0.05, lmax=63, 5-point, absorber), two
    steps at the explicit stability limit of its centrifugal term."""
    C = W.SCALE
    dt = _stable_dt(C.dr, C.lmax)
    psi = W.random_state(C.N, C.lmax, seed=31)
    absorber_r = C.R - C.absorber_width
    got, sig, _ = _run(C.N, C.dr, C.lmax, C.stencil, tableau, dt, 2, psi, absorber_r=absorber_r,
                       t0=0.37 * C.duration)
    want, wsig = _oracle(C.N, C.dr, C.lmax, C.stencil, tableau, dt, 2, psi, absorber_r=absorber_r,
                         t0=0.37 * C.duration)
    _check(got, sig, want, wsig, tableau)


def test_rk_deterministic():
    """Same input twice: bit-identical state and sigma (fixed reduction order)."""
    N, dr, L, st = 517, 0.2, 13, 3
    psi = W.random_state(N, L, seed=2)
    a, sa, _ = _run(N, dr, L, st, "dormand_prince", _stable_dt(dr, L), 4, psi)
    b, sb, _ = _run(N, dr, L, st, "dormand_prince", _stable_dt(dr, L), 4, psi)
    assert np.array_equal(a, b) and sa == sb


def test_rk_classic_matches_rk4_path():
    """The classic tableau through the general stage kernel and the dedicated
    RK4 kernels compute the same method (different association orders)."""
    N, dr, L, st = 1000, 0.05, 9, 5
    dt = _stable_dt(dr, L)
    psi = W.random_state(N, L, seed=9)
    got, sig, _ = _run(N, dr, L, st, "classic", dt, 5, psi)
    t = make(N, dr, L, st, pulse=PULSE)
    t.set_state(psi)
    t.time = 70.0
    t.propagate("rk4", 4, dt, 5)
    ref = t.get_state()
    t.close()
    assert sig == 0.0
    assert rel_l2(got, ref) <= 1e-13, rel_l2(got, ref)


def test_rk_arguments_and_edges():
    from paper_1308_1856_gb300 import TDSEError, _binding as C
    import ctypes
    N, dr, L = 33, 0.2, 5
    psi = W.random_state(N, L, seed=1)
    t = make(N, dr, L, 5, pulse=PULSE)
    t.set_state(psi)
    # zero steps: state, time and sigma unchanged
    assert t.propagate_rk("dormand_prince", 0.01, 0) == 0.0
    assert np.array_equal(t.get_state(), psi) and t.time == 0.0
    for bad in (lambda: t.propagate_rk("fehlberg", 0.0, 1), lambda: t.propagate_rk("fehlberg", -1.0, 1),
                lambda: t.propagate_rk("fehlberg", 0.01, -1)):
        with pytest.raises(TDSEError) as e:
            bad()
        assert e.value.code == C.TDSE_ERR_ARG
    sig = ctypes.c_double()
    assert C.tdse_propagate_rk(t.h, 6, 0.01, 1, ctypes.byref(sig)) == C.TDSE_ERR_ARG
    assert C.tdse_propagate_rk(t.h, -1, 0.01, 1, ctypes.byref(sig)) == C.TDSE_ERR_ARG
    # sigma may be NULL
    assert C.tdse_propagate_rk(t.h, C.TDSE_RK_MERSON, 0.001, 1, None) == C.TDSE_OK
    # a step far beyond the stability limit overflows to Inf: reported, handle still usable
    with pytest.raises(TDSEError) as e:
        t.propagate_rk("euler", 1e3, 200)
    assert e.value.code == C.TDSE_ERR_NONFINITE
    t.set_state(psi)
    t.time = 0.0
    t.propagate_rk("classic", 0.001, 1)
    assert np.all(np.isfinite(t.get_state()))
    # FP64 only
    t.set_options(precision="mixed")
    with pytest.raises(TDSEError) as e:
        t.propagate_rk("classic", 0.001, 1)
    assert e.value.code == C.TDSE_ERR_ARG
    t.close()
