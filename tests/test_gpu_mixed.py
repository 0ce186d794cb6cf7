"""Mixed precision (FP32 stencil on the hi/lo split of psi, complex64 work
vectors, FP64 state, dots, norms and tridiagonal exponential) against the FP64
oracle.

Tolerances come from the arithmetic: the FP32 operator is accurate to a few
FP32 roundings (~1e-7 relative to |Hx|); a step changes psi by ~dt |H psi|, so
one step differs from FP64 by ~1e-9..1e-8 relative; on the well-conditioned
small grid the populations of a many-step run must stay within the 1e-6
relative target.
"""
import numpy as np
import pytest

import oracle
import tdse_workloads as W
from gpu_helpers import apply_h_gpu, grid_of, make, rel_l2

pytestmark = pytest.mark.gpu


def _mixed(N, dr, L, st, **kw):
    t = make(N, dr, L, st, **{k: v for k, v in kw.items() if k != "precision"})
    t.set_options(ghost=kw.get("ghost", 0), offset=kw.get("offset", 0.0),
                  absorber=kw.get("absorber_r") is not None, absorber_r=kw.get("absorber_r") or 0.0,
                  r_b=kw.get("r_b", 10.0), precision="mixed")
    return t


@pytest.mark.parametrize("N,dr,L,st", [(7, 0.3, 2, 3), (33, 0.2, 5, 5), (257, 0.1, 6, 5),
                                       (1000, 0.05, 9, 5), (517, 0.2, 13, 3)])
@pytest.mark.parametrize("ghost,offset", [(0, 0.0), (1, -0.02)])
def test_mixed_apply_h(N, dr, L, st, ghost, offset):
    g = grid_of(N, dr, L, st, ghost=ghost, offset=offset)
    t = _mixed(N, dr, L, st, ghost=ghost, offset=offset)
    for x in (W.smooth_state(N, dr, L, seed=3, offset=offset), W.random_state(N, L, seed=4)):
        for E in (0.0, 0.0534):
            got = apply_h_gpu(t, E, x)
            want = oracle.apply_H(g, E, x)
            assert rel_l2(got, want) <= 2e-6, rel_l2(got, want)
    t.close()


def test_mixed_difference_form_keeps_smooth_accuracy():
    """On a smooth state the difference-form FP32 Laplacian stays within a
    few FP32 roundings (~1e-7..1e-6 relative) although |c0| / |H psi| ~ 1e3 on
    this grid (a plain FP32 stencil would lose ~3 more digits)."""
    N, dr, L = 4000, 0.05, 3
    x = W.hydrogen_1s(N, dr, L)
    g = grid_of(N, dr, L, 5)
    t = _mixed(N, dr, L, 5)
    got = apply_h_gpu(t, 0.0, x)
    want = oracle.apply_H(g, 0.0, x)
    t.close()
    assert rel_l2(got, want) <= 1e-6, rel_l2(got, want)


# explicit methods only at steps inside their stability region (rho(H) dt below
# ~2.8 for RK4 / ~3.4 for Taylor-8): outside it the FP32 rounding noise in the
# stiff modes is amplified by the step polynomial itself
ONE_STEP_CASES = [
    ((500, 0.2, 4, 3), "taylor", 8, 0.01), ((500, 0.2, 4, 3), "rk4", 4, 0.005),
    ((500, 0.2, 4, 3), "lanczos", 12, 0.05), ((500, 0.2, 4, 3), "taylor", 1, 0.001),
    ((500, 0.2, 4, 3), "lanczos", 1, 0.01),
    ((1000, 0.05, 9, 5), "taylor", 8, 1e-4), ((1000, 0.05, 9, 5), "rk4", 4, 1e-4),
    ((1000, 0.05, 9, 5), "lanczos", 12, 0.05), ((1000, 0.05, 9, 5), "lanczos", 1, 0.01),
    ((13, 0.25, 0, 5), "taylor", 8, 0.01), ((13, 0.25, 0, 5), "rk4", 4, 0.005),
    ((13, 0.25, 0, 5), "lanczos", 12, 0.05),
]


@pytest.mark.parametrize("geom,method,order,dt", ONE_STEP_CASES)
def test_mixed_one_step(geom, method, order, dt):
    N, dr, L, st = geom
    pulse = oracle.Pulse(E0=0.0534, omega=0.057, ncycles=2)
    psi = W.smooth_state(N, dr, L, seed=5)
    t = _mixed(N, dr, L, st, pulse=pulse)
    t.set_state(psi)
    t.time = 30.0
    t.propagate(method, order, dt, 1)
    got = t.get_state()
    t.close()
    want, _ = oracle.propagate(grid_of(N, dr, L, st), psi, method, order, dt, 1, t0=30.0, pulse=pulse)
    assert rel_l2(got, want) <= 1e-7, rel_l2(got, want)


@pytest.mark.parametrize("method,order,dt,nsteps", [("taylor", 8, 0.01, 400), ("rk4", 4, 0.01, 400),
                                                    ("lanczos", 12, 0.05, 200)])
def test_mixed_many_steps_populations(method, order, dt, nsteps):
    """Small configuration grid, full field, stable dt: l-populations above
    1e-10 within 1e-6 relative of the FP64 oracle, and the norm (their sum)
    within the same 1e-6 (the mixed Lanczos basis is orthogonal only to FP32
    accuracy, so its norm drifts by ~1e-10 per step)."""
    c = W.SMALL
    pulse = oracle.Pulse(E0=c.E0, omega=c.omega, ncycles=c.ncycles)
    psi0 = W.hydrogen_1s(c.N, c.dr, c.lmax)
    t = _mixed(c.N, c.dr, c.lmax, c.stencil, pulse=pulse)
    t.time = 50.0
    t.propagate(method, order, dt, nsteps)
    got = t.get_state()
    ob = t.observables()
    t.close()
    g = grid_of(c.N, c.dr, c.lmax, c.stencil)
    want, _ = oracle.propagate(g, psi0, method, order, dt, nsteps, t0=50.0, pulse=pulse)
    ow = oracle.observables(g, want, psi0[0], r_b=10.0)
    big = ow["l_pop"] > 1e-10
    rel = np.abs(ob["l_pop"][big] - ow["l_pop"][big]) / ow["l_pop"][big]
    assert rel.max() <= 1e-6, rel
    assert abs(ob["norm"] - ow["norm"]) <= 1e-6
    assert abs(ob["dipole"] - ow["dipole"]) <= 1e-6 * max(1e-3, abs(ow["dipole"]))
    assert rel_l2(got, want) <= 1e-6


def test_mixed_scale_one_step():
    """Full at-scale grid (N=8000, lmax=63, 5-point, mask), one step of each
    method from a smooth state, against the FP64 oracle."""
    C = W.SCALE
    pulse = oracle.Pulse(E0=C.E0, omega=C.omega, ncycles=C.ncycles)
    psi = W.smooth_state(C.N, C.dr, C.lmax, seed=31, lmax_populated=20)
    g = grid_of(C.N, C.dr, C.lmax, C.stencil)
    mask = oracle.Mask(C.R - C.absorber_width)
    for method, order in C.methods:
        dt = C.dt if method == "lanczos" else C.dt_stable
        t = _mixed(C.N, C.dr, C.lmax, C.stencil, pulse=pulse, absorber_r=C.R - C.absorber_width)
        t.set_state(psi)
        t.time = 0.3 * C.duration
        t.propagate(method, order, dt, 1)
        got = t.get_state()
        t.close()
        want, _ = oracle.propagate(g, psi, method, order, dt, 1, t0=0.3 * C.duration, pulse=pulse, mask=mask)
        assert rel_l2(got, want) <= 1e-7, (method, rel_l2(got, want))


def test_mixed_and_fp64_switch_on_one_handle():
    """Switching precision on a handle keeps the state consistent."""
    N, dr, L = 300, 0.1, 3
    psi = W.smooth_state(N, dr, L, seed=8)
    t = make(N, dr, L, 5)
    t.set_state(psi)
    t.propagate("lanczos", 8, 0.02, 3)
    t.set_options(precision="mixed")
    t.propagate("lanczos", 8, 0.02, 3)
    t.set_options(precision="fp64")
    t.propagate("lanczos", 8, 0.02, 3)
    got = t.get_state()
    t.close()
    want, _ = oracle.propagate(grid_of(N, dr, L, 5), psi, "lanczos", 8, 0.02, 9)
    assert rel_l2(got, want) <= 1e-7
