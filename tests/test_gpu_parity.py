"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Tolerances (relative L2 over the whole state): one step from a shared input
<= 1e-12; many steps on a well-conditioned case <= 1e-10.  Both sides compute
in IEEE FP64 with different association orders (Horner vs forward Taylor sum,
fused RK accumulation, blocked reductions), so the differences sit at the
1e-16..1e-14 level per step and grow only with the conditioning of the run.
"""
import math

import numpy as np
import pytest

import oracle
import tdse_workloads as W
from gpu_helpers import apply_h_gpu, grid_of, make, rel_l2

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-12
RUN_TOL = 1e-10

# ragged sizes: smaller than one block, not a multiple of the tile, several tiles
GEOMS = [
    (1, 0.2, 0, 5), (2, 0.2, 1, 5), (7, 0.3, 2, 3), (13, 0.25, 0, 5), (33, 0.2, 5, 5),
    (129, 0.1, 3, 3), (257, 0.1, 6, 5), (1000, 0.05, 9, 5), (517, 0.2, 13, 3),
]


@pytest.mark.parametrize("N,dr,L,st", GEOMS)
@pytest.mark.parametrize("ghost,offset", [(0, 0.0), (1, -0.02)])
def test_apply_h(N, dr, L, st, ghost, offset):
    x = W.random_state(N, L, seed=N + L)
    t = make(N, dr, L, st, ghost=ghost, offset=offset)
    g = grid_of(N, dr, L, st, ghost=ghost, offset=offset)
    for E in (0.0, 0.0534, -0.31):
        got = apply_h_gpu(t, E, x)
        want = oracle.apply_H(g, E, x)
        assert rel_l2(got, want) <= 1e-14, (E, rel_l2(got, want))
    t.close()


def test_apply_h_table_potential_and_charge():
    N, dr, L = 300, 0.1, 4
    r = W.radial_grid(N, dr)
    v = -1.0 / r - 0.5 * np.exp(-r) / r          # a screened SAE-like potential
    x = W.random_state(N, L, seed=3)
    t = make(N, dr, L, 5, vtable=v)
    got = apply_h_gpu(t, 0.02, x)
    want = oracle.apply_H(grid_of(N, dr, L, 5, vtable=v), 0.02, x)
    assert rel_l2(got, want) <= 1e-14
    t.close()
    t = make(N, dr, L, 3, Z=2.0)
    got = apply_h_gpu(t, 0.02, x)
    want = oracle.apply_H(grid_of(N, dr, L, 3, Z=2.0), 0.02, x)
    assert rel_l2(got, want) <= 1e-14
    t.close()


def _one_run(N, dr, L, st, method, order, dt, nsteps, *, t0=30.0, seed=5, absorber_r=None,
             pulse=None, psi=None):
    pulse = pulse or oracle.Pulse(E0=0.0534, omega=0.057, ncycles=2)
    if psi is None:
        psi = W.smooth_state(N, dr, L, seed=seed)
    t = make(N, dr, L, st, pulse=pulse, absorber_r=absorber_r)
    t.set_state(psi)
    t.time = t0
    t.propagate(method, order, dt, nsteps)
    got = t.get_state()
    assert abs(t.time - (t0 + nsteps * dt)) <= 1e-12 * max(1.0, t0)
    t.close()
    mask = oracle.Mask(absorber_r) if absorber_r is not None else None
    want, kmin = oracle.propagate(grid_of(N, dr, L, st), psi, method, order, dt, nsteps, t0=t0,
                                  pulse=pulse, mask=mask)
    return got, want


@pytest.mark.parametrize("N,dr,L,st", [(500, 0.2, 4, 3), (1000, 0.05, 9, 5), (257, 0.1, 6, 5),
                                       (13, 0.25, 0, 5)])
@pytest.mark.parametrize("method,order,dt", [("taylor", 8, 0.01), ("taylor", 1, 0.001),
                                             ("taylor", 12, 0.002), ("rk4", 4, 0.005),
                                             ("lanczos", 12, 0.05), ("lanczos", 1, 0.01),
                                             ("lanczos", 5, 0.02)])
def test_one_step(N, dr, L, st, method, order, dt):
    got, want = _one_run(N, dr, L, st, method, order, dt, 1)
    assert rel_l2(got, want) <= STEP_TOL


@pytest.mark.parametrize("method,order,dt,nsteps", [("taylor", 8, 0.01, 200), ("rk4", 4, 0.01, 200),
                                                    ("lanczos", 12, 0.05, 100)])
def test_many_steps_small_config(method, order, dt, nsteps):
    """The small configuration's grid (N=500, dr=0.2, lmax=4, 3-point) at stable steps."""
    c = W.SMALL
    psi = W.hydrogen_1s(c.N, c.dr, c.lmax)
    got, want = _one_run(c.N, c.dr, c.lmax, c.stencil, method, order, dt, nsteps, t0=0.0, psi=psi)
    assert rel_l2(got, want) <= RUN_TOL


def test_absorber_mask_steps():
    """cos^(1/8) mask over the last 5 a.u. of a 20 a.u. box, every method."""
    for method, order, dt in (("taylor", 10, 0.002), ("rk4", 4, 0.002), ("lanczos", 10, 0.02)):
        got, want = _one_run(400, 0.05, 5, 5, method, order, dt, 20, absorber_r=15.0, seed=9)
        assert rel_l2(got, want) <= RUN_TOL, method


def test_lanczos_breakdown_on_eigenstate():
    """A grid eigenstate spans a 1-dimensional Krylov space (happy breakdown)."""
    N, dr, L = 40, 0.25, 2
    g = grid_of(N, dr, L, 5)
    H = oracle.dense_H(g, 0.0)
    lam, V = np.linalg.eigh(H)
    phi = (1.7 * V[:, 3]).reshape(L + 1, N).astype(complex)
    t = make(N, dr, L, 5)
    t.set_state(phi)
    t.propagate("lanczos", 8, 0.05, 4)
    got = t.get_state()
    t.close()
    want = np.exp(-1j * lam[3] * 0.2) * phi
    assert rel_l2(got, want) <= 1e-12


def test_zero_state_and_zero_steps():
    N, dr, L = 50, 0.2, 2
    for method, order in (("taylor", 4), ("rk4", 4), ("lanczos", 6)):
        t = make(N, dr, L, 5, pulse=oracle.Pulse(E0=0.1, omega=0.3, ncycles=2))
        t.set_state(np.zeros((L + 1, N), complex))
        t.propagate(method, order, 0.01, 3)
        assert np.all(t.get_state() == 0)
        psi = W.smooth_state(N, dr, L, seed=1)
        t.set_state(psi)
        t.propagate(method, order, 0.01, 0)
        assert np.array_equal(t.get_state(), psi)
        t.close()


def test_observables_parity():
    N, dr, L = 600, 0.1, 7
    psi = W.random_state(N, L, seed=12) * 3.0
    ref = W.smooth_state(N, dr, 0, seed=2)[0]
    for r_b in (10.0, 35.55, 1e9, 0.0):
        t = make(N, dr, L, 5, r_b=r_b)
        t.set_state(psi)
        t.set_reference(ref)
        got = t.observables()
        t.close()
        want = oracle.observables(grid_of(N, dr, L, 5), psi, ref, r_b=r_b)
        for key in ("norm", "dipole", "yield", "p_ground"):
            assert abs(got[key] - want[key]) <= 1e-13 * max(1.0, abs(want[key])), (key, r_b)
        assert np.allclose(got["l_pop"], want["l_pop"], rtol=1e-13, atol=0)


def test_initial_state_matches_generator():
    c = W.SMALL
    t = make(c.N, c.dr, c.lmax, c.stencil)
    got = t.get_state()
    ob = t.observables()
    t.close()
    want = W.hydrogen_1s(c.N, c.dr, c.lmax)
    assert rel_l2(got, want) <= 1e-15
    assert abs(ob["norm"] - 1.0) <= 1e-14 and abs(ob["p_ground"] - 1.0) <= 1e-14


def test_nonfinite_detected():
    """Taylor-8 at the small configuration's stated dt = 0.05 overflows."""
    from paper_1308_1856_gb300 import TDSEError
    c = W.SMALL
    t = make(c.N, c.dr, c.lmax, c.stencil, pulse=oracle.Pulse(c.E0, c.omega, c.ncycles))
    t.propagate("taylor", 8, 0.05, 400)
    with pytest.raises(TDSEError) as ei:
        t.observables()
    assert ei.value.code == -4
    t.close()
