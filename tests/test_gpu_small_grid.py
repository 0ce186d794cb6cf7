"""The small-grid path: a whole tdse_propagate call in one thread-block
cluster launch (state and work vectors in shared memory, halos through
distributed shared memory, grid sums in a fixed order).

- Taylor and RK4 perform the same per-point FP64 operations as the
  multi-launch kernels, so both paths give bitwise the same state.
- Lanczos differs from the multi-launch path only in how its grid sums
  associate: one step from the same state matches the oracle within 1e-12.
- The cluster's shape is covered by ragged grids: N smaller than a CTA's
  columns, a last CTA with one or two columns, both stencils (halo 1 and 2),
  lmax = 0, Krylov dimension 1 and Taylor order 1 (its copy stage), the
  absorber, the odd ghost and an offset grid.
- The path is taken only where it applies.
The whole-pulse runs of the small configuration (tests/test_gpu_floor.py)
run on this path too, and assert so.
"""
import numpy as np
import pytest

import oracle
import tdse_workloads as W
from gpu_helpers import grid_of, make, rel_l2

pytestmark = pytest.mark.gpu

PULSE = oracle.Pulse(E0=0.0534, omega=0.057, ncycles=2)

GRIDS = [  # N, dr, L, stencil, ghost, offset, absorber_r
    (2, 0.3, 0, 3, 0, 0.0, None),
    (7, 0.3, 2, 5, 0, 0.0, None),
    (13, 0.25, 1, 5, 1, 0.0, None),
    (33, 0.2, 5, 3, 0, -0.02, 4.0),
    (257, 0.1, 6, 5, 0, 0.0, 20.0),
    (500, 0.2, 4, 3, 0, 0.0, 60.0),
    (1003, 0.05, 9, 5, 1, 0.0, 40.0),
]


def _run(grid, method, order, dt, nsteps, mode, psi, t0=30.0):
    N, dr, L, st, ghost, offset, ra = grid
    t = make(N, dr, L, st, ghost=ghost, offset=offset, pulse=PULSE, absorber_r=ra)
    t.set_small_grid_path(mode)
    t.set_state(psi)
    t.time = t0
    t.propagate(method, order, dt, nsteps)
    used = t.small_grid_path_used
    got = t.get_state()
    t.close()
    return got, used


def _stable_dt(grid, dt):
    N, dr, L = grid[0], grid[1], grid[2]
    return min(dt, 2.5 / (2.7 / dr ** 2 + L * (L + 1) / (2 * dr ** 2) + 1.0 / dr))


@pytest.mark.parametrize("grid", GRIDS, ids=[f"N{g[0]}L{g[2]}s{g[3]}" for g in GRIDS])
@pytest.mark.parametrize("method,order", [("taylor", 8), ("taylor", 1), ("rk4", 4)])
def test_explicit_methods_bitwise_equal_to_multi_launch(grid, method, order):
    N, dr, L = grid[0], grid[1], grid[2]
    dt = _stable_dt(grid, 0.01) * (0.25 if order == 1 else 1.0)
    psi = W.smooth_state(N, dr, L, seed=21)
    a, used_a = _run(grid, method, order, dt, 7, "force", psi)
    b, used_b = _run(grid, method, order, dt, 7, "off", psi)
    assert used_a and not used_b
    assert np.array_equal(a.view(np.float64), b.view(np.float64))


@pytest.mark.parametrize("grid", GRIDS, ids=[f"N{g[0]}L{g[2]}s{g[3]}" for g in GRIDS])
@pytest.mark.parametrize("m", [1, 5, 12, 16])
def test_lanczos_matches_oracle(grid, m):
    N, dr, L, st, ghost, offset, ra = grid
    psi = W.smooth_state(N, dr, L, seed=22)
    dt = 0.02
    got, used = _run(grid, "lanczos", m, dt, 1, "force", psi)
    assert used
    g = grid_of(N, dr, L, st, ghost=ghost, offset=offset)
    mask = oracle.Mask(ra) if ra is not None else None
    want, _ = oracle.propagate(g, psi, "lanczos", m, dt, 1, t0=30.0, pulse=PULSE, mask=mask)
    assert rel_l2(got, want) <= 1e-12, rel_l2(got, want)
    # six steps in one launch, and on the multi-launch path, at a step where
    # the Krylov propagator converges (rho(H) dt <= m/2): both within 10 x the
    # oracle's own rounding floor (its FP64 distance to its long-double build
    # over the same steps) of the long-double oracle
    rho = (2.7 if st == 5 else 2.0) / dr ** 2 + L * (L + 1) / (2 * (dr + offset) ** 2) + 1.0 / (dr + offset)
    dtc = min(dt, 0.5 * m / rho)
    a, _ = _run(grid, "lanczos", m, dtc, 6, "force", psi)
    b, used_b = _run(grid, "lanczos", m, dtc, 6, "off", psi)
    assert not used_b
    f64, _ = oracle.propagate(g, psi, "lanczos", m, dtc, 6, t0=30.0, pulse=PULSE, mask=mask)
    fld, _ = oracle.propagate(g, psi, "lanczos", m, dtc, 6, t0=30.0, pulse=PULSE, mask=mask, precision="fld")
    floor = max(rel_l2(f64, fld), 1e-15)
    assert rel_l2(a, fld) <= 10 * floor, (rel_l2(a, fld), floor)
    assert rel_l2(b, fld) <= 10 * floor, (rel_l2(b, fld), floor)


def test_explicit_methods_match_oracle_small_config():
    """Taylor-8 and RK4 on the small configuration, 20 steps in one launch."""
    c = W.SMALL
    grid = (c.N, c.dr, c.lmax, c.stencil, 0, 0.0, None)
    psi = W.smooth_state(c.N, c.dr, c.lmax, seed=23)
    g = grid_of(c.N, c.dr, c.lmax, c.stencil)
    for method, order in (("taylor", 8), ("rk4", 4)):
        got, used = _run(grid, method, order, 0.01, 20, "auto", psi)
        assert used
        want, _ = oracle.propagate(g, psi, method, order, 0.01, 20, t0=30.0, pulse=PULSE)
        assert rel_l2(got, want) <= 1e-12, (method, rel_l2(got, want))


def test_path_selection():
    c = W.SMALL
    # the small configuration takes it by default
    t = make(c.N, c.dr, c.lmax, c.stencil, pulse=PULSE)
    t.propagate("lanczos", 12, 0.05, 2)
    assert t.small_grid_path_used
    # per-step observables keep the multi-launch path (they run between steps)
    t.record_dipole(8)
    t.propagate("lanczos", 12, 0.05, 2)
    assert not t.small_grid_path_used
    t.close()
    # mixed precision and the velocity gauge keep the multi-launch path
    t = make(c.N, c.dr, c.lmax, c.stencil, pulse=PULSE)
    t.set_options(precision="mixed")
    t.propagate("lanczos", 12, 0.05, 1)
    assert not t.small_grid_path_used
    t.close()
    t = make(c.N, c.dr, c.lmax, c.stencil, pulse=PULSE, gauge="velocity")
    t.propagate("lanczos", 12, 0.05, 1)
    assert not t.small_grid_path_used
    t.close()
    # a grid above the default size takes it only when forced
    N, dr, L = 2000, 0.1, 15
    psi = W.smooth_state(N, dr, L, seed=24)
    grid = (N, dr, L, 5, 0, 0.0, None)
    a, used_auto = _run(grid, "taylor", 4, 1e-4, 3, "auto", psi)
    b, used_force = _run(grid, "taylor", 4, 1e-4, 3, "force", psi)
    assert not used_auto and used_force
    assert np.array_equal(a.view(np.float64), b.view(np.float64))
    # zero steps change nothing
    t = make(c.N, c.dr, c.lmax, c.stencil, pulse=PULSE)
    x = t.get_state()
    t.propagate("taylor", 8, 0.01, 0)
    assert np.array_equal(t.get_state(), x)
    t.close()


def test_lanczos_norm_left_for_the_next_call():
    """A Lanczos run on the cluster path leaves ||psi|| where the next
    multi-launch call starts from it: split runs equal the oracle's whole run."""
    c = W.SMALL
    psi = W.hydrogen_1s(c.N, c.dr, c.lmax)
    t = make(c.N, c.dr, c.lmax, c.stencil, pulse=PULSE)
    t.set_state(psi)
    t.propagate("lanczos", 12, 0.05, 3)
    assert t.small_grid_path_used
    t.set_small_grid_path("off")
    t.propagate("lanczos", 12, 0.05, 3)
    got = t.get_state()
    t.close()
    want, _ = oracle.propagate(grid_of(c.N, c.dr, c.lmax, c.stencil), psi, "lanczos", 12, 0.05, 6, pulse=PULSE)
    assert rel_l2(got, want) <= 1e-12, rel_l2(got, want)
