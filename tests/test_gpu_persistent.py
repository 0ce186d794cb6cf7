"""The one-launch Lanczos path of larger grids (tdse_set_persistent_path):
every step of a call in one cooperative launch.  Its work split and the
order of every reduction are the multi-launch path's, so the states are
compared BITWISE with that path (and, through it, with the oracle by the
parity tests, which take this path on their larger FP64 grids).  Covered:
both stencils, ragged grids smaller than a wave, Krylov dimensions 1, 12, 16
and 32, a pulse and an absorber, calls split differently, the scalars it
leaves for the next call, the observables, and the cases it must leave to the
multi-launch path (per-step observables, the velocity gauge, mixed precision)."""
import numpy as np
import pytest

import oracle
import tdse_workloads as W
from gpu_helpers import grid_of, make, rel_l2

pytestmark = pytest.mark.gpu

PULSE = oracle.Pulse(E0=0.0534, omega=0.057, ncycles=2)


def _run(N, dr, L, st, m, dt, splits, path, psi, absorber_r=None, t0=40.0, small="off"):
    t = make(N, dr, L, st, pulse=PULSE, absorber_r=absorber_r)
    t.set_small_grid_path(small)
    t.set_persistent_path(path)
    t.set_state(psi)
    t.time = t0
    used = []
    for n in splits:
        t.propagate("lanczos", m, dt, n)
        used.append(t.persistent_path_used)
    out = t.get_state()
    ob = t.observables()
    t.close()
    return out, ob, used


@pytest.mark.parametrize("N,dr,L,st,m,dt,absorber", [
    (2000, 0.1, 15, 5, 12, 0.002, 150.0),
    (1001, 0.2, 3, 3, 16, 0.01, None),
    (33, 0.3, 0, 5, 1, 0.01, None),
    (517, 0.1, 9, 5, 32, 0.002, 40.0),
    (700, 0.15, 6, 3, 12, 0.005, 80.0),
])
def test_persistent_equals_multi_launch_bitwise(N, dr, L, st, m, dt, absorber):
    psi = W.smooth_state(N, dr, L, seed=N + L)
    a, oa, ua = _run(N, dr, L, st, m, dt, [5], "off", psi, absorber)
    b, ob, ub = _run(N, dr, L, st, m, dt, [5], "force", psi, absorber)
    assert ua == [False] and ub == [True]
    assert np.array_equal(a, b)
    for k in ("norm", "dipole", "yield", "p_ground"):
        assert oa[k] == ob[k], k


def test_persistent_calls_split_and_scalars_carried():
    """3 + 1 + 4 steps on the one-launch path equal 8 steps in one call and
    8 multi-launch steps (the scalars each call leaves in the handle are
    the multi-launch path's); by default the multi-launch path runs."""
    N, dr, L, st = 3000, 0.1, 7, 5
    psi = W.smooth_state(N, dr, L, seed=5)
    a, _, ua = _run(N, dr, L, st, 12, 0.003, [3, 1, 4], "force", psi, 250.0)
    b, _, _ = _run(N, dr, L, st, 12, 0.003, [8], "force", psi, 250.0)
    c, _, uc = _run(N, dr, L, st, 12, 0.003, [8], "auto", psi, 250.0)
    assert ua == [True, True, True] and uc == [False]
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_persistent_matches_oracle():
    # a step at which Lanczos-12 converges (rho(H) dt = m / 2): two correct
    # implementations then agree to rounding
    N, dr, L, st, m = 1500, 0.1, 11, 5, 12
    dt = W.converging_dt(N, dr, L, m, st)
    psi = W.smooth_state(N, dr, L, seed=8)
    got, _, used = _run(N, dr, L, st, m, dt, [6], "force", psi, 120.0)
    assert used == [True]
    g = grid_of(N, dr, L, st)
    want, _ = oracle.propagate(g, psi, "lanczos", m, dt, 6, t0=40.0, pulse=PULSE, mask=oracle.Mask(120.0))
    assert rel_l2(got, want) <= 1e-12, rel_l2(got, want)


def test_persistent_left_to_multi_launch():
    """Per-step observables, the velocity gauge and mixed precision run on the
    multi-launch path even when the one-launch path is forced."""
    N, dr, L = 2000, 0.1, 9
    psi = W.smooth_state(N, dr, L, seed=3)
    t = make(N, dr, L, 5, pulse=PULSE)
    t.set_persistent_path("force")
    t.set_state(psi)
    t.record_dipole(4)
    t.propagate("lanczos", 12, 0.002, 2)
    assert not t.persistent_path_used
    t.record_dipole(0)
    t.propagate("lanczos", 12, 0.002, 2)
    assert t.persistent_path_used
    t.close()
    t = make(N, dr, L, 5, pulse=PULSE, gauge="velocity")
    t.set_persistent_path("force")
    t.set_state(psi)
    t.propagate("lanczos", 12, 0.002, 2)
    assert not t.persistent_path_used
    t.close()
    t = make(N, dr, L, 5, pulse=PULSE)
    t.set_options(precision="mixed")
    t.set_persistent_path("force")
    t.set_state(psi)
    t.propagate("lanczos", 12, 0.002, 2)
    assert not t.persistent_path_used
    t.close()
    from paper_1308_1856_gb300 import _binding as C
    t = make(50, 0.2, 1, 5)
    assert C.tdse_set_persistent_path(t.h, 7) == C.TDSE_ERR_ARG
    t.close()
