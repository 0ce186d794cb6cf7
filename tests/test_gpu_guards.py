"""Debug guard bands (TDSE_GUARD_BYTES): every path of the handle on ragged
grids (sizes that end inside a tile, lmax = 0, both stencils, the odd
ghost) leaves the 0xff bands around every device buffer intact, and the
bands do not change any result (bitwise against handles without them)."""
import numpy as np
import pytest

import oracle
import tdse_workloads as W
from gpu_helpers import make

pytestmark = pytest.mark.gpu

PULSE = oracle.Pulse(E0=0.0534, omega=0.057, ncycles=2)


def _exercise(N, dr, L, st, ghost, prec, gauge):
    t = make(N, dr, L, st, ghost=ghost, pulse=PULSE, absorber_r=0.7 * N * dr, gauge=gauge)
    t.set_options(ghost=ghost, absorber=True, absorber_r=0.7 * N * dr, precision=prec, gauge=gauge)
    t.set_state(W.random_state(N, L, seed=N + L))
    t.time = 30.0
    t.record(1, 40)
    t.record_dipole(40)
    if N * dr > 2.0:
        t.flux_setup(0.5 * N * dr, np.cos(np.linspace(0.0, np.pi, 9)))
    dt = 0.2 / (2.7 / dr ** 2 + L * (L + 1) / (2 * dr ** 2))
    out = []
    for method, order in (("taylor", 6), ("rk4", 4), ("lanczos", 8), ("lanczos", 1)):
        t.propagate(method, order, dt, 3)
        out.append(t.get_state())
    if prec == "fp64":
        for tb in ("euler", "fehlberg", "dormand_prince", "merson"):
            t.propagate_rk(tb, dt, 2)
            out.append(t.get_state())
    ob = t.observables()
    out.append(np.concatenate([[ob["norm"], ob["dipole"], ob["yield"], ob["p_ground"]], ob["l_pop"]]))
    out.append(t.dipole_moments())
    out.append(t.records()["zdot"])
    blob = t.checkpoint()
    t.restore(blob)
    if prec == "fp64" and gauge == "length":
        t.propagate_imag("lanczos", 8, 0.05, 2)
        out.append(t.get_state())
    t.check_guards()
    t.close()
    return out


@pytest.mark.parametrize("N,dr,L,st,ghost,prec,gauge", [
    (1, 0.2, 0, 5, 0, "fp64", "length"), (7, 0.3, 2, 3, 1, "fp64", "length"),
    (33, 0.2, 5, 5, 0, "fp64", "velocity"), (257, 0.1, 6, 5, 1, "mixed", "length"),
    (517, 0.2, 13, 3, 0, "mixed", "length"), (1000, 0.05, 9, 5, 0, "fp64", "velocity")])
def test_guard_bands_stay_intact(monkeypatch, N, dr, L, st, ghost, prec, gauge):
    monkeypatch.delenv("TDSE_GUARD_BYTES", raising=False)
    plain = _exercise(N, dr, L, st, ghost, prec, gauge)
    monkeypatch.setenv("TDSE_GUARD_BYTES", "4096")
    guarded = _exercise(N, dr, L, st, ghost, prec, gauge)
    for a, b in zip(plain, guarded):
        assert np.array_equal(a, b, equal_nan=True)
