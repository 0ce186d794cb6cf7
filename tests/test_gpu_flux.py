"""Sec. 4 dipole velocity/acceleration and the flux through r = r_b on the GPU
against the oracle: one-shot moments on ragged grids (both stencils, the odd
ghost, both gauges, the at-scale grid), the per-step dipole series, the flux
and PAD integrals along a propagation, and the argument checks.

Tolerances.  The moments are dr-weighted sums of O(G) products; both sides
round each product once and sum in different orders, so the difference is a
few unit roundoffs of the sum of absolute terms.  Those are bounded by
norm * r_max (<z>), norm / dr (<zdot>: the first-derivative weights) and
norm / dr^2 + |E| norm (<zddot>: 1/r^2 at r = dr); the test allows 1e-12 of
each bound.  The flux is an O(L) sum at one radius, held to 1e-12 of
sum_l |f_l| |D1 f_l| (its absolute terms), the densities the same with the
harmonics' weight; the time integrals add the trapezoid's per-step sums, so
they carry the per-step bound times the elapsed time."""
import math

import numpy as np
import pytest

import oracle
import tdse_workloads as W
from gpu_helpers import grid_of, make

pytestmark = pytest.mark.gpu

PULSE = oracle.Pulse(E0=0.0534, omega=0.057, ncycles=2)


def _scales(psi, dr, N, E):
    norm = dr * float(np.sum(np.abs(psi) ** 2))
    return np.array([norm * N * dr, norm / dr, norm / dr ** 2 + abs(E) * norm])


@pytest.mark.parametrize("N,dr,L,st,ghost,gauge", [
    (7, 0.3, 2, 3, 0, "length"), (33, 0.2, 5, 5, 0, "length"), (257, 0.1, 6, 5, 1, "length"),
    (517, 0.2, 13, 3, 0, "velocity"), (1000, 0.05, 9, 5, 0, "velocity"), (1000, 0.05, 9, 5, 1, "length")])
def test_dipole_moments_vs_oracle(N, dr, L, st, ghost, gauge):
    psi = W.random_state(N, L, seed=N + L)
    t0 = 70.0
    tt = make(N, dr, L, st, ghost=ghost, pulse=PULSE, gauge=gauge)
    tt.set_state(psi)
    tt.time = t0
    got = tt.dipole_moments()
    tt.close()
    g = grid_of(N, dr, L, st, ghost=ghost, gauge=1 if gauge == "velocity" else 0)
    want = oracle.dipole_moments(g, psi, t0, PULSE)
    tol = 1e-12 * _scales(psi, dr, N, oracle.field(PULSE, t0))
    assert np.all(np.abs(got - want) <= tol), (got, want, tol)


def test_dipole_moments_at_scale_and_table_potential():
    C = W.SCALE
    psi = W.smooth_state(C.N, C.dr, C.lmax, seed=31, lmax_populated=20)
    t0 = 0.37 * C.duration
    pulse = oracle.Pulse(E0=C.E0, omega=C.omega, ncycles=C.ncycles)
    tt = make(C.N, C.dr, C.lmax, C.stencil, pulse=pulse)
    tt.set_state(psi)
    tt.time = t0
    got = tt.dipole_moments()
    tt.close()
    want = oracle.dipole_moments(grid_of(C.N, C.dr, C.lmax, C.stencil), psi, t0, pulse)
    assert np.all(np.abs(got - want) <= 1e-12 * _scales(psi, C.dr, C.N, oracle.field(pulse, t0))), (got, want)
    # a tabulated potential has no acceleration form
    N, dr, L = 300, 0.1, 4
    r = W.radial_grid(N, dr)
    v = -1.0 / r - 0.5 * np.exp(-r) / r
    x = W.random_state(N, L, seed=3)
    tt = make(N, dr, L, 5, vtable=v, pulse=PULSE)
    tt.set_state(x)
    tt.time = 70.0
    got = tt.dipole_moments()
    tt.close()
    want = oracle.dipole_moments(grid_of(N, dr, L, 5, vtable=v), x, 70.0, PULSE)
    assert math.isnan(got[2]) and math.isnan(want[2])
    assert np.all(np.abs(got[:2] - want[:2]) <= 1e-12 * _scales(x, dr, N, 0.0)[:2])


@pytest.mark.parametrize("method,order,dt,prec", [("lanczos", 12, 0.05, "fp64"), ("taylor", 8, 0.005, "fp64"),
                                                  ("rk4", 4, 0.005, "fp64"), ("lanczos", 12, 0.05, "mixed")])
def test_dipole_series_along_a_run(method, order, dt, prec):
    """The series recorded after every step equals the oracle's moments of the
    oracle's state after that step (capacity 6 of 8 steps: the last two are
    not recorded)."""
    N, dr, L, st = 500, 0.2, 4, 3
    psi = W.smooth_state(N, dr, L, seed=7)
    t0 = 40.0
    tt = make(N, dr, L, st, pulse=PULSE)
    tt.set_options(precision=prec)
    tt.set_state(psi)
    tt.time = t0
    tt.record_dipole(6)
    tt.propagate(method, order, dt, 8)
    ser = tt.dipole_series()
    tt.close()
    assert ser.shape == (6, 4)
    g = grid_of(N, dr, L, st)
    x = psi
    tol_rel = 1e-10 if prec == "fp64" else 1e-6
    for n in range(6):
        x, _ = oracle.propagate(g, x, method, order, dt, 1, t0=t0 + n * dt, pulse=PULSE)
        t = t0 + (n + 1) * dt
        want = oracle.dipole_moments(g, x, t, PULSE)
        assert abs(ser[n, 0] - t) <= 1e-12
        tol = tol_rel * _scales(x, dr, N, oracle.field(PULSE, t))
        assert np.all(np.abs(ser[n, 1:] - want) <= tol), (n, ser[n], want, tol)


def _oracle_flux_run(g, psi, method, order, dt, n, t0, r_b, ct, pulse, mask=None):
    tot, per = oracle.flux(g, psi, r_b, ct, t=t0, pulse=pulse)
    y, pad = 0.0, np.zeros(len(ct))
    x = psi
    for i in range(n):
        x, _ = oracle.propagate(g, x, method, order, dt, 1, t0=t0 + i * dt, pulse=pulse, mask=mask)
        t1, p1 = oracle.flux(g, x, r_b, ct, t=t0 + (i + 1) * dt, pulse=pulse)
        y += 0.5 * dt * (tot + t1)
        pad += 0.5 * dt * (per + p1)
        tot, per = t1, p1
    return tot, per, y, pad


@pytest.mark.parametrize("gauge,st", [("length", 5), ("velocity", 5), ("length", 3)])
def test_flux_and_pad_along_a_run(gauge, st):
    """An outgoing packet crossing r_b = 12 in a field: flux, densities at 19
    angles and their trapezoid time integrals over 100 Lanczos-12 steps at a
    step where the propagator converges (rho(H) dt ~ 6)."""
    N, dr, L = 400, 0.1, 6
    r = dr * np.arange(1, N + 1)
    rng = np.random.default_rng(4)
    c = rng.normal(size=L + 1) + 1j * rng.normal(size=L + 1)
    c[L - 1:] = 0
    psi = c[:, None] * np.exp(-(r - 11.0) ** 2 / 4.5 + 1j * r)[None, :]
    psi /= math.sqrt(dr * np.vdot(psi, psi).real)
    ct = np.cos(np.linspace(0.0, np.pi, 19))
    t0, dt, n = 30.0, 0.005, 100
    tt = make(N, dr, L, st, pulse=PULSE, gauge=gauge)
    tt.set_state(psi)
    tt.time = t0
    tt.flux_setup(12.0, ct)
    f0 = tt.flux()
    tt.propagate("lanczos", 12, dt, n)
    got = tt.flux()
    tt.close()
    g = grid_of(N, dr, L, st, gauge=1 if gauge == "velocity" else 0)
    w0, _ = oracle.flux(g, psi, 12.0, ct, t=t0, pulse=PULSE)
    # bounds: |f| |D1 f| ~ |f|^2 / dr at r_b, times (L+1) terms (x Y^2 ~ (2L+1)/(4 pi) for densities)
    b = float(np.sum(np.abs(psi[:, 119]) ** 2)) / dr + 1.0
    bd = b * (2 * L + 1) / (4 * np.pi)
    assert f0["yield"] == 0.0 and np.all(f0["pad"] == 0.0)
    assert abs(f0["flux"] - w0) <= 1e-12 * b
    tot, per, y, pad = _oracle_flux_run(g, psi, "lanczos", 12, dt, n, t0, 12.0, ct, PULSE)
    # the states themselves differ by ~1e-12 relative after 100 steps
    assert abs(got["flux"] - tot) <= 1e-10 * b, (got["flux"], tot)
    assert np.all(np.abs(got["density"] - per) <= 1e-10 * bd)
    assert abs(got["yield"] - y) <= 1e-10 * b * n * dt, (got["yield"], y)
    assert np.all(np.abs(got["pad"] - pad) <= 1e-10 * bd * n * dt)
    assert y > 0.02, "the packet must cross r_b"


def test_flux_at_scale_mixed_and_fp64():
    """At-scale grid, r_b = 10 a.u. and 180 angles, 4 Lanczos-12 steps at a
    converging dt (rho(H) dt ~ 4): FP64 against the oracle, mixed within 1e-6
    of FP64 (relative to the flux scale)."""
    C = W.SCALE
    psi = W.smooth_state(C.N, C.dr, C.lmax, seed=31, lmax_populated=20)
    pulse = oracle.Pulse(E0=C.E0, omega=C.omega, ncycles=C.ncycles)
    ct = np.cos((np.arange(180) + 0.5) * np.pi / 180)
    t0, dt, n = 0.37 * C.duration, 5e-6, 4
    res = {}
    for prec in ("fp64", "mixed"):
        tt = make(C.N, C.dr, C.lmax, C.stencil, pulse=pulse, absorber_r=C.R - C.absorber_width)
        tt.set_options(absorber=True, absorber_r=C.R - C.absorber_width, r_b=10.0, precision=prec)
        tt.set_state(psi)
        tt.time = t0
        tt.flux_setup(10.0, ct)
        tt.propagate("lanczos", 12, dt, n)
        res[prec] = tt.flux()
        tt.close()
    g = grid_of(C.N, C.dr, C.lmax, C.stencil)
    tot, per, y, pad = _oracle_flux_run(g, psi, "lanczos", 12, dt, n, t0, 10.0, ct, pulse,
                                        mask=oracle.Mask(C.R - C.absorber_width))
    b = float(np.sum(np.abs(psi[:, 199]) ** 2)) / C.dr + 1e-3
    bd = b * (2 * C.lmax + 1) / (4 * np.pi)
    f = res["fp64"]
    assert abs(f["flux"] - tot) <= 1e-11 * b and np.all(np.abs(f["density"] - per) <= 1e-11 * bd)
    assert abs(f["yield"] - y) <= 1e-11 * b * n * dt and np.all(np.abs(f["pad"] - pad) <= 1e-11 * bd * n * dt)
    m = res["mixed"]
    assert abs(m["flux"] - f["flux"]) <= 1e-6 * b and np.all(np.abs(m["density"] - f["density"]) <= 1e-6 * bd)


def test_flux_and_series_arguments():
    from paper_1308_1856_gb300 import TDSEError, _binding as C
    N, dr, L = 100, 0.1, 3
    tt = make(N, dr, L, 5, pulse=PULSE)
    tt.set_state(W.random_state(N, L, seed=1))
    with pytest.raises(TDSEError) as e:
        tt.flux()                                   # not set up
    assert e.value.code == C.TDSE_ERR_ARG
    for bad in (lambda: tt.flux_setup(50.0), lambda: tt.flux_setup(5.0, [0.5, 1.5]),
                lambda: tt.flux_setup(float("inf")), lambda: tt.record_dipole(-1)):
        with pytest.raises(TDSEError) as e:
            bad()
        assert e.value.code == C.TDSE_ERR_ARG
    tt.flux_setup(5.0, [1.0, 0.0, -1.0])
    tt.propagate("lanczos", 8, 0.01, 2)
    assert tt.flux()["density"].shape == (3,)
    tt.flux_setup(0.0)                              # off
    with pytest.raises(TDSEError):
        tt.flux()
    tt.record_dipole(3)
    tt.propagate("lanczos", 8, 0.01, 2)
    assert tt.dipole_series().shape == (2, 4)
    tt.propagate_rk("dormand_prince", 0.001, 2)    # the RK pairs record too; capacity 3 stops the series
    s = tt.dipole_series()
    assert s.shape == (3, 4) and np.all(np.diff(s[:, 0]) > 0)
    tt.record_dipole(0)
    assert tt.dipole_series().shape == (0, 4)
    # imaginary time records nothing
    tt.record_dipole(4)
    tt.propagate_imag("lanczos", 8, 0.1, 2)
    assert tt.dipole_series().shape == (0, 4)
    tt.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_record_rows_equal_the_separate_calls(prec):
    """The per-step record (every 2nd step, capacity 4 of 5 recordable steps)
    of one 10-step call: each row equals what tdse_observables,
    tdse_dipole_moments and tdse_flux_read return after the same steps taken
    two per call (the step times then accumulate differently, so the states
    agree to rounding, 1e-12 relative, not bitwise)."""
    N, dr, L = 400, 0.1, 6
    psi = W.smooth_state(N, dr, L, seed=9)
    ct = np.cos(np.linspace(0.0, np.pi, 5))

    def fresh():
        t = make(N, dr, L, 5, pulse=PULSE)
        t.set_options(precision=prec, r_b=10.0)
        t.set_state(psi)
        t.time = 30.0
        t.flux_setup(12.0, ct)
        return t
    a = fresh()
    a.record(2, 4)
    a.propagate("lanczos", 12, 0.01, 10)
    rec = a.records()
    a.close()
    assert len(rec["t"]) == 4
    b = fresh()

    def close(x, y):
        return abs(x - y) <= 1e-12 * max(1.0, abs(y))
    for n in range(4):
        b.propagate("lanczos", 12, 0.01, 2)
        ob, dm, fl = b.observables(), b.dipole_moments(), b.flux()
        assert abs(rec["t"][n] - (30.0 + 2 * (n + 1) * 0.01)) <= 1e-12
        for key in ("norm", "dipole", "yield", "p_ground"):
            assert close(rec[key][n], ob[key]), key
        assert np.all(np.abs(rec["l_pop"][n] - ob["l_pop"]) <= 1e-12)
        assert close(rec["z"][n], dm[0]) and close(rec["zdot"][n], dm[1]) and close(rec["zddot"][n], dm[2])
        assert close(rec["flux"][n], fl["flux"]) and close(rec["flux_yield"][n], fl["yield"])
    b.close()
    # without a flux setup the flux columns are NaN; capacity 0 turns recording off
    c = make(N, dr, L, 5, pulse=PULSE)
    c.record(1, 3)
    c.propagate("rk4", 4, 0.002, 2)
    r = c.records()
    assert len(r["t"]) == 2 and np.all(np.isnan(r["flux"]))
    c.record(1, 0)
    c.propagate("rk4", 4, 0.002, 2)
    assert len(c.records()["t"]) == 0
    c.close()
