"""The batched Sec. 4 observables after every step against the oracle: the
dipole series (<z>, <zdot>, <zddot> of every instance) and the flux through
each instance's r_b with its angular densities and their time integrals.

Dipole series.

Two checks per entry.  (1) The kernel alone: entry n equals the oracle's
moments of the GPU's own state after step n (read back step by step), to
1e-12 of the moments' absolute-term bounds (norm r_max, norm / dr,
norm / dr^2 + |E| norm), the rounding of two summation orders.  (2) Along the
run: entry n equals the oracle's moments of the oracle's own propagation to
the propagator's tolerance (1e-10 FP64, 1e-6 mixed) of the same bounds.
An instance's entries are bitwise the same alone and in the mix, and whether
its steps run one call at a time (uncaptured) or in one call (a replayed
step graph)."""
import numpy as np
import pytest

import oracle
import tdse_workloads as W

pytestmark = pytest.mark.gpu

SPECS = [
    dict(N=300, dr=0.2, lmax=4, krylov=12, dt=0.02, E0=0.0534, omega=0.057, ncycles=2),
    dict(N=517, dr=0.1, lmax=9, krylov=8, dt=5e-4, E0=0.03, omega=0.11, ncycles=3, absorber_r=40.0),
    dict(N=129, dr=0.25, lmax=2, krylov=5, dt=0.02, E0=0.08, omega=0.2, ncycles=2, cep=0.4,
         shape="sin2_a"),
    dict(N=33, dr=0.3, lmax=0, krylov=1, dt=0.05),
]
VELOCITY = [
    dict(N=500, dr=0.2, lmax=4, krylov=12, dt=0.02, E0=0.0534, omega=0.057, ncycles=2, gauge="velocity"),
    dict(N=1000, dr=0.1, lmax=15, krylov=16, dt=4e-4, E0=0.05, omega=0.057, ncycles=4, absorber_r=80.0,
         gauge="velocity", shape="sin2_a"),
]


def _grid(s, stencil=5):
    return oracle.Grid(N=s["N"], h=s["dr"], L=s["lmax"], stencil=stencil, Z=s.get("Z", 1.0),
                       gauge=1 if s.get("gauge") == "velocity" else 0)


def _pulse(s):
    return oracle.Pulse(E0=s.get("E0", 0.0), omega=s.get("omega", 0.057), ncycles=s.get("ncycles", 2.0),
                        cep=s.get("cep", 0.0), shape=1 if s.get("shape") == "sin2_a" else 0)


def _scales(psi, s, t):
    dr, N = s["dr"], s["N"]
    norm = dr * float(np.sum(np.abs(psi) ** 2))
    E = oracle.field(_pulse(s), t)
    return np.array([norm * N * dr, norm / dr, norm / dr ** 2 + abs(E) * norm])


def _per_step(specs, precision, stencil, nsteps, cap):
    """Series and the state after every step, one step per call."""
    from paper_1308_1856_gb300 import Batch
    b = Batch(specs, precision=precision, stencil=stencil)
    b.record_dipole(cap)
    states = [[] for _ in specs]
    for _ in range(nsteps):
        b.propagate(1)
        for i in range(len(specs)):
            states[i].append(b.get_state(i))
    ser = [b.dipole_series(i) for i in range(len(specs))]
    b.close()
    return ser, states


@pytest.mark.parametrize("precision,stencil,specs", [("fp64", 5, SPECS + VELOCITY), ("fp64", 3, SPECS),
                                                     ("mixed", 5, SPECS), ("mixed", 3, SPECS)])
def test_batch_dipole_series_kernel_vs_oracle(precision, stencil, specs):
    nsteps, cap = 5, 4
    ser, states = _per_step(specs, precision, stencil, nsteps, cap)
    for i, s in enumerate(specs):
        assert ser[i].shape == (cap, 4), (i, ser[i].shape)
        g, p = _grid(s, stencil), _pulse(s)
        for n in range(cap):
            t = (n + 1) * s["dt"]
            assert abs(ser[i][n, 0] - t) <= 1e-15 * max(1.0, t)
            want = oracle.dipole_moments(g, states[i][n], t, p)
            tol = 1e-12 * _scales(states[i][n], s, t)
            assert np.all(np.abs(ser[i][n, 1:] - want) <= tol), (i, n, ser[i][n], want, tol)


@pytest.mark.parametrize("precision,tol_rel", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_batch_dipole_series_along_the_run(precision, tol_rel):
    from paper_1308_1856_gb300 import Batch
    specs = SPECS + (VELOCITY if precision == "fp64" else [])
    nsteps = 12
    b = Batch(specs, precision=precision)
    b.record_dipole(nsteps)
    b.propagate(nsteps)
    for i, s in enumerate(specs):
        ser = b.dipole_series(i)
        assert ser.shape == (nsteps, 4)
        g, p = _grid(s), _pulse(s)
        mask = oracle.Mask(s["absorber_r"]) if "absorber_r" in s else None
        x = W.hydrogen_1s(s["N"], s["dr"], s["lmax"])
        for n in range(nsteps):
            x, _ = oracle.propagate(g, x, "lanczos", s["krylov"], s["dt"], 1, t0=n * s["dt"], pulse=p, mask=mask)
            t = (n + 1) * s["dt"]
            want = oracle.dipole_moments(g, x, t, p)
            tol = tol_rel * _scales(x, s, t)
            assert np.all(np.abs(ser[n, 1:] - want) <= tol), (i, n, ser[n], want, tol)
    b.close()


def test_batch_dipole_series_is_independent_of_mix_and_split():
    from paper_1308_1856_gb300 import Batch
    specs = SPECS + VELOCITY
    nsteps = 7
    ser1, _ = _per_step(specs, "fp64", 5, nsteps, nsteps)
    b = Batch(specs, precision="fp64")
    b.record_dipole(nsteps)
    b.propagate(nsteps)                  # one segment: a replayed step graph
    assert b.graph_steps >= nsteps
    for i in range(len(specs)):
        assert np.array_equal(b.dipole_series(i), ser1[i]), i
    b.close()
    alone = Batch([specs[1]], precision="fp64")
    alone.record_dipole(nsteps)
    alone.propagate(3)
    alone.propagate(nsteps - 3)
    assert np.array_equal(alone.dipole_series(0), ser1[1])
    alone.close()


def test_batch_dipole_series_capacity_reset_and_time():
    from paper_1308_1856_gb300 import Batch
    s = SPECS[0]
    b = Batch([s, SPECS[2]], precision="fp64")
    b.propagate(2)
    b.record_dipole(3)
    assert b.dipole_series(0).shape == (0, 4)
    b.propagate(5)                       # entries for steps 3, 4, 5 only
    ser = b.dipole_series(0)
    assert ser.shape == (3, 4)
    assert np.allclose(ser[:, 0], [3 * s["dt"], 4 * s["dt"], 5 * s["dt"]], rtol=0, atol=1e-14)
    b.record_dipole(2)                   # discards the record
    assert b.dipole_series(1).shape == (0, 4)
    t0 = 33.0
    b.set_time(0, t0)
    b.propagate(1)
    got = b.dipole_series(0)
    assert got.shape == (1, 4) and abs(got[0, 0] - (t0 + s["dt"])) <= 1e-13
    want = oracle.dipole_moments(_grid(s), b.get_state(0), t0 + s["dt"], _pulse(s))
    assert np.all(np.abs(got[0, 1:] - want) <= 1e-12 * _scales(b.get_state(0), s, t0 + s["dt"]))
    n0 = b.launches
    b.propagate(1)
    per_step_on = b.launches - n0
    b.record_dipole(0)                   # off: no entries, one launch fewer per step
    n0 = b.launches
    b.propagate(1)
    assert b.launches - n0 == per_step_on - 1
    assert b.dipole_series(0).shape == (0, 4)
    with pytest.raises(Exception):
        b.record_dipole(-1)
    b.close()


# ---- the flux through r = r_b (Eqs. (flux), (pad), (yield)) ------------------
# Outgoing packets that cross each instance's r_b during the run.
FLUX_SPECS = [
    dict(N=400, dr=0.1, lmax=6, krylov=12, dt=0.005, E0=0.0534, omega=0.057, ncycles=2, r_b=12.0),
    dict(N=300, dr=0.2, lmax=4, krylov=12, dt=0.02, E0=0.08, omega=0.2, ncycles=2, cep=0.4, r_b=30.0,
         shape="sin2_a"),
    dict(N=129, dr=0.25, lmax=2, krylov=8, dt=0.01, r_b=20.05),
]
FLUX_VELOCITY = [
    dict(N=400, dr=0.1, lmax=6, krylov=12, dt=0.005, E0=0.0534, omega=0.057, ncycles=2, r_b=12.0,
         gauge="velocity"),
]
CT = np.cos(np.linspace(0.0, np.pi, 19))


def _packet(s, seed):
    N, dr, L = s["N"], s["dr"], s["lmax"]
    r = dr * np.arange(1, N + 1)
    rng = np.random.default_rng(seed)
    c = rng.normal(size=L + 1) + 1j * rng.normal(size=L + 1)
    r0 = s["r_b"] - 1.0
    psi = c[:, None] * np.exp(-(r - r0) ** 2 / 4.5 + 1j * r)[None, :]
    return psi / np.sqrt(dr * np.vdot(psi, psi).real)


def _flux_bounds(psi, s):
    ib = int(np.ceil(s["r_b"] / s["dr"] - 1.5))
    b = float(np.sum(np.abs(psi[:, ib]) ** 2)) / s["dr"] + 1e-3
    return b, b * (2 * s["lmax"] + 1) / (4 * np.pi)


@pytest.mark.parametrize("precision,stencil,specs", [("fp64", 5, FLUX_SPECS + FLUX_VELOCITY), ("fp64", 3, FLUX_SPECS),
                                                     ("mixed", 5, FLUX_SPECS)])
def test_batch_flux_kernel_vs_oracle(precision, stencil, specs):
    """Flux, densities and their integrals against the oracle's flux of the
    GPU's own states after every step, integrated by the trapezoid rule here:
    1e-12 of the absolute-term bound b = sum_l |f_l(r_b)|^2 / dr (x (2L+1)/(4 pi)
    for the densities; x the elapsed time for the integrals)."""
    from paper_1308_1856_gb300 import Batch
    n = 6
    b = Batch(specs, precision=precision, stencil=stencil)
    psis = [_packet(s, 11 + i) for i, s in enumerate(specs)]
    t0s = [20.0 + 3 * i for i in range(len(specs))]
    for i in range(len(specs)):
        b.set_state(i, psis[i])
        b.set_time(i, t0s[i])
    b.flux_setup(CT)
    f0 = [b.flux(i) for i in range(len(specs))]
    states = [[p] for p in psis]
    for _ in range(n):
        b.propagate(1)
        for i in range(len(specs)):
            states[i].append(b.get_state(i))
    for i, s in enumerate(specs):
        g, p = _grid(s, stencil), _pulse(s)
        bb, bd = _flux_bounds(psis[i], s)
        w0, wd0 = oracle.flux(g, psis[i], s["r_b"], CT, t=t0s[i], pulse=p)
        assert f0[i]["yield"] == 0.0 and np.all(f0[i]["pad"] == 0.0)
        assert abs(f0[i]["flux"] - w0) <= 1e-12 * bb and np.all(np.abs(f0[i]["density"] - wd0) <= 1e-12 * bd)
        y, pad, tot, per = 0.0, np.zeros(len(CT)), w0, wd0
        for k in range(n):
            t1, p1 = oracle.flux(g, states[i][k + 1], s["r_b"], CT, t=t0s[i] + (k + 1) * s["dt"], pulse=p)
            y += 0.5 * s["dt"] * (tot + t1)
            pad += 0.5 * s["dt"] * (per + p1)
            tot, per = t1, p1
        got = b.flux(i)
        T = n * s["dt"]
        assert abs(got["flux"] - tot) <= 1e-12 * bb, (i, got["flux"], tot)
        assert np.all(np.abs(got["density"] - per) <= 1e-12 * bd), i
        assert abs(got["yield"] - y) <= 1e-12 * bb * T, (i, got["yield"], y)
        assert np.all(np.abs(got["pad"] - pad) <= 1e-12 * bd * T), i
    b.close()


def test_batch_flux_along_the_run_and_alone():
    """100 Lanczos-12 steps of packets crossing r_b against the oracle's own
    propagation (1e-10 of the bounds, as the single-instance flux test); an
    instance's integrals are bitwise the same alone and in the batch."""
    from paper_1308_1856_gb300 import Batch
    specs = FLUX_SPECS[:1] + FLUX_VELOCITY
    n = 100
    b = Batch(specs, precision="fp64")
    psis = [_packet(s, 21 + i) for i, s in enumerate(specs)]
    for i in range(len(specs)):
        b.set_state(i, psis[i])
        b.set_time(i, 30.0)
    b.flux_setup(CT)
    b.propagate(n)
    got = [b.flux(i) for i in range(len(specs))]
    b.close()
    for i, s in enumerate(specs):
        g, p = _grid(s), _pulse(s)
        bb, bd = _flux_bounds(psis[i], s)
        tot, per = oracle.flux(g, psis[i], s["r_b"], CT, t=30.0, pulse=p)
        y, pad, x = 0.0, np.zeros(len(CT)), psis[i]
        for k in range(n):
            x, _ = oracle.propagate(g, x, "lanczos", s["krylov"], s["dt"], 1, t0=30.0 + k * s["dt"], pulse=p)
            t1, p1 = oracle.flux(g, x, s["r_b"], CT, t=30.0 + (k + 1) * s["dt"], pulse=p)
            y += 0.5 * s["dt"] * (tot + t1)
            pad += 0.5 * s["dt"] * (per + p1)
            tot, per = t1, p1
        T = n * s["dt"]
        assert abs(got[i]["flux"] - tot) <= 1e-10 * bb, (i, got[i]["flux"], tot)
        assert np.all(np.abs(got[i]["density"] - per) <= 1e-10 * bd)
        assert abs(got[i]["yield"] - y) <= 1e-10 * bb * T, (i, got[i]["yield"], y)
        assert np.all(np.abs(got[i]["pad"] - pad) <= 1e-10 * bd * T)
        assert y > 0.02, "the packet must cross r_b"
    alone = Batch([specs[1]], precision="fp64")
    alone.set_state(0, psis[1])
    alone.set_time(0, 30.0)
    alone.flux_setup(CT)
    alone.propagate(40)
    alone.propagate(n - 40)
    a = alone.flux(0)
    alone.close()
    for k in ("flux", "yield", "density", "pad"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(got[1][k])), k


def test_batch_flux_arguments():
    from paper_1308_1856_gb300 import Batch, TDSEError, _binding as C
    b = Batch(FLUX_SPECS, precision="fp64")
    with pytest.raises(TDSEError) as e:
        b.flux(0)                                    # not set up
    assert e.value.code == C.TDSE_ERR_ARG
    with pytest.raises(TDSEError):
        b.flux_setup([0.5, 1.5])                     # outside [-1, 1]
    b.flux_setup(None)                               # the total only
    b.propagate(2)
    f = b.flux(0)
    assert f["density"].shape == (0,) and np.isfinite(f["flux"])
    b.flux_setup(enable=False)
    b.propagate(1)
    with pytest.raises(TDSEError):
        b.flux(0)
    b.close()
    far = dict(FLUX_SPECS[2], r_b=1000.0)            # r_b beyond the box
    b = Batch([far], precision="fp64")
    with pytest.raises(TDSEError):
        b.flux_setup(CT)
    b.close()
