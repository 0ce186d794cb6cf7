"""The batched dipole series (Sec. 4: <z>, <zdot>, <zddot> after every step of
every instance) against the oracle.

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
