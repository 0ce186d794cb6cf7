"""Checkpoint and resume: a run interrupted by a checkpoint, loaded into a
fresh handle and continued, gives bitwise the state (and the flux integrals)
of the uninterrupted run, for every propagator, both precisions and both
gauges; the argument checks."""
import numpy as np
import pytest

import oracle
import tdse_workloads as W
from gpu_helpers import make

pytestmark = pytest.mark.gpu

PULSE = oracle.Pulse(E0=0.0534, omega=0.057, ncycles=2)
N, DR, L = 517, 0.2, 7


def _handle(prec, gauge, flux):
    t = make(N, DR, L, 5, pulse=PULSE, gauge=gauge, absorber_r=80.0)
    t.set_options(absorber=True, absorber_r=80.0, r_b=10.0, precision=prec, gauge=gauge)
    if flux:
        t.flux_setup(12.0, np.cos(np.linspace(0.0, np.pi, 7)))
    return t


def _go(t, method, order, dt, n):
    if method in ("taylor", "rk4", "lanczos"):
        t.propagate(method, order, dt, n)
    else:
        t.propagate_rk(method, dt, n)


@pytest.mark.parametrize("prec,gauge", [("fp64", "length"), ("fp64", "velocity"), ("mixed", "length")])
@pytest.mark.parametrize("method,order,dt", [("lanczos", 12, 0.05), ("taylor", 8, 0.005), ("rk4", 4, 0.005),
                                             ("dormand_prince", 0, 0.004)])
def test_resume_is_bitwise(prec, gauge, method, order, dt):
    if prec == "mixed" and method == "dormand_prince":
        pytest.skip("the embedded pairs run in FP64")
    psi = W.smooth_state(N, DR, L, seed=3)
    flux = prec == "fp64"
    a = _handle(prec, gauge, flux)
    a.set_state(psi)
    a.time = 40.0
    if flux:
        a.flux_setup(12.0, np.cos(np.linspace(0.0, np.pi, 7)))
    _go(a, method, order, dt, 6)
    blob = a.checkpoint()
    _go(a, method, order, dt, 6)
    want, want_t = a.get_state(), a.time
    want_f = a.flux() if flux else None
    a.close()
    b = _handle(prec, gauge, flux)
    b.restore(blob)
    assert b.time == 40.0 + 6 * dt or abs(b.time - (40.0 + 6 * dt)) <= 1e-12
    _go(b, method, order, dt, 6)
    got = b.get_state()
    assert np.array_equal(got, want) and b.time == want_t
    if flux:
        f = b.flux()
        assert f["flux"] == want_f["flux"] and f["yield"] == want_f["yield"]
        assert np.array_equal(f["pad"], want_f["pad"]) and np.array_equal(f["density"], want_f["density"])
    b.close()


def test_checkpoint_arguments():
    from paper_1308_1856_gb300 import TDSEError, _binding as C
    a = _handle("fp64", "length", False)
    blob = a.checkpoint()
    with pytest.raises(TDSEError):
        a.restore(blob[:100])                        # too short
    with pytest.raises(TDSEError):
        a.restore(b"X" * len(blob))                  # not a checkpoint
    other = make(N + 1, DR, L, 5)
    with pytest.raises(TDSEError):
        other.restore(blob)                          # another grid
    other.close()
    f = _handle("fp64", "length", True)
    with pytest.raises(TDSEError):
        f.restore(blob)                              # the handle has a flux setup, the checkpoint none
    f.close()
    # into the other precision: allowed, the norm is recomputed
    m = _handle("mixed", "length", False)
    m.restore(blob)
    m.propagate("lanczos", 12, 0.05, 2)
    m.close()
    assert C.tdse_checkpoint_bytes(None) == 0
    a.close()
