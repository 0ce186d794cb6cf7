"""The velocity gauge (Sec. 2) on the GPU against the oracle: the operator,
single steps of every method, a whole pulse, gauge invariance against the
GPU's own length gauge, and the argument checks."""
import numpy as np
import pytest

import oracle
import tdse_workloads as W
from gpu_helpers import apply_h_gpu, grid_of, make, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,dr,L,st", [(7, 0.3, 2, 3), (33, 0.2, 5, 5), (257, 0.1, 6, 5),
                                       (1000, 0.05, 9, 5), (517, 0.2, 13, 3)])
def test_velocity_apply_h(N, dr, L, st):
    g = grid_of(N, dr, L, st, gauge=1)
    t = make(N, dr, L, st, gauge="velocity")
    # Both sides round each term once but in different orders (the GPU's
    # diagonal c0 + l(l+1)/(2r^2) + V is one table entry), so the difference is
    # a few unit roundoffs of the largest terms: |c0| |x| ~ 1.25/dr^2 |x|
    # against |Hx|.  Random states have no cancellation (|Hx| ~ |c0| |x|);
    # smooth ones cancel down to |Hx| ~ |x|, i.e. up to ~1e3 at dr = 0.05.
    for x, tol in ((W.smooth_state(N, dr, L, seed=3), 1e-12), (W.random_state(N, L, seed=4), 1e-13)):
        for A in (0.0, 1.7, -31.0):
            got = apply_h_gpu(t, A, x)
            want = oracle.apply_H(g, A, x)
            assert rel_l2(got, want) <= tol, (A, tol, rel_l2(got, want))
    t.close()


@pytest.mark.parametrize("method,order,dt", [("taylor", 8, 0.01), ("rk4", 4, 0.005), ("lanczos", 12, 0.05),
                                             ("lanczos", 1, 0.01)])
@pytest.mark.parametrize("geom", [(500, 0.2, 4, 3), (1000, 0.05, 9, 5)])
def test_velocity_one_step(method, order, dt, geom):
    N, dr, L, st = geom
    if method != "lanczos":
        dt = min(dt, 2.5 / (2.7 / dr ** 2 + L * (L + 1) / (2 * dr ** 2)))   # stable explicit step
    pulse = oracle.Pulse(E0=0.0534, omega=0.057, ncycles=2)
    psi = W.smooth_state(N, dr, L, seed=5)
    t = make(N, dr, L, st, pulse=pulse, gauge="velocity")
    t.set_state(psi)
    t.time = 70.0
    t.propagate(method, order, dt, 1)
    got = t.get_state()
    t.close()
    want, _ = oracle.propagate(grid_of(N, dr, L, st, gauge=1), psi, method, order, dt, 1, t0=70.0, pulse=pulse)
    assert rel_l2(got, want) <= 1e-12, rel_l2(got, want)


def test_velocity_full_pulse_and_gauge_invariance():
    """A one-cycle pulse on a small grid from the imaginary-time ground state
    (5027 Lanczos-10 steps).  Over this many steps an FP64 result depends on
    the order of its sums: the FP64 oracle itself drifts ~1.5e-11 from its
    long-double build (the floor).  So, as for every rounding-limited run
    (tests/test_gpu_floor.py), the GPU state is held to 10 x max(floor, 1e-15)
    against the long-double oracle, and the populations and p_ground to 1e-10
    of the long-double oracle's.  After the pulse the velocity-gauge
    populations match the GPU's length-gauge run to the step error."""
    N, dr, L = 300, 0.1, 6
    pulse = oracle.Pulse(E0=0.05, omega=0.25, ncycles=1)
    dt = 0.005
    n = int(np.ceil(pulse.duration() / dt))
    # the start state comes from the oracle (no oracle input comes from the GPU)
    psi0, _ = oracle.propagate_imag(grid_of(N, dr, L, 5), W.hydrogen_1s(N, dr, L), "lanczos", 12, 0.5, 40)
    out = {}
    for gauge in ("length", "velocity"):
        t = make(N, dr, L, 5, pulse=pulse, gauge=gauge)
        t.set_state(psi0)
        t.set_reference(psi0[0])
        t.propagate("lanczos", 10, dt, n)
        out[gauge] = (t.get_state(), t.observables())
        t.close()
    got, ob = out["velocity"]
    g = grid_of(N, dr, L, 5, gauge=1)
    f64, _ = oracle.propagate(g, psi0, "lanczos", 10, dt, n, pulse=pulse)
    fld, _ = oracle.propagate(g, psi0, "lanczos", 10, dt, n, pulse=pulse, precision="fld")
    floor = rel_l2(f64, fld)
    gpu = rel_l2(got, fld)
    print(f"velocity full pulse: floor={floor:.3e} gpu_vs_long_double={gpu:.3e} gpu_vs_f64={rel_l2(got, f64):.3e}")
    assert gpu <= 10 * max(floor, 1e-15), (gpu, floor)
    ow = oracle.observables(g, fld, psi0[0], r_b=10.0, precision="fld")
    assert abs(ob["p_ground"] - ow["p_ground"]) <= 1e-10 and np.abs(ob["l_pop"] - ow["l_pop"]).max() <= 1e-10
    ol = out["length"][1]
    assert abs(ob["p_ground"] - ol["p_ground"]) <= 1e-4, (ob["p_ground"], ol["p_ground"])
    assert np.abs(ob["l_pop"] - ol["l_pop"]).max() <= 1e-4
    assert 1 - ol["p_ground"] >= 1e-3


def test_velocity_arguments():
    from paper_1308_1856_gb300 import TDSEError
    t = make(50, 0.2, 2, 5)
    with pytest.raises(TDSEError):
        t.set_options(gauge="velocity", ghost=1)
    with pytest.raises(TDSEError):
        t.set_options(gauge="velocity", ghost=1, precision="mixed")
    t.set_options(gauge="velocity", precision="mixed")
    t.set_options(gauge="velocity")
    t.close()


def _mixed_velocity(N, dr, L, st, pulse=None):
    t = make(N, dr, L, st, pulse=pulse, gauge="velocity")
    t.set_options(gauge="velocity", precision="mixed")
    return t


@pytest.mark.parametrize("N,dr,L,st", [(7, 0.3, 2, 3), (33, 0.2, 5, 5), (257, 0.1, 6, 5), (517, 0.2, 13, 3)])
def test_mixed_velocity_apply_h(N, dr, L, st):
    """Mixed precision in the velocity gauge: the FP32 operator, whose
    coupling takes the first derivatives of rows l -+ 1 from part-by-part
    differences like the Laplacian, stays within a few FP32 roundings of the
    FP64 oracle's (2e-6 relative, the bound of the length-gauge mixed operator)."""
    g = grid_of(N, dr, L, st, gauge=1)
    t = _mixed_velocity(N, dr, L, st)
    for x in (W.smooth_state(N, dr, L, seed=3), W.random_state(N, L, seed=4)):
        for A in (0.0, 1.7, -31.0):
            got = apply_h_gpu(t, A, x)
            want = oracle.apply_H(g, A, x)
            assert rel_l2(got, want) <= 2e-6, (A, rel_l2(got, want))
    t.close()


@pytest.mark.parametrize("method,order,dt", [("taylor", 8, 0.01), ("rk4", 4, 0.005), ("lanczos", 12, 0.05),
                                             ("lanczos", 1, 0.01)])
def test_mixed_velocity_one_step(method, order, dt):
    """One step of each method in mixed precision and the velocity gauge
    against the FP64 oracle: ~dt |H psi| times the operator's FP32 error, held
    to 1e-7 as in the length gauge."""
    N, dr, L, st = 500, 0.2, 4, 3
    if method != "lanczos":
        dt = min(dt, 2.5 / (2.7 / dr ** 2 + L * (L + 1) / (2 * dr ** 2)))   # stable explicit step
    pulse = oracle.Pulse(E0=0.0534, omega=0.057, ncycles=2)
    psi = W.smooth_state(N, dr, L, seed=5)
    t = _mixed_velocity(N, dr, L, st, pulse=pulse)
    t.set_state(psi)
    t.time = 70.0
    t.propagate(method, order, dt, 1)
    got = t.get_state()
    t.close()
    want, _ = oracle.propagate(grid_of(N, dr, L, st, gauge=1), psi, method, order, dt, 1, t0=70.0, pulse=pulse)
    assert rel_l2(got, want) <= 1e-7, rel_l2(got, want)


def test_mixed_velocity_many_steps_populations():
    """100 Lanczos-12 steps of the small configuration's grid in the velocity
    gauge: the l-populations above 1e-10 within 1e-6 relative of the FP64
    oracle, the norm within 1e-6 (the target of the mixed path)."""
    c = W.SMALL
    pulse = oracle.Pulse(E0=c.E0, omega=c.omega, ncycles=c.ncycles)
    psi0 = W.hydrogen_1s(c.N, c.dr, c.lmax)
    t = _mixed_velocity(c.N, c.dr, c.lmax, c.stencil, pulse=pulse)
    t.set_state(psi0)
    t.time = 50.0
    t.propagate("lanczos", 12, 0.05, 100)
    got = t.get_state()
    ob = t.observables()
    t.close()
    g = grid_of(c.N, c.dr, c.lmax, c.stencil, gauge=1)
    want, _ = oracle.propagate(g, psi0, "lanczos", 12, 0.05, 100, t0=50.0, pulse=pulse)
    ow = oracle.observables(g, want, psi0[0], r_b=10.0)
    big = ow["l_pop"] > 1e-10
    rel = np.abs(ob["l_pop"][big] - ow["l_pop"][big]) / ow["l_pop"][big]
    assert rel.max() <= 1e-6, rel
    assert abs(ob["norm"] - ow["norm"]) <= 1e-6
    assert rel_l2(got, want) <= 1e-6, rel_l2(got, want)


def test_sinea_pulse_field_and_vector_potential_match_the_oracle():
    """The host's E(t) and A(t) of the sin^2-on-A pulse ("SineA", Eq.
    (VecSinSinCosE)) equal the oracle's (independent code, both FP64 on the
    host) to rounding over the whole pulse and after it."""
    pulse = oracle.Pulse(E0=0.1688, omega=0.5512, ncycles=10, cep=0.3, shape=1)
    t = make(20, 0.2, 1, 5, pulse=pulse)
    T = pulse.duration()
    for s in np.linspace(-1.0, T + 3.0, 257):
        e, a = t.field(s), t.vector_potential(s)
        # the same formula in independent code: a few unit roundoffs of the carrier terms
        assert abs(e - oracle.field(pulse, s)) <= 1e-14, s
        assert abs(a - oracle.vecpot(pulse, s)) <= 1e-12 * max(1.0, abs(a)), s
    t.close()


@pytest.mark.parametrize("gauge", ["length", "velocity"])
@pytest.mark.parametrize("method,order,dt", [("lanczos", 12, 0.02), ("taylor", 8, 0.005), ("rk4", 4, 0.005)])
def test_sinea_steps_vs_oracle(gauge, method, order, dt):
    """Ten steps under the SineA pulse from mid-pulse on a ragged grid."""
    N, dr, L = 517, 0.2, 7
    pulse = oracle.Pulse(E0=0.1688, omega=0.5512, ncycles=4, shape=1)
    psi = W.smooth_state(N, dr, L, seed=11)
    t = make(N, dr, L, 5, pulse=pulse, gauge=gauge)
    t.set_state(psi)
    t.time = 0.4 * pulse.duration()
    t.propagate(method, order, dt, 10)
    got = t.get_state()
    t.close()
    g = grid_of(N, dr, L, 5, gauge=1 if gauge == "velocity" else 0)
    want, _ = oracle.propagate(g, psi, method, order, dt, 10, t0=0.4 * pulse.duration(), pulse=pulse)
    assert rel_l2(got, want) <= 1e-11, rel_l2(got, want)
