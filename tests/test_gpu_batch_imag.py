"""Imaginary time in the batch engine (Sec. 3): many grids relaxed at once by
Lanczos steps with exp(-T dtau), renormalised after each step, against
oracle.propagate_imag; the instances' pulses, gauges and absorbers play no
part, their times do not change, and an instance's result does not depend on
its batch.  Tolerances as the single-instance imaginary-time tests: states
1e-12 relative L2 over 5 steps at converging dtau, energies 1e-11 relative."""
import numpy as np
import pytest

import oracle
import tdse_workloads as W
from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

# dtau (the spec's dt) keeps rho(H) dtau within the Krylov dimension's reach
SPECS = [
    dict(N=300, dr=0.2, lmax=4, krylov=12, dt=0.005, E0=0.0534, omega=0.057, ncycles=2, absorber_r=30.0),
    dict(N=517, dr=0.1, lmax=7, krylov=12, dt=0.002, E0=0.03, omega=0.11, ncycles=3),
    dict(N=13, dr=0.25, lmax=0, krylov=12, dt=0.005),
    dict(N=129, dr=0.25, lmax=2, krylov=1, dt=0.05, E0=0.08, omega=0.2, ncycles=2, cep=0.4, shape="sin2_a"),
    dict(N=300, dr=0.2, lmax=3, krylov=8, dt=0.005, E0=0.0534, omega=0.057, ncycles=2, gauge="velocity",
         absorber_r=40.0),
    dict(N=200, dr=0.2, lmax=2, krylov=6, dt=0.005, Z=2.0),
]


def _grid(s):
    return oracle.Grid(N=s["N"], h=s["dr"], L=s["lmax"], stencil=5, Z=s.get("Z", 1.0))


def _smooth(s, seed):
    return W.smooth_state(s["N"], s["dr"], s["lmax"], seed=seed)


def test_batch_imag_matches_oracle():
    from paper_1308_1856_gb300 import Batch
    n = 5
    b = Batch(SPECS, precision="fp64")
    psis = [_smooth(s, 9 + i) for i, s in enumerate(SPECS)]
    for i, p in enumerate(psis):
        b.set_state(i, p)
        b.set_time(i, 17.0)
    e = b.propagate_imag(n)
    for i, s in enumerate(SPECS):
        want, e_orc = oracle.propagate_imag(_grid(s), psis[i], "lanczos", s["krylov"], s["dt"], n)
        got = b.get_state(i)
        assert rel_l2(got, want) <= 1e-12, (i, rel_l2(got, want))
        assert abs(e[i] - e_orc) <= 1e-11 * max(1.0, abs(e_orc)), (i, e[i], e_orc)
        assert b.time(i) == 17.0
        assert abs(b.observables(i)["norm"] - 1.0) <= 1e-13
    b.close()


def test_batch_imag_ground_states():
    """From the 1s state, 100 steps (dtau = 0.5; 0.1 for Z = 2) reach the grid ground states:
    the paper's ~ -0.47 a.u. at dr = 0.2 (5-point), and for Z = 2 at dr = 0.1
    exactly Z^2 times that (r -> Z r maps the Z = 2 grid onto the Z = 1 grid
    of twice the spacing, and H onto Z^2 H), each equal to the oracle's; one
    batch relaxes all of them."""
    from paper_1308_1856_gb300 import Batch
    specs = [dict(N=500, dr=0.2, lmax=0, krylov=12, dt=0.5),
             dict(N=500, dr=0.2, lmax=2, krylov=12, dt=0.5, E0=0.05, omega=0.057, ncycles=2),
             dict(N=400, dr=0.1, lmax=0, krylov=12, dt=0.1, Z=2.0)]
    b = Batch(specs, precision="fp64")
    e = b.propagate_imag(100)
    for i, s in enumerate(specs):
        want, e_orc = oracle.propagate_imag(_grid(s), W.hydrogen_1s(s["N"], s["dr"], s["lmax"]), "lanczos",
                                            s["krylov"], s["dt"], 100)
        assert abs(e[i] - e_orc) <= 1e-12 * max(1.0, abs(e_orc)), (i, e[i], e_orc)
        assert rel_l2(b.get_state(i), want) <= 1e-10, i
    assert abs(e[0] - (-0.4714542026506671)) <= 1e-10
    assert abs(e[1] - e[0]) <= 1e-12            # the field plays no part; l > 0 stays empty
    assert abs(e[2] - 4.0 * e[0]) <= 1e-9
    b.close()


def test_batch_imag_alone_and_then_real_time():
    """An instance relaxed in the mix equals itself relaxed alone (bitwise);
    real-time Lanczos steps after the relaxation start from the relaxed state
    at the instance's unchanged time and match the oracle."""
    from paper_1308_1856_gb300 import Batch
    n = 5
    b = Batch(SPECS, precision="fp64")
    psis = [_smooth(s, 30 + i) for i, s in enumerate(SPECS)]
    for i, p in enumerate(psis):
        b.set_state(i, p)
    b.propagate_imag(n)
    mix1 = b.get_state(1)
    relaxed0 = b.get_state(0)
    b.propagate(4)
    s = SPECS[0]
    pulse = oracle.Pulse(E0=s["E0"], omega=s["omega"], ncycles=s["ncycles"])
    want, _ = oracle.propagate(_grid(s), relaxed0, "lanczos", s["krylov"], s["dt"], 4, pulse=pulse,
                               mask=oracle.Mask(s["absorber_r"]))
    assert rel_l2(b.get_state(0), want) <= 1e-12
    assert abs(b.time(0) - 4 * s["dt"]) <= 1e-15
    b.close()
    alone = Batch([SPECS[1]], precision="fp64")
    alone.set_state(0, psis[1])
    alone.propagate_imag(2)
    alone.propagate_imag(n - 2)
    assert np.array_equal(alone.get_state(0), mix1)
    alone.close()


def test_batch_imag_arguments():
    from paper_1308_1856_gb300 import Batch, TDSEError
    b = Batch(SPECS[:2], precision="mixed")
    with pytest.raises(TDSEError):
        b.propagate_imag(3)                    # FP64 batches only
    b.close()
    b = Batch(SPECS[:2], precision="fp64")
    with pytest.raises(TDSEError):
        b.propagate_imag(-1)
    assert np.all(np.isnan(b.propagate_imag(0)))   # no step yet: no estimate
    b.close()
