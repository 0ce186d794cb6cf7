"""The server (continuous batching under a device-memory budget) on the GPU:
its results equal the batch's and the oracle's, a request gives bitwise the
same state alone and in a mix however its steps are split into step batches,
admission is FIFO within the budget, and released memory is reused."""
import numpy as np
import pytest

import oracle
import tdse_workloads as W
from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

SPECS = [
    dict(N=300, dr=0.2, lmax=4, krylov=12, dt=0.02, E0=0.0534, omega=0.057, ncycles=2),
    dict(N=517, dr=0.1, lmax=9, krylov=8, dt=5e-4, E0=0.03, omega=0.11, ncycles=3, absorber_r=40.0),
    dict(N=129, dr=0.25, lmax=2, krylov=5, dt=0.02, E0=0.08, omega=0.2, ncycles=2, cep=0.4),
    dict(N=1000, dr=0.1, lmax=15, krylov=16, dt=4e-4, E0=0.05, omega=0.057, ncycles=4, absorber_r=80.0),
    dict(N=33, dr=0.3, lmax=0, krylov=1, dt=0.05),
    dict(N=64, dr=0.2, lmax=3, krylov=3, dt=0.005, E0=0.1, omega=0.3, ncycles=2),
]


def _drain(srv, k, release=False):
    """Step until nothing is queued or running; returns finished ids in order.
    Finished requests keep their slot and memory until released, so without
    `release` the caller must leave room for every request."""
    out = []
    for _ in range(10000):
        st = srv.stats()
        if st["queued"] == 0 and st["running"] == 0:
            break
        assert st["running"] > 0 or st["resident"] < srv.max_resident, "no room left to admit"
        srv.step(k)
        fin = srv.poll()
        out += fin
        if release:
            for rid in fin:
                srv.release(rid)
    srv.sync()
    return out + srv.poll()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_server_equals_batch_and_oracle(precision):
    from paper_1308_1856_gb300 import Batch, Server
    nsteps = 23
    srv = Server(64 << 20, max_resident=16, precision=precision)
    ids = [srv.submit(s, nsteps) for s in SPECS]
    fin = _drain(srv, 10)
    assert sorted(fin) == sorted(ids)
    b = Batch(SPECS, precision=precision)
    b.propagate(nsteps)
    tol = 1e-10 if precision == "fp64" else 1e-6
    for i, (rid, s) in enumerate(zip(ids, SPECS)):
        got = srv.get_state(rid)
        assert np.array_equal(got, b.get_state(i)), i
        g = oracle.Grid(N=s["N"], h=s["dr"], L=s["lmax"], stencil=5)
        psi0 = W.hydrogen_1s(s["N"], s["dr"], s["lmax"])
        pulse = oracle.Pulse(E0=s.get("E0", 0.0), omega=s.get("omega", 0.057), ncycles=s.get("ncycles", 2.0),
                             cep=s.get("cep", 0.0))
        mask = oracle.Mask(s["absorber_r"]) if "absorber_r" in s else None
        want, _ = oracle.propagate(g, psi0, "lanczos", s["krylov"], s["dt"], nsteps, pulse=pulse, mask=mask)
        assert rel_l2(got, want) <= tol, (i, rel_l2(got, want))
        ob = srv.observables(rid)
        ow = oracle.observables(g, want, psi0[0], r_b=10.0)
        assert abs(ob["norm"] - ow["norm"]) <= 10 * tol
        assert srv.status(rid) == (Server.FINISHED, nsteps, nsteps)
    b.close()
    for rid in ids:
        srv.release(rid)
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_server_alone_equals_in_the_mix(precision):
    """The same request alone (steps in batches of 7) and admitted late into a
    running mix (batches of 100, other requests finishing around it) ends in
    bitwise the same state."""
    from paper_1308_1856_gb300 import Server
    target = SPECS[3]
    alone = Server(32 << 20, max_resident=4, precision=precision)
    a = alone.submit(target, 40)
    _drain(alone, 7)
    ref = alone.get_state(a)
    alone.close()
    mix = Server(64 << 20, max_resident=16, precision=precision)
    first = [mix.submit(s, 30 + 11 * i) for i, s in enumerate(SPECS)]
    mix.step(13)                         # the others are mid-run when the target arrives
    t = mix.submit(target, 40)
    later = [mix.submit(s, 17) for s in SPECS[:3]]
    _drain(mix, 100)
    assert np.array_equal(mix.get_state(t), ref)
    assert mix.stats()["finished_total"] == len(first) + 1 + len(later)
    mix.close()


def test_server_budget_fifo_and_reuse():
    """Room for two requests at a time: the rest wait in order, memory is
    reused after release, and every request ends where it would alone."""
    from paper_1308_1856_gb300 import Batch, Server
    spec = dict(N=800, dr=0.1, lmax=11, krylov=10, dt=0.002, E0=0.05, omega=0.1, ncycles=2)
    probe = Server(1 << 20, max_resident=1)
    per = probe.instance_bytes(spec)
    probe.close()
    srv = Server(2 * per + 4096, max_resident=8)
    ids = [srv.submit(dict(spec, cep=0.1 * i), 25) for i in range(5)]
    srv.step(10)
    st = srv.stats()
    assert st["running"] == 2 and st["queued"] == 3
    assert [srv.status(i)[0] for i in ids] == [1, 1, 0, 0, 0]
    order = []
    for _ in range(100):
        srv.step(10)
        fin = srv.poll()
        for rid in fin:
            order.append(rid)
            got = srv.get_state(rid)
            b = Batch([dict(spec, cep=0.1 * (rid - ids[0]))])
            b.propagate(25)
            assert np.array_equal(got, b.get_state(0))
            b.close()
            srv.release(rid)
        if len(order) == len(ids):
            break
    assert order == ids
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()


def test_server_errors():
    from paper_1308_1856_gb300 import Server, TDSEError
    srv = Server(1 << 20, max_resident=2)
    big = dict(N=16000, dr=0.1, lmax=127, krylov=16, dt=0.02)
    with pytest.raises(TDSEError):
        srv.submit(big, 10)                 # larger than the whole budget
    with pytest.raises(TDSEError):
        srv.submit(dict(SPECS[4], krylov=0), 10)
    rid = srv.submit(SPECS[4], 5)
    srv2_ids = [srv.submit(SPECS[4], 5) for _ in range(3)]
    with pytest.raises(TDSEError):
        srv.observables(srv2_ids[-1])       # still queued: not resident
    srv.release(srv2_ids[-1])               # cancel a queued request
    fin = _drain(srv, 2, release=True)
    assert fin == [rid] + srv2_ids[:-1]
    with pytest.raises(TDSEError):
        srv.release(12345)
    srv.close()


def test_server_autotune_and_graph_segments():
    """Autotuning on the running requests and step batches long enough to be
    replayed as graphs leave every request's result unchanged (bitwise)."""
    from paper_1308_1856_gb300 import Server
    ref = Server(64 << 20, max_resident=16)
    ids = [ref.submit(s, 9 + 4 * i) for i, s in enumerate(SPECS)]
    for _ in range(40):
        if ref.stats()["running"] == 0 and ref.stats()["queued"] == 0:
            break
        ref.step(1)                          # one-step runs: no graphs
    want = {i: ref.get_state(r) for i, r in enumerate(ids)}
    ref.close()
    srv = Server(64 << 20, max_resident=16)
    ids = [srv.submit(s, 9 + 4 * i) for i, s in enumerate(SPECS)]
    srv.step(2)
    chosen = srv.autotune()
    assert chosen["prefetch_rows"] in (0, 3, 6, 10)
    srv.step(100)                            # segments of several steps
    srv.sync()
    for i, r in enumerate(ids):
        assert np.array_equal(srv.get_state(r), want[i]), i
    srv.close()
