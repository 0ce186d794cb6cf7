"""The allocation-free observables entry point against the handle-based one
and against the oracle.

tdse_observables_noalloc serves callers that cannot call cudaMalloc (for
example code running inside someone else's graph capture); it keeps its block
partials in a fixed device array instead of allocating.  This file is named so
that pytest collects it last.  The calls below run back to back on one stream,
each on a different state, so every call starts from the shared array as the
previous one left it:
  1, 2. two states of one grid (offset grid, a reference wave);
  3.    a different grid shape (one block per partial wave, lmax near the
        limit), no reference (p_ground = 0), r_b exactly on a grid point;
  4.    a state holding a NaN: the non-finite slot reads 1.
Each output is compared with tdse_observables on the same state (the same sums
in the same order: 1e-13) and with oracle.observables (index-order sums: within
1e-13 of the sum of the absolute terms).
"""
import ctypes

import numpy as np
import pytest

import oracle
import tdse_workloads as W
from gpu_helpers import grid_of, make

pytestmark = pytest.mark.gpu

TOL = 1e-13
KEYS = ("norm", "dipole", "yield", "p_ground")


def _noalloc(N, dr, L, offset, r_b, psi_dev, ref_dev, out_dev, stream):
    from paper_1308_1856_gb300 import _binding as B
    return B.tdse_observables_noalloc(N, dr, L, offset, r_b, ctypes.c_void_p(psi_dev),
                                      ctypes.c_void_p(ref_dev) if ref_dev else None,
                                      ctypes.c_void_p(out_dev), ctypes.c_void_p(stream))


def _abs_bounds(psi, ref, N, dr, L, offset):
    """Sums of the absolute values of the terms of each observable, the scale
    of the rounding of any summation order."""
    r = np.arange(1, N + 1) * dr + offset
    a = np.abs(psi) ** 2
    kap = np.array([np.sqrt((l + 1.0) ** 2 / (4.0 * (l + 1.0) ** 2 - 1.0)) for l in range(L)])
    dip = 2.0 * dr * float(np.sum(kap[:, None] * np.abs(r[None, :] * (psi[:-1].conj() * psi[1:]).real))) if L else 0.0
    ov = dr * float(np.sum(np.abs(ref) * np.abs(psi[0]))) if ref is not None else 0.0
    nrm = dr * float(a.sum())
    return {"norm": nrm, "dipole": dip, "yield": max(1.0, nrm), "p_ground": 4.0 * ov * ov}


def _run(N, dr, L, offset, r_b, psi, ref, stream):
    import torch
    t = make(N, dr, L, 5, offset=offset, r_b=r_b)
    t.set_state(psi)
    # the handle's reference defaults to its 1s state: a zero wave stands for "none"
    t.set_reference(ref if ref is not None else np.zeros(N, dtype=np.complex128))
    finite = bool(np.all(np.isfinite(psi)))
    want = t.observables() if finite else None
    psi_dev = torch.from_numpy(np.ascontiguousarray(psi)).cuda()
    ref_dev = torch.from_numpy(np.ascontiguousarray(ref)).cuda() if ref is not None else None
    out_dev = torch.full((L + 6,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    rc = _noalloc(N, dr, L, offset, r_b, psi_dev.data_ptr(), ref_dev.data_ptr() if ref_dev is not None else 0,
                  out_dev.data_ptr(), stream.cuda_stream)
    assert rc == 0
    stream.synchronize()
    got = out_dev.cpu().numpy()
    t.close()
    return got, want


def _check(got, want, psi, ref, N, dr, L, offset, r_b):
    # against the handle: the same sums in the same order
    for k, key in enumerate(KEYS):
        assert abs(got[k] - want[key]) <= TOL * max(1.0, abs(want[key])), (key, got[k], want[key])
    assert np.allclose(got[4:L + 5], want["l_pop"], rtol=TOL, atol=0)
    assert got[L + 5] == 0.0
    # against the oracle
    g = grid_of(N, dr, L, 5, offset=offset)
    ow = oracle.observables(g, psi, ref, r_b=r_b)
    bounds = _abs_bounds(psi, ref, N, dr, L, offset)
    for k, key in enumerate(KEYS):
        assert abs(got[k] - ow[key]) <= TOL * max(1.0, bounds[key]), (key, got[k], ow[key])
    assert np.allclose(got[4:L + 5], ow["l_pop"], rtol=TOL, atol=0)
    return ow


def test_noalloc_observables_in_a_row():
    import torch
    stream = torch.cuda.Stream()
    # calls 1 and 2: one grid, two states, a reference wave
    N, dr, L, offset, r_b = 1500, 0.1, 11, -0.02, 23.4
    ref = W.smooth_state(N, dr, 0, seed=77, offset=offset)[0]
    for psi in (W.random_state(N, L, seed=5) * 2.0, W.smooth_state(N, dr, L, seed=6, offset=offset)):
        got, want = _run(N, dr, L, offset, r_b, psi, ref, stream)
        _check(got, want, psi, ref, N, dr, L, offset, r_b)
    # call 3: N < 256 (one block per partial wave), lmax near the limit, no
    # reference, and r_b exactly on grid point 40 of an offset grid, where a
    # fused multiply-add would round r_40 = 40 dr + offset one unit higher
    # (3.9800000000000004 instead of 3.98) and drop the point from the inside
    from paper_1308_1856_gb300 import _binding as B
    N, dr, L, offset = 200, 0.1, B.TDSE_NOALLOC_MAX_LMAX - 3, -0.02
    r_b = 40 * dr + offset
    psi = W.random_state(N, L, seed=9)
    got, want = _run(N, dr, L, offset, r_b, psi, None, stream)
    ow = _check(got, want, psi, None, N, dr, L, offset, r_b)
    assert got[3] == 0.0 and want["p_ground"] == 0.0 and ow["p_ground"] == 0.0
    r = np.arange(1, N + 1) * dr + offset
    assert r[39] == r_b
    inside = dr * float(np.sum(np.abs(psi[:, r <= r_b]) ** 2))
    assert abs(got[2] - (1.0 - inside)) <= TOL * max(1.0, got[0])
    row40 = dr * float(np.sum(np.abs(psi[:, 39]) ** 2))
    assert abs(got[2] - (1.0 - inside)) < 0.5 * row40     # the point at r_b is inside
    # call 4: a state holding a NaN (a host-side input, not a device fault)
    bad = W.smooth_state(N, dr, L, seed=10)
    bad[3, 17] = complex(np.nan, 0.0)
    got, _ = _run(N, dr, L, offset, r_b, bad, None, stream)
    assert got[L + 5] == 1.0 and not np.isfinite(got[0])


def test_noalloc_rejects_oversized_and_bad_arguments():
    import torch
    from paper_1308_1856_gb300 import _binding as B
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    assert _noalloc(10, 0.1, B.TDSE_NOALLOC_MAX_LMAX + 1, 0.0, 5.0, p, 0, p, 0) == B.TDSE_ERR_ARG
    assert _noalloc(0, 0.1, 1, 0.0, 5.0, p, 0, p, 0) == B.TDSE_ERR_ARG
    assert _noalloc(10, 0.1, 1, 0.0, 5.0, 0, 0, p, 0) == B.TDSE_ERR_ARG
    assert _noalloc(10, 0.1, 1, 0.0, 5.0, p + 8, 0, p, 0) == B.TDSE_ERR_ARG
    assert _noalloc(10, 0.1, 1, -0.2, 5.0, p, 0, p, 0) == B.TDSE_ERR_ARG    # r_1 <= 0
