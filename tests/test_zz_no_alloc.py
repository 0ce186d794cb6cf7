"""The allocation-free observables entry point against the handle-based one.

tdse_observables_noalloc serves callers that cannot call cudaMalloc (for
example code running inside someone else's graph capture); it keeps its block
partials in a fixed device array instead of allocating.  This file is named so
that pytest collects it last.  The test makes two calls in a row, each on a
different state, and compares every output with tdse_observables on the same
state.
"""
import ctypes

import numpy as np
import pytest

import tdse_workloads as W
from gpu_helpers import make

pytestmark = pytest.mark.gpu

TOL = 1e-13


def _noalloc(N, dr, L, offset, r_b, psi_dev, ref_dev, out_dev, stream):
    from paper_1308_1856_gb300 import _binding as B
    return B.tdse_observables_noalloc(N, dr, L, offset, r_b, ctypes.c_void_p(psi_dev),
                                      ctypes.c_void_p(ref_dev) if ref_dev else None,
                                      ctypes.c_void_p(out_dev), ctypes.c_void_p(stream))


def test_noalloc_observables_match_handle_twice():
    import torch
    N, dr, L, offset, r_b = 1500, 0.1, 11, -0.02, 23.4
    ref = W.smooth_state(N, dr, 0, seed=77, offset=offset)[0]
    states = [W.random_state(N, L, seed=5) * 2.0, W.smooth_state(N, dr, L, seed=6, offset=offset)]
    stream = torch.cuda.Stream()
    ref_dev = torch.from_numpy(ref.copy()).cuda()
    for psi in states:
        t = make(N, dr, L, 5, offset=offset, r_b=r_b)
        t.set_state(psi)
        t.set_reference(ref)
        want = t.observables()
        psi_dev = torch.empty((L + 1, N), dtype=torch.complex128, device="cuda")
        t.get_state_device(psi_dev.data_ptr())
        t.sync()
        out_dev = torch.full((L + 5,), float("nan"), dtype=torch.float64, device="cuda")
        rc = _noalloc(N, dr, L, offset, r_b, psi_dev.data_ptr(), ref_dev.data_ptr(),
                      out_dev.data_ptr(), stream.cuda_stream)
        assert rc == 0
        stream.synchronize()
        got = out_dev.cpu().numpy()
        t.close()
        for k, key in enumerate(("norm", "dipole", "yield", "p_ground")):
            assert abs(got[k] - want[key]) <= TOL * max(1.0, abs(want[key])), key
        assert np.allclose(got[4:], want["l_pop"], rtol=TOL, atol=0)


def test_noalloc_rejects_oversized_and_bad_arguments():
    import torch
    from paper_1308_1856_gb300 import _binding as B
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    assert _noalloc(10, 0.1, B.TDSE_NOALLOC_MAX_LMAX + 1, 0.0, 5.0, p, 0, p, 0) == B.TDSE_ERR_ARG
    assert _noalloc(0, 0.1, 1, 0.0, 5.0, p, 0, p, 0) == B.TDSE_ERR_ARG
    assert _noalloc(10, 0.1, 1, 0.0, 5.0, 0, 0, p, 0) == B.TDSE_ERR_ARG
    assert _noalloc(10, 0.1, 1, 0.0, 5.0, p + 8, 0, p, 0) == B.TDSE_ERR_ARG
