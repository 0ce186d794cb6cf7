"""Shared helpers of the GPU tests (device memory through torch, runs through the C ABI)."""
import numpy as np

import oracle


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def make(N, dr, L, stencil, *, ghost=0, offset=0.0, Z=1.0, vtable=None, pulse=None,
         absorber_r=None, r_b=10.0, gauge="length"):
    from paper_1308_1856_gb300 import TDSE
    t = TDSE(N, dr, L, stencil=stencil, Z=Z, v_table=vtable)
    t.set_options(ghost=ghost, offset=offset, absorber=absorber_r is not None,
                  absorber_r=absorber_r or 0.0, r_b=r_b, gauge=gauge)
    if pulse is not None:
        t.set_pulse(pulse.E0, pulse.omega, pulse.ncycles, pulse.cep,
                    shape="sin2_a" if getattr(pulse, "shape", 0) == 1 else "sin2_e")
    return t


def grid_of(N, dr, L, stencil, *, ghost=0, offset=0.0, Z=1.0, vtable=None, gauge=0):
    return oracle.Grid(N=N, h=dr, L=L, stencil=stencil, ghost=ghost, offset=offset, Z=Z,
                       vtable=vtable, gauge=gauge)


def apply_h_gpu(t, E, x: np.ndarray) -> np.ndarray:
    import torch
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()
    yd = torch.empty_like(xd)
    torch.cuda.synchronize()
    t.apply_h(E, xd.data_ptr(), yd.data_ptr())
    t.sync()
    return yd.cpu().numpy()
