"""The C-ABI library without a GPU: it builds, loads, exports every symbol the
header declares, and rejects invalid arguments before touching the device."""
import ctypes
import re
import os

import pytest

import paper_1308_1856_gb300 as P
from paper_1308_1856_gb300 import _binding as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "tdse.h")


def _declared():
    txt = open(HEADER).read()
    return set(re.findall(r"^\s*(?:const\s+)?(?:int|double|unsigned long long|long long|long|size_t|char|void)\s*\*?\s*(tdse_\w+)\s*\(",
                          txt, re.M))


@pytest.fixture(scope="module")
def lib():
    return B.load(build_if_missing=True)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert names == set(B.SIGNATURES)


def test_invalid_create_arguments_rejected(lib):
    h = ctypes.c_void_p()
    for args in [(0, 0.1, 3, 5), (10, 0.0, 3, 5), (10, 0.1, -1, 5), (10, 0.1, 3, 4), (10, -1.0, 3, 3)]:
        rc = B.tdse_create(*args, 1.0, None, ctypes.byref(h))
        assert rc == B.TDSE_ERR_ARG, args
        assert not h.value
    assert B.tdse_create(10, 0.1, 3, 5, 1.0, None, None) == B.TDSE_ERR_ARG


def test_null_handle_calls(lib):
    assert B.tdse_destroy(None) == 0
    assert B.tdse_last_error(None) == b"null handle"
    assert B.tdse_propagate(None, 0, 4, 0.1, 1) == B.TDSE_ERR_ARG
    assert B.tdse_sync(None) == B.TDSE_ERR_ARG
    assert B.tdse_launch_count(None) == 0
    assert B.tdse_propagate_rk(None, B.TDSE_RK_DORMAND_PRINCE, 0.1, 1, None) == B.TDSE_ERR_ARG
    assert B.tdse_propagate_imag(None, 2, 12, 0.1, 1, None) == B.TDSE_ERR_ARG
    assert B.tdse_dipole_moments(None, None, None, None) == B.TDSE_ERR_ARG
    assert B.tdse_dipole_series(None, 10) == B.TDSE_ERR_ARG
    assert B.tdse_dipole_series_read(None, None, 0, None) == B.TDSE_ERR_ARG
    assert B.tdse_flux_setup(None, 10.0, 0, None) == B.TDSE_ERR_ARG
    assert B.tdse_flux_read(None, None, None, None, None) == B.TDSE_ERR_ARG


def test_library_is_sm103a_build():
    assert os.path.exists(B.library_path())
    from paper_1308_1856_gb300 import build as bld
    assert "arch=compute_103a,code=sm_103a" in " ".join(bld.ARCH)


def test_server_arguments_rejected_without_touching_the_device(lib):
    h = ctypes.c_void_p()
    for args in [(0, 16, 5, 0), (1 << 20, 0, 5, 0), (1 << 20, 16, 4, 0), (1 << 20, 16, 5, 2)]:
        assert B.tdse_server_create(*args, ctypes.byref(h)) == B.TDSE_ERR_ARG, args
        assert not h.value
    assert B.tdse_server_destroy(None) == 0
    assert B.tdse_server_last_error(None) == b"null server"
    assert B.tdse_server_step(None, 10, None) == B.TDSE_ERR_ARG
    assert B.tdse_server_release(None, 1) == B.TDSE_ERR_ARG
    assert B.tdse_server_sync(None) == B.TDSE_ERR_ARG


def _spec(**kw):
    d = dict(N=1000, dr=0.1, lmax=15, Z=1.0, E0=0.05, omega=0.057, ncycles=2.0, cep=0.0, krylov=12,
             dt=0.02, absorber_r=50.0, r_b=10.0, gauge=0, pulse_shape=0)
    d.update(kw)
    return B.tdse_instance_spec(*[d[f] for f, _ in B.tdse_instance_spec._fields_])


def test_server_instance_bytes(lib):
    """Device bytes of one request: every array of the instance, each rounded
    up to 256 bytes (counted here from the list of arrays, not the code)."""
    def up(x):
        return (x + 255) // 256 * 256

    for N, L, m in [(1000, 15, 12), (2000, 127, 16), (33, 0, 1), (16000, 63, 8)]:
        G = N * (L + 1)
        nchunk = max(-(-((N + 31) // 32) * (L + 1) // 64), -(-G // 2048))
        ndip = -(-((N + 31) // 32) * (L + 1) // 64)    # dipole chunks: 4 partial sums each
        common = up(16 * G) + up(8 * N) * 2 + up(8 * (L + 2)) + up(8 * nchunk) + up(32 * ndip) + up(16 * N)
        fp64 = common + up(8 * G) + up(16 * G * m)
        mixed = common + up(4 * G) + 2 * up(8 * G) + up(8 * G * m) + up(4 * N) + up(4 * (L + 2))
        s = _spec(N=N, lmax=L, krylov=m)
        assert B.tdse_server_instance_bytes(ctypes.byref(s), B.TDSE_FP64) == fp64
        assert B.tdse_server_instance_bytes(ctypes.byref(s), B.TDSE_MIXED) == mixed
    # a velocity-gauge instance also keeps 1/r
    for N, L, m in [(1000, 15, 12), (33, 0, 1)]:
        G = N * (L + 1)
        nchunk = max(-(-((N + 31) // 32) * (L + 1) // 64), -(-G // 2048))
        ndip = -(-((N + 31) // 32) * (L + 1) // 64)    # dipole chunks: 4 partial sums each
        common = up(16 * G) + up(8 * N) * 2 + up(8 * (L + 2)) + up(8 * nchunk) + up(32 * ndip) + up(16 * N)
        s = _spec(N=N, lmax=L, krylov=m, gauge=1)
        assert B.tdse_server_instance_bytes(ctypes.byref(s), B.TDSE_FP64) == common + up(8 * G) + up(16 * G * m) + up(8 * N)
        # ... and a mixed one keeps it in FP32 (4 bytes)
        mixed = common + up(4 * G) + 2 * up(8 * G) + up(8 * G * m) + up(4 * N) + up(4 * (L + 2)) + up(4 * N)
        assert B.tdse_server_instance_bytes(ctypes.byref(s), B.TDSE_MIXED) == mixed
    bad = _spec(krylov=0)
    assert B.tdse_server_instance_bytes(ctypes.byref(bad), B.TDSE_FP64) == 0
    assert B.tdse_server_instance_bytes(ctypes.byref(_spec(gauge=2)), B.TDSE_FP64) == 0
    assert B.tdse_server_instance_bytes(ctypes.byref(_spec(pulse_shape=5)), B.TDSE_FP64) == 0
    assert B.tdse_server_instance_bytes(ctypes.byref(_spec(dt=-1.0)), B.TDSE_FP64) == 0


def test_header_is_plain_c99(tmp_path):
    """include/tdse.h compiles on its own as C99 (no C++ or CUDA types leak
    into the boundary) and every declared function links against the library."""
    import subprocess
    src = tmp_path / "use_header.c"
    names = sorted(_declared())
    body = "\n".join(f"  (void)&{n};" for n in names)
    src.write_text(f'#include "tdse.h"\nint main(void) {{\n{body}\n  return 0;\n}}\n')
    exe = tmp_path / "use_header"
    lib = B.library_path()
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                        os.path.dirname(HEADER), str(src), "-o", str(exe), lib,
                        f"-Wl,-rpath,{os.path.dirname(lib)}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
