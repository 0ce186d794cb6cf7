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
    return set(re.findall(r"^\s*(?:const\s+)?(?:int|double|long long|char|void)\s*\*?\s*(tdse_\w+)\s*\(",
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


def test_library_is_sm103a_build():
    assert os.path.exists(B.library_path())
    from paper_1308_1856_gb300 import build as bld
    assert "arch=compute_103a,code=sm_103a" in " ".join(bld.ARCH)
