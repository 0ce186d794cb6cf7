"""Programmatic dependent launch: every kernel launched through launch_pdl may
start while the kernel before it on the stream is still running, so it must
call pdl_wait() before its first access to device memory, and may call
pdl_trigger() only after that wait (so at most two kernels of the chain are
resident).  A source-level check over csrc/: for each kernel named in a
launch_pdl call, the statements before pdl_wait() declare shared memory or
compute from by-value arguments only (no subscript, no '->')."""
import pathlib
import re

import pytest

CSRC = pathlib.Path(__file__).resolve().parent.parent / "paper_1308_1856_gb300" / "csrc"


def _sources():
    return {p.name: p.read_text() for p in sorted(CSRC.glob("*.cu"))}


def _strip_comments(text):
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.sub(r"//[^\n]*", "", text)


def _pdl_kernels(srcs):
    names = set()
    for text in srcs.values():
        for m in re.finditer(r"launch_pdl\(\s*([A-Za-z_]\w*)", _strip_comments(text)):
            names.add(m.group(1))
    return sorted(names)


def _kernel_body(text, name):
    """Body of the __global__ function `name` (text between its braces)."""
    text = _strip_comments(text)
    for m in re.finditer(r"\b" + re.escape(name) + r"\s*\(", text):
        head = text[max(0, m.start() - 300):m.start()]
        if "__global__" not in head or ";" in head[head.rfind("__global__"):]:
            continue
        # the parameter list, then the opening brace of the body
        depth, i = 0, m.end() - 1
        while True:
            c = text[i]
            depth += (c == "(") - (c == ")")
            i += 1
            if depth == 0:
                break
        j = text.index("{", i)
        depth, k = 0, j
        while True:
            c = text[k]
            depth += (c == "{") - (c == "}")
            k += 1
            if depth == 0:
                return text[j + 1:k - 1]
    return None


def test_pdl_kernels_found():
    names = _pdl_kernels(_sources())
    # the single-instance chains of both precisions and the small exponential
    for want in ("lanczos_a_kernel", "lanczos_b_kernel", "lanczos_combine_kernel", "norm_kernel",
                 "taylor_stage_kernel", "rk_stage_kernel", "rk_general_stage_kernel", "lanczos_expm_kernel",
                 "mx_lanczos_a_kernel", "mx_lanczos_b_kernel", "mx_lanczos_combine_kernel", "mx_split_kernel",
                 "mx_taylor_stage_kernel", "mx_rk_stage_kernel"):
        assert want in names, want


@pytest.mark.parametrize("name", _pdl_kernels(_sources()))
def test_pdl_kernel_waits_before_memory(name):
    bodies = [b for b in (_kernel_body(t, name) for t in _sources().values()) if b is not None]
    assert bodies, f"no __global__ definition of {name}"
    for body in bodies:
        assert "pdl_wait();" in body, name
        pre = body[:body.index("pdl_wait();")]
        stmts = [s.strip() for s in pre.split(";") if s.strip()]
        for s in stmts:
            if s.startswith("__shared__"):
                continue
            assert "[" not in s and "->" not in s, (name, s)
        if "pdl_trigger();" in body:
            assert body.index("pdl_trigger();") > body.index("pdl_wait();"), name


def test_launch_pdl_sets_programmatic_serialization():
    text = (CSRC / "tdse_internal.cuh").read_text()
    assert "cudaLaunchAttributeProgrammaticStreamSerialization" in text
    assert "programmaticStreamSerializationAllowed = 1" in text
    assert 'asm volatile("griddepcontrol.wait;" ::: "memory")' in text
