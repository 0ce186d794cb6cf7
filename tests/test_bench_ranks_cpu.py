"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): every
rank runs an independent replica; the reported time is the slowest rank's
and the units are summed over ranks."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = [120.0, 175.5][rank]
        units = [1e9, 3e9][rank]
        out.put((rank,) + bench.combine_over_ranks(ms, units, ws))
    finally:
        dist.destroy_process_group()


def test_combine_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms, units in res:
        assert ms == 175.5 and units == 4e9, rank


def test_combine_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_over_ranks(12.5, 7.0, 1) == (12.5, 7.0)


def test_reference_arm_prints_contract_line():
    """bench.py --impl reference times the oracle on the host and prints one
    JSON line with the contract's keys (no GPU needed)."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["unit"] == d["e2e"]["unit"] == d["cpu_baseline"]["unit"]


def test_rk_step_flop_count():
    """Per-point FP64 flops of one step through the general RK stage kernel:
    s applications of H (23 each), the inner stages' sums (4 per term), the
    last stage's two sums (one when the tableau is first-same-as-last) and
    |Delta|^2, counted here term by term."""
    import bench
    assert bench.rk_step_flops_per_gp(1) == 23 + 8 + 4
    assert bench.rk_step_flops_per_gp(4) == 4 * 23 + (4 + 8 + 12) + 8 * 4 + 4
    assert bench.rk_step_flops_per_gp(7, fsal=True) == 7 * 23 + (4 + 8 + 12 + 16 + 20 + 24) + 4 * 7 + 4
    assert bench.RK_STAGES["dormand_prince"] == 7 and bench.RK_FSAL == ("dormand_prince",)
