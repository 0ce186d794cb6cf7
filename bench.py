"""Throughput benchmark of the FD-TDSE hot path on the at-scale configuration.

Workload ("scale"): hydrogen, N = 8000 radial points, dr = 0.05 a.u. (box 400),
lmax = 63, 5-point stencil, complex128 state, sin^2 pulse (E0 = 0.0534,
omega = 0.057, 4 cycles), cos^(1/8) mask over the last 50 a.u.  One benchmark
step advances six resident states by one time step each: Taylor order 12,
classic RK4 and Lanczos with Krylov dimension 12, each in FP64 and in mixed
precision (FP32 stencil, FP64 state/dots/norms/expm).  Lanczos runs at
dt = 0.02; the explicit Taylor/RK4 propagators are unstable at that dt on this
grid (rho(H) dt ~ 1.6e4), so they run at their stable dt = 4e-6 -- the work
per step does not depend on dt.  Metric: grid-point * steps per second summed
over the propagators (6 * 512000 grid points per benchmark step).

L2 (129 MB) is flushed before every timed propagator step by writing a 256 MB
buffer; each propagator step is timed by CUDA events on the library's stream
(the flush sits outside the events).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): every rank runs an independent replica (the path has no
exchange step); value is the sum over ranks of grid-point*steps divided by the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np

import tdse_workloads as W

CFG = W.SCALE
ALL_METHODS = [(m, o, dt, p) for p in ("fp64", "mixed")
               for m, o, dt in (("taylor", 12, CFG.dt_stable), ("rk4", 4, CFG.dt_stable),
                                ("lanczos", 12, CFG.dt))]
METHODS = list(ALL_METHODS)
HBM_PEAK_GBS = 6783.1       # measured copy bandwidth of this GB300 pool (MEASURED_PEAKS.json)
METRIC = "grid-point*steps/s"
FP64_FMA_PER_CLK_PER_SM = 2          # measured on GB300 (FP64 FMA throughput probe)
SMS = 152
SM_MAX_MHZ = 2070.0
FP64_PEAK_TFLOPS = SMS * FP64_FMA_PER_CLK_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12   # 1.259


# Algorithmic FP64 flops per grid point of each kernel kind (FMA = 2), 5-point stencil:
# H x: per real component D x (1) + c1 (x-1 + x+1) (3) + c2 (x-2 + x+2) (3)
#      + two coupling terms (4) = 11, twice, plus the coupling coefficient (1) = 23.
H5_FLOPS = 23
KERNEL_FLOPS_PER_GP = {
    "taylor_stage": H5_FLOPS + 4,            # + psi + (-i s) H v
    "rk_stage": H5_FLOPS + 8,                # + g_next and acc updates (stages 1-3)
    "lanczos_a": H5_FLOPS + 6 + 4,           # + sigma H u - c u_prev, + alpha partial
    "lanczos_b": 8,                          # z - a u, + |.|^2
    "lanczos_combine": 8 * 12 + 4,           # sum of 12 complex products + norm
}
# Algorithmic HBM bytes per grid point of the mixed kernels (complex64 work
# vectors 8 B, split of psi 16 B, FP32 diagonal table 4 B; one read of every
# operand and one write of every output).
MIXED_BYTES_PER_GP = {
    "lanczos_a": 8 + 8 + 8 + 4,              # U_j, U_{j-1} (or the split), z, diag
    "lanczos_b": 8 + 8 + 8,                  # z, U_j, U_{j+1}
    "taylor_stage": 16 + 8 + 8 + 4,          # split, w_in, w_out, diag
    "rk_stage": 16 + 8 + 8 + 16 + 4,         # split, k_in, k_out, acc (hi,lo), diag
    "lanczos_combine": 8 * 11 + 16 + 16 + 16,   # 11 Krylov vectors, psi r/w, split
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples taken while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_uuid(dev: int) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


def start_state(seed: int = 31):
    return W.smooth_state(CFG.N, CFG.dr, CFG.lmax, seed=seed, lmax_populated=20)


# dram__bytes_read.sum + dram__bytes_write.sum per launch from the ncu captures
# summarised under profiles/ (null once a kernel changes after its capture)
MEASURED_TRAFFIC = {"lanczos_a": 19.9e6, "taylor_stage": 12.4e6, "rk_stage": 12.4e6}


def make_handle(stream_ptr: int, precision: str = "fp64"):
    from paper_1308_1856_gb300 import TDSE
    t = TDSE(CFG.N, CFG.dr, CFG.lmax, stencil=CFG.stencil)
    t.set_options(absorber=True, absorber_r=CFG.R - CFG.absorber_width, r_b=10.0,
                  precision=precision)
    t.set_pulse(CFG.E0, CFG.omega, CFG.ncycles)
    t.set_stream(stream_ptr)
    return t


def run_ours(args, ws, rank, local):
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)              # a real stream (not the legacy default stream)
    torch.cuda.set_stream(stream)
    psi0 = start_state()
    handles = {}
    for name, order, dt, prec in METHODS:
        t = make_handle(stream.cuda_stream, prec)
        t.set_state(psi0)
        t.time = 0.3 * CFG.duration
        handles[(name, prec)] = t
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    G = CFG.G

    def one_step(events=None):
        for idx, (name, order, dt, prec) in enumerate(METHODS):
            flush.fill_(float(idx))
            if events is not None:
                events[idx][0].record(stream)
            handles[(name, prec)].propagate(name, order, dt, 1)
            if events is not None:
                events[idx][1].record(stream)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_uuid(local))
    sampler.start()
    launches0 = sum(h.launches for h in handles.values())
    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
            for _ in METHODS] for _ in range(args.steps)]
    wall0 = time.perf_counter()
    for k in range(args.steps):
        one_step(evs[k])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    launches = sum(h.launches for h in handles.values()) - launches0
    per_method_ms = {f"{name}-{order}/{prec}": sum(evs[k][i][0].elapsed_time(evs[k][i][1])
                                                    for k in range(args.steps))
                     for i, (name, order, _, prec) in enumerate(METHODS)}
    total_ms = sum(per_method_ms.values())
    if ws > 1:
        tt = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(tt.item())
        torch.distributed.barrier()
    for h in handles.values():
        h.sync()                          # raises on Inf/NaN
    # ---- per-kernel durations (a separate profiled pass over the same steps) ----
    for h in handles.values():
        h.profile(True)
    for _ in range(max(2, min(args.steps, 5))):
        one_step()
    prof = {}
    for (mname, prec), h in handles.items():
        for kname, (ms, n) in h.profile_read().items():
            if n:
                a, b = prof.get((prec, kname), (0.0, 0))
                prof[(prec, kname)] = (a + ms, b + n)
        h.profile(False)
    kernel_share = {f"{k}/{p}": ms for (p, k), (ms, n) in prof.items()}
    fp64_kernels = {k: v for k, v in prof.items() if k[0] == "fp64"}
    roofline = None
    if fp64_kernels:
        top = max(fp64_kernels, key=lambda k: fp64_kernels[k][0])
        top_ms, top_n = prof[top]
        avg_ms = top_ms / top_n
        flops = KERNEL_FLOPS_PER_GP.get(top[1], H5_FLOPS) * G
        achieved = flops / (avg_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": f"{top[1]} (fp64)", "achieved": achieved,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                    "traffic": MEASURED_TRAFFIC.get(top[1]), "flops_per_launch": flops,
                    "avg_launch_ms": avg_ms,
                    "peak_source": "FP64: 152 SMs x 2 FMA/clk/SM x 2 flop x 2070 MHz (derived)"}
    mixed_kernels = {k: v for k, v in prof.items() if k[0] == "mixed" and k[1] in MIXED_BYTES_PER_GP}
    roofline_mixed = None
    if mixed_kernels:
        topm = max(mixed_kernels, key=lambda k: mixed_kernels[k][0])
        mms, mn = prof[topm]
        mavg = mms / mn
        mbytes = MIXED_BYTES_PER_GP[topm[1]] * G
        mach = mbytes / (mavg * 1e-3) / 1e9
        roofline_mixed = {"bound": "hbm", "kernel": f"{topm[1]} (mixed)", "achieved": mach,
                          "peak": HBM_PEAK_GBS, "unit": "GB/s", "frac": mach / HBM_PEAK_GBS,
                          "traffic": None, "bytes_per_launch": mbytes, "avg_launch_ms": mavg,
                          "peak_source": "measured HBM copy bandwidth (MEASURED_PEAKS.json) of measured"}
    # ---- end-to-end through the C ABI with host buffers ----
    pinned_in = torch.from_numpy(psi0.view(np.float64).copy()).pin_memory()
    pinned_out = [torch.empty_like(pinned_in).pin_memory() for _ in METHODS]
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    obs = None
    for _ in range(e2e_steps):
        for i, (name, order, dt, prec) in enumerate(METHODS):
            h = handles[(name, prec)]
            h.set_state_ptr(pinned_in.data_ptr())
            h.propagate(name, order, dt, 1)
            h.get_state_ptr(pinned_out[i].data_ptr())
            obs = h.observables()
    e2e_s = time.perf_counter() - e0
    nm = len(METHODS)
    h2d = nm * G * 16
    d2h = nm * (G * 16 + 8 * (CFG.lmax + 5))
    gp_steps = nm * G * args.steps * ws
    value = gp_steps / (total_ms * 1e-3)
    e2e_value = nm * G * e2e_steps * ws / e2e_s if e2e_steps else None
    result = {
        "metric": METRIC, "value": value, "unit": "grid-point*steps/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "+".join(sorted({"f64" if p == "fp64" else "f32+f64" for _, _, _, p in METHODS})),
        "data": "synthetic",
        "config": {"workload": "scale: hydrogen N=8000 dr=0.05 lmax=63 5-point, cos^(1/8) mask; "
                               "one step each of Taylor-12 and RK4 (dt=4e-6) and Lanczos-12 (dt=0.02), "
                               "in FP64 and in mixed precision",
                   "grid_points": G, "methods": [f"{m}-{o}/{p}" for m, o, _, p in METHODS],
                   "parallelism": f"replicas x{ws}", "l2": "flushed (256 MB write) before every timed propagator step"},
        "methods_ms_per_step": {k: v / args.steps for k, v in per_method_ms.items()},
        "methods_gp_steps_per_s": {k: G * args.steps / (v * 1e-3) for k, v in per_method_ms.items()},
        "roofline": roofline if roofline is not None else roofline_mixed,
        "roofline_mixed": roofline_mixed,
        "kernel_ms_share": {k: round(ms / sum(kernel_share.values()), 4) for k, ms in kernel_share.items()},
        "e2e": {"value": e2e_value, "unit": "grid-point*steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "gpu_launches": launches, "wall_s": wall, "clocks": clocks,
        "final_norm_lanczos": obs["norm"] if obs else None,
    }
    for h in handles.values():
        h.close()
    return result


def cpu_oracle_sample(budget_s: float = 12.0):
    """The oracle (serial C) on a bounded sample of the same workload: whole
    benchmark steps (Taylor-12, RK4, Lanczos-12 on the full grid) until the
    time budget is used."""
    import oracle
    g = oracle.Grid(N=CFG.N, h=CFG.dr, L=CFG.lmax, stencil=CFG.stencil)
    pulse = oracle.Pulse(CFG.E0, CFG.omega, CFG.ncycles)
    mask = oracle.Mask(CFG.R - CFG.absorber_width)
    fp64 = [(m, o, dt) for m, o, dt, p in ALL_METHODS if p == "fp64"]
    psi = {m: start_state() for m, _, _ in fp64}
    t0 = time.perf_counter()
    steps = 0
    while True:
        for name, order, dt in fp64:
            psi[name], _ = oracle.propagate(g, psi[name], name, order, dt, 1, t0=0.3 * CFG.duration,
                                            pulse=pulse, mask=mask)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= 50:
            break
    return 3 * CFG.G * steps / el, steps, el


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--method", default="all", choices=["all", "taylor", "rk4", "lanczos"],
                    help="restrict to one propagator (profiling runs)")
    ap.add_argument("--precision", default="all", choices=["all", "fp64", "mixed"],
                    help="restrict to one precision (profiling runs)")
    args = ap.parse_args()
    METHODS[:] = [m for m in ALL_METHODS if (args.method in ("all", m[0]))
                  and (args.precision in ("all", m[3]))]
    ws, rank, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return 0
        v, steps, el = cpu_oracle_sample(budget_s=min(60.0, 12.0 * max(1, args.steps) / 4))
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "grid-point*steps/s",
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * el / steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "scale (same as ours)", "grid_points": CFG.G},
                "cpu_baseline": {"value": v, "unit": "grid-point*steps/s", "cores": 1, "kind": "oracle",
                                 "sample": f"{steps} full benchmark steps on the full grid in {el:.1f} s"},
                "e2e": {"value": v, "unit": "grid-point*steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0
    if ws > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    from oracle import build as ob
    res = run_ours(args, ws, rank, local)
    if rank == 0:
        if not args.no_cpu_baseline:
            ob.build()
            v, steps, el = cpu_oracle_sample()
            res["cpu_baseline"] = {"value": v, "unit": "grid-point*steps/s", "cores": 1, "kind": "oracle",
                                   "sample": f"{steps} full benchmark steps (Taylor-12 + RK4 + Lanczos-12 "
                                             f"on the full grid) in {el:.1f} s, serial"}
        print(json.dumps(res))
    if ws > 1:
        import torch
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
