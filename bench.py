"""Throughput benchmark of the FD-TDSE hot path.

Headline (value, ms_per_step, dtype f64, roofline, e2e, cpu_baseline): the
batched configuration in FP64 -- 256 seeded uneven instances (N 2000-16000,
dr = 0.1, lmax 15-127, Krylov dimension 8-16, 5-point stencil, sin^2 pulses
of 1e13-5e14 W/cm^2, 400-1600 nm, 2-6 cycles, dt = 0.02, cos^(1/8) mask over
the last 50 a.u.), one Lanczos step of every instance per benchmark step,
replayed from a captured step graph (the batch captures the step on the
second identical call and replays it from then on).  Metric: grid-point *
steps per second (1.66e8 grid points per step).

Every other configuration is reported in its own field ("configs" holds a
compact summary at the end of the line):
  c1  small configuration (N=500, dr=0.2, lmax=4, 3-point, 2,500 points):
      Taylor-8, RK4 and Lanczos-12 per step on the one-launch cluster path and
      on the multi-launch path;
  c2  at-scale grid (N=8000, dr=0.05, lmax=63, 5-point, mask; 512,000 points)
      in FP64: Taylor-12, RK4 (both at their stable dt = 4e-6; the work per
      step does not depend on dt) and Lanczos-12 (dt = 0.02);
  c3  the same in mixed precision, with its error against the FP64 oracle
      (norm, partial-wave populations, dipole series) at a converging step;
  c4  the batched configuration in mixed precision, and both precisions at a
      per-instance converging step (rho(H) dt = m/2) with their errors
      against the FP64 oracle on sampled instances;
  c5  the served configuration (Poisson arrivals, continuous batching under a
      150 GB budget, step batches of 100): p50/p99 time to completion;
  hpsi  the operator alone (tdse_apply_h) on the at-scale grid.
Further legs: the embedded RK pairs, the per-step observables, the FP64 FMA
probe and the serial oracle (cpu_baseline) on the host cores.

L2 (129 MB) is flushed before every timed step by writing a 256 MB buffer;
each step is timed by CUDA events on the library's stream (the flush sits
outside the events).

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
METRIC = "grid-point*steps/s"
UNIT = "grid-point*steps/s"
BATCH_COUNT = 256
BATCH_SEED = 1308
BATCH_DT = 0.02            # the batched configuration states no step; that of the at-scale one
BATCH_ABSORBER = 50.0      # nor an absorber; the same cos^(1/8) mask over the last 50 a.u.
E2E_GROUPS = 4             # instance groups whose copies overlap the others' compute (e2e leg)
FP64_FMA_PER_CLK_PER_SM = 2          # FP64 FMA lanes per SM per clock on GB300 (tdse_fma_throughput)
RECIPE_SM_MAX_MHZ = 2070.0           # maximum SM clock of the GB300 (profiling recipe)
FALLBACK_HBM_GBS = 6800.0            # the profiling recipe's fallback copy bandwidth


def measured_peaks():
    """HBM copy bandwidth and the SM clock from MEASURED_PEAKS.json (written
    on the GPU pool), else the profiling recipe's fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", RECIPE_SM_MAX_MHZ)), "measured"
    except (OSError, ValueError, KeyError):
        return FALLBACK_HBM_GBS, RECIPE_SM_MAX_MHZ, "fallback"


HBM_PEAK_GBS, SM_MAX_MHZ, PEAK_KIND = measured_peaks()

# Algorithmic FP64 flops per grid point of each kernel kind (FMA = 2), 5-point stencil:
# H x: per real component D x (1) + c1 (x-1 + x+1) (3) + c2 (x-2 + x+2) (3)
#      + two coupling terms (4) = 11, twice, plus the coupling coefficient (1) = 23.
H5_FLOPS = 23
KERNEL_FLOPS_PER_GP = {
    "apply_h": H5_FLOPS,
    "taylor_stage": H5_FLOPS + 4,            # + psi + (-i s) H v
    "rk_stage": H5_FLOPS + 8,                # + g_next and acc updates (stages 1-3)
    "lanczos_a": H5_FLOPS + 6 + 4,           # + sigma H u - c u_prev, + alpha partial
    "lanczos_b": 8,                          # z - a u, + |.|^2
    # a whole Lanczos-12 step in one launch (tdse_persist.cu): 12 A phases,
    # 11 B phases and the combine (11 complex terms + c_0 psi, mask, |.|^2)
    "lanczos_persistent": 12 * (H5_FLOPS + 6 + 4) + 11 * 8 + (11 * 8 + 6 + 4),
}
# Algorithmic HBM bytes per grid point of the FP64 kernels (complex128 16 B,
# diagonal table 8 B; one read of every operand and one write of every output).
FP64_BYTES_PER_GP = {
    "apply_h": 16 + 8 + 16,                  # x, diag, y
    "taylor_stage": 16 + 16 + 8 + 16,        # v_in, psi, diag, v_out
    "lanczos_persistent": 12 * 56 + 11 * 48 + (12 * 16 + 16),   # as the phases of the multi-launch path
    "rk_stage": 16 + 16 + 16 + 8 + 16 + 16,  # g, psi, acc_in, diag, acc_out, g_next
    "lanczos_a": 16 + 16 + 8 + 16,           # U_j, U_{j-1}, diag, z
    "lanczos_b": 16 + 16 + 16,               # z, U_j, U_{j+1}
}
# Dipole moments kernel, per grid point: |f|^2 (4), w Re(f_l^* f_{l+1}) (5),
# the unscaled first derivative (8), w Im(f_{l+1}^* D1 f_l) (5) and
# w (l+1) Im(f_{l+1}^* f_l) (5).
DIPOLE_FLOPS_PER_GP = 27
# Algorithmic HBM bytes per grid point of the mixed kernels (complex64 work
# vectors 8 B, split of psi 16 B, FP32 diagonal table 4 B; one read of every
# operand and one write of every output).
MIXED_BYTES_PER_GP = {
    "apply_h": 16 + 4 + 16,                  # x (complex128), diag, y (complex128)
    "lanczos_a": 8 + 8 + 8 + 4,              # U_j, U_{j-1} (or the split), z, diag
    "lanczos_b": 8 + 8 + 8,                  # z, U_j, U_{j+1}
    "taylor_stage": 16 + 8 + 8 + 4,          # split, w_in, w_out, diag
    "rk_stage": 16 + 8 + 8 + 16 + 4,         # split, k_in, k_out, acc (hi,lo), diag
    "lanczos_combine": 8 * 11 + 16 + 16 + 16,   # 11 Krylov vectors, psi r/w, split
}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per algorithmic
# grid point of one launch, from the ncu captures summarised under profiles/:
# the batched kernels on the first 16 instances of the batched configuration
# (phases where all 16 are active, 10.66M points per launch), scaled here to a
# full launch by its points; the single-instance kernels on the at-scale grid
# (512000 points).  An entry is removed when its kernel changes after capture.
MEASURED_TRAFFIC_PER_POINT = {
    ("batched", "fp64", "lanczos_a"): (537.5e6 + 165.8e6) / 10664737,
    ("batched", "fp64", "lanczos_b"): (343.0e6 + 138.5e6) / 10664737,
    ("batched", "mixed", "lanczos_a"): (218.7e6 + 56.2e6) / 10664737,
    ("batched", "mixed", "lanczos_b"): (171.2e6 + 52.7e6) / 10664737,
    # ("single", "fp64", "taylor_stage") was 20.6e6 / 512000; removed since the
    # kernel gained its programmatic-launch wait and trigger.
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def sig(x, n=4):
    """x rounded to n significant digits (compact JSON)."""
    if x is None or not isinstance(x, (int, float)) or not math.isfinite(x) or x == 0:
        return x
    return float(f"{x:.{n}g}")


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


class Device:
    """The device, its stream, an L2 flush buffer and the FP64 peak."""

    def __init__(self, local: int):
        import torch
        torch.cuda.set_device(local)
        self.torch = torch
        self.dev = torch.device("cuda", local)
        self.stream = torch.cuda.Stream(self.dev)          # a real stream (not the legacy default stream)
        torch.cuda.set_stream(self.stream)
        self.sptr = self.stream.cuda_stream
        self.flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=self.dev)
        self.sms = torch.cuda.get_device_properties(local).multi_processor_count
        # FP64 peak: SMs (device) x FMA lanes/clk/SM (probe) x 2 flop x maximum SM clock
        self.fp64_peak = self.sms * FP64_FMA_PER_CLK_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
        self.peak_source = (f"FP64: {self.sms} SMs x {FP64_FMA_PER_CLK_PER_SM} FMA/clk/SM x 2 flop x "
                            f"{SM_MAX_MHZ:g} MHz (derived; the FMA probe measures it)")

    def flush(self, k=0.0):
        self.flush_buf.fill_(float(k))

    def events(self, n):
        E = self.torch.cuda.Event
        return [(E(enable_timing=True), E(enable_timing=True)) for _ in range(n)]

    def sync(self):
        self.torch.cuda.synchronize()


def start_state(seed: int = 31):
    return W.smooth_state(CFG.N, CFG.dr, CFG.lmax, seed=seed, lmax_populated=20)


def make_handle(sptr: int, precision: str = "fp64"):
    from paper_1308_1856_gb300 import TDSE
    t = TDSE(CFG.N, CFG.dr, CFG.lmax, stencil=CFG.stencil)
    t.set_options(absorber=True, absorber_r=CFG.R - CFG.absorber_width, r_b=10.0, precision=precision)
    t.set_pulse(CFG.E0, CFG.omega, CFG.ncycles)
    t.set_stream(sptr)
    return t


def batched_request_spec(x, dt=BATCH_DT):
    return dict(N=x.N, dr=x.dr, lmax=x.lmax, krylov=x.krylov, dt=dt, E0=x.E0, omega=x.omega,
                ncycles=x.ncycles, absorber_r=x.N * x.dr - BATCH_ABSORBER)


class HandleRow:
    """One single-instance propagator on the at-scale grid."""
    kind = "single"

    def __init__(self, method, order, dt, prec, sptr, psi0):
        self.method, self.order, self.dt, self.prec = method, order, dt, prec
        self.name = f"{method}-{order}/{prec}"
        self.h = make_handle(sptr, prec)
        self.h.set_state(psi0)
        self.h.time = 0.3 * CFG.duration
        self.gp = CFG.G
        self.e2e_bytes = (CFG.G * 16, CFG.G * 16 + 8 * (CFG.lmax + 5))

    def step(self):
        self.h.propagate(self.method, self.order, self.dt, 1)

    def kernel_points(self, kind):
        """algorithmic grid points of one step that a kernel kind processes"""
        if kind in ("lanczos_a", "taylor_stage"):
            return self.order * self.gp
        if kind == "lanczos_b":
            return (self.order - 1) * self.gp
        if kind == "rk_stage":
            return 4 * self.gp
        return self.gp

    def e2e_step(self, pin_in, pin_out):
        self.h.set_state_ptr(pin_in.data_ptr())
        self.step()
        self.h.get_state_ptr(pin_out.data_ptr())
        return self.h.observables()

    def close(self):
        self.h.close()


class BatchRow:
    """256 uneven instances (seed 1308), one Lanczos step of every instance per
    benchmark step (tdse_batch_propagate(1): from the second identical call on,
    a replay of the captured step graph)."""
    kind = "batched"

    def __init__(self, prec, sptr, count=BATCH_COUNT, schedule=None, dts=None):
        from paper_1308_1856_gb300 import Batch
        self.specs = W.batched_specs(count, BATCH_SEED)
        self.prec = prec
        self.name = f"batched-{count}/{prec}"
        self.dts = dts or [BATCH_DT] * count
        self.b = Batch([batched_request_spec(x, dt) for x, dt in zip(self.specs, self.dts)], stencil=5,
                       precision=prec)
        self.b.set_stream(sptr)
        if schedule is None:
            self.schedule = self.b.autotune()     # before the warm-up; not timed
        else:                                     # a fixed schedule (profiling runs)
            pf, ring, sb, eb = schedule
            self.b.set_schedule(pf, sb, eb, ring_rows=ring)
            self.schedule = self.b.schedule()
        self.gp = self.b.points
        self.G = [x.N * (x.lmax + 1) for x in self.specs]
        self.e2e_bytes = (self.gp * 16, self.gp * 16)

    @property
    def h(self):
        return self.b

    def step(self):
        self.b.propagate(1)

    def kernel_points(self, kind):
        m = [x.krylov for x in self.specs]
        if kind == "lanczos_a":
            return sum(g * mi for g, mi in zip(self.G, m))
        if kind == "lanczos_b":
            return sum(g * (mi - 1) for g, mi in zip(self.G, m))
        return self.gp

    def e2e_step(self, pin_in, pin_out):
        # every state in, one step, every state out, the copies of one group of
        # instances overlapping the compute of another (tdse_batch_propagate_io)
        self.b.propagate_io(pin_in.data_ptr(), pin_out.data_ptr(), 1, groups=E2E_GROUPS)
        return self.b.observables(0)

    def close(self):
        self.b.close()


def combine_over_ranks(total_ms: float, units: float, ws: int, device="cpu"):
    """Slowest rank's timed milliseconds and the units all ranks processed
    (replicas: no data exchange, only these two scalars)."""
    if ws == 1:
        return total_ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def time_rows(D: Device, rows, steps, warmup):
    """warmup untimed steps, then `steps` timed steps of every row (L2 flushed
    before each, CUDA events around each); ms per row summed over the steps."""
    for _ in range(warmup):
        for k, r in enumerate(rows):
            D.flush(k)
            r.step()
    D.sync()
    evs = [D.events(len(rows)) for _ in range(steps)]
    for s in range(steps):
        for k, r in enumerate(rows):
            D.flush(k)
            evs[s][k][0].record(D.stream)
            r.step()
            evs[s][k][1].record(D.stream)
    D.sync()
    return {r.name: sum(evs[s][k][0].elapsed_time(evs[s][k][1]) for s in range(steps))
            for k, r in enumerate(rows)}


def profile_rows(D: Device, rows, steps=2):
    """Per-kernel durations from a profiled pass over the same steps (events
    around every launch): {(row kind, precision, kernel): [ms, launches, points]}."""
    for r in rows:
        r.h.profile(True)
    for s in range(steps):
        for k, r in enumerate(rows):
            D.flush(k)
            r.step()
    prof = {}
    for r in rows:
        for kname, (ms, n) in r.h.profile_read().items():
            if n:
                a = prof.setdefault((r.kind, r.prec, kname), [0.0, 0, 0])
                a[0] += ms
                a[1] += n
                a[2] += steps * r.kernel_points(kname)
        r.h.profile(False)
    return prof


def roofline_of(D: Device, key, prof):
    """Roofline object of one kernel: FP64 kernels against the FP64 ALU peak
    (with their HBM fraction beside it), mixed kernels against HBM."""
    ms, n, pts = prof[key]
    kind, prec, k = key
    per = MEASURED_TRAFFIC_PER_POINT.get(key)
    traffic = None if per is None else per * pts / n
    if prec == "fp64":
        flops = KERNEL_FLOPS_PER_GP.get(k, H5_FLOPS) * pts
        achieved = flops / (ms * 1e-3) / 1e12
        nbytes = FP64_BYTES_PER_GP.get(k, 0) * pts
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"bound": "alu", "kernel": f"{k} ({kind}, fp64)", "achieved": achieved, "peak": D.fp64_peak,
                "unit": "TFLOP/s", "frac": achieved / D.fp64_peak, "traffic": traffic,
                "flops_per_launch": flops / n, "avg_launch_ms": ms / n,
                "hbm_gbs": gbs, "hbm_frac": gbs / HBM_PEAK_GBS, "peak_source": D.peak_source}
    nbytes = MIXED_BYTES_PER_GP[k] * pts
    achieved = nbytes / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": f"{k} ({kind}, mixed)", "achieved": achieved, "peak": HBM_PEAK_GBS,
            "unit": "GB/s", "frac": achieved / HBM_PEAK_GBS, "traffic": traffic,
            "bytes_per_launch": nbytes / n, "avg_launch_ms": ms / n,
            "peak_source": f"HBM copy bandwidth of {PEAK_KIND} (MEASURED_PEAKS.json)"}


def dominant_roofline(D, prof, prec):
    keys = [k for k in prof if k[1] == prec and (k[2] in KERNEL_FLOPS_PER_GP if prec == "fp64"
                                                  else k[2] in MIXED_BYTES_PER_GP)]
    if not keys:
        return None
    return roofline_of(D, max(keys, key=lambda k: prof[k][0]), prof)


def e2e_rows(D: Device, rows, steps, psi0, warmup=2):
    """The same steps end to end through the C ABI with host buffers: every
    step copies every state in from pinned host memory, advances it, copies
    it out and reads its observables.  Untimed passes first: the first copies
    through freshly pinned buffers pay one-off mapping costs, and a batch's
    pipelined copies size their groups by the compute / copy ratio that its
    previous call measured (tdse_batch_propagate_io), so the second pass is
    the first with calibrated groups."""
    torch = D.torch
    pins = []
    for r in rows:
        src = psi0 if r.kind == "single" else r.b.get_states()
        pin_in = torch.from_numpy(np.ascontiguousarray(src).view(np.float64).copy()).pin_memory()
        pins.append((pin_in, torch.empty_like(pin_in).pin_memory()))
    for _ in range(warmup):
        for r, (pi, po) in zip(rows, pins):
            r.e2e_step(pi, po)
    D.sync()
    per_row = {}
    t0 = time.perf_counter()
    for _ in range(steps):
        for r, (pi, po) in zip(rows, pins):
            a = time.perf_counter()
            r.e2e_step(pi, po)
            per_row[r.name] = per_row.get(r.name, 0.0) + time.perf_counter() - a
    wall = time.perf_counter() - t0
    gp = sum(r.gp for r in rows) * steps
    return {"value": gp / wall, "unit": UNIT, "h2d_bytes_per_step": sum(r.e2e_bytes[0] for r in rows),
            "d2h_bytes_per_step": sum(r.e2e_bytes[1] for r in rows), "steps": steps, "warmup": warmup,
            "ms_per_step_by_row": {k: 1e3 * v / steps for k, v in per_row.items()}}


# ---------------------------------------------------------------------------
# The serial oracle on the host cores (cpu_baseline, --impl reference)
# ---------------------------------------------------------------------------
def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def lpt_partition(weights, parts):
    """Longest-processing-time assignment of items to `parts` workers."""
    order = sorted(range(len(weights)), key=lambda i: -weights[i])
    load = [0.0] * parts
    out = [[] for _ in range(parts)]
    for i in order:
        w = min(range(parts), key=lambda p: load[p])
        out[w].append(i)
        load[w] += weights[i]
    return out


def _oracle_batch_worker(args):
    """One worker of the batched oracle: its instances of the batched FP64
    configuration, `warmup + steps` Lanczos steps each from the 1s state at
    t = 0; (grid points per step, seconds of the timed steps)."""
    ids, warmup, steps = args
    import oracle
    specs = W.batched_specs(BATCH_COUNT, BATCH_SEED)
    inst = []
    for i in ids:
        x = specs[i]
        g = oracle.Grid(N=x.N, h=x.dr, L=x.lmax, stencil=5)
        inst.append((x, g, W.hydrogen_1s(x.N, x.dr, x.lmax), oracle.Pulse(E0=x.E0, omega=x.omega, ncycles=x.ncycles),
                     oracle.Mask(x.N * x.dr - BATCH_ABSORBER)))
    gp = sum(x.N * (x.lmax + 1) for x, *_ in inst)
    el = 0.0
    for n in range(warmup + steps):
        t0 = time.perf_counter()
        for k, (x, g, psi, pulse, mask) in enumerate(inst):
            out, _ = oracle.propagate(g, psi, "lanczos", x.krylov, BATCH_DT, 1, t0=n * BATCH_DT, pulse=pulse,
                                      mask=mask)
            inst[k] = (x, g, out, pulse, mask)
        if n >= warmup:
            el += time.perf_counter() - t0
    return gp, el


ORACLE_SAMPLE = 32          # instances of the batched configuration the oracle runs per step
ORACLE_SAMPLE_SEED = 1312


def oracle_sample_ids():
    """A seeded sample of the batched configuration's instances (the metric is
    per grid point, so a sample of the instances measures it)."""
    rng = np.random.default_rng(ORACLE_SAMPLE_SEED)
    return sorted(int(i) for i in rng.choice(BATCH_COUNT, ORACLE_SAMPLE, replace=False))


def oracle_batched(workers: int, steps: int, warmup: int):
    """The batched FP64 configuration on the serial oracle: a seeded sample of
    ORACLE_SAMPLE of its instances, spread over `workers` processes (spawned:
    the parent may hold a CUDA context) and balanced by grid points times
    Krylov dimension; one Lanczos step of every sampled instance per step.
    Returns grid-point steps of the sample / the slowest worker's time."""
    specs = W.batched_specs(BATCH_COUNT, BATCH_SEED)
    ids = oracle_sample_ids()
    sub = lpt_partition([specs[i].N * (specs[i].lmax + 1) * specs[i].krylov for i in ids], workers)
    parts = [[ids[k] for k in p] for p in sub]
    jobs = [(p, warmup, steps) for p in parts if p]
    if workers <= 1:
        res = [_oracle_batch_worker(j) for j in jobs]
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(len(jobs)) as pool:
            res = pool.map(_oracle_batch_worker, jobs)
    gp = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    return gp * steps / el, el, len(jobs)


def oracle_scale_sample(budget_s: float = 6.0):
    """The oracle on whole steps of the at-scale grid (Taylor-12, RK4,
    Lanczos-12 in FP64) until the time budget is used: grid-point steps/s."""
    import oracle
    g = oracle.Grid(N=CFG.N, h=CFG.dr, L=CFG.lmax, stencil=CFG.stencil)
    pulse = oracle.Pulse(CFG.E0, CFG.omega, CFG.ncycles)
    mask = oracle.Mask(CFG.R - CFG.absorber_width)
    rows = (("taylor", 12, CFG.dt_stable), ("rk4", 4, CFG.dt_stable), ("lanczos", 12, CFG.dt))
    psi = {m: start_state() for m, _, _ in rows}
    t0 = time.perf_counter()
    steps = 0
    while True:
        for name, order, dt in rows:
            psi[name], _ = oracle.propagate(g, psi[name], name, order, dt, 1, t0=0.3 * CFG.duration,
                                            pulse=pulse, mask=mask)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= 50:
            break
    return 3 * CFG.G * steps / el, steps, el


def oracle_small_us(nsteps=100):
    """The oracle on the small configuration: us per step of each method."""
    import oracle
    c = W.SMALL
    g = oracle.Grid(N=c.N, h=c.dr, L=c.lmax, stencil=c.stencil)
    pulse = oracle.Pulse(c.E0, c.omega, c.ncycles)
    psi = W.hydrogen_1s(c.N, c.dr, c.lmax)
    out = {}
    for method, order, dt in (("taylor", 8, 0.01), ("rk4", 4, 0.01), ("lanczos", 12, 0.05)):
        t0 = time.perf_counter()
        oracle.propagate(g, psi, method, order, dt, nsteps, pulse=pulse)
        out[f"{method}-{order}"] = 1e6 * (time.perf_counter() - t0) / nsteps
    return out


# ---------------------------------------------------------------------------
# Legs
# ---------------------------------------------------------------------------
def run_headline(D, args, ws):
    """The batched configuration in FP64 (the headline) and in mixed precision."""
    rows = {p: BatchRow(p, D.sptr, count=args.batch_count, schedule=args.schedule.get(p))
            for p in ("fp64", "mixed") if args.precision in ("all", p)}
    out = {}
    for p, r in rows.items():
        steps = args.steps if p == "fp64" else max(5, args.steps // 2)
        for _ in range(args.warmup):
            D.flush()
            r.step()
        D.sync()
        if ws > 1 and p == "fp64":
            D.torch.distributed.barrier()
        D.sync()
        sampler = ClockSampler(gpu_uuid(D.dev.index)) if p == "fp64" else None
        if sampler:
            sampler.start()
        l0, g0 = r.b.launches, r.b.graph_steps
        evs = D.events(steps)
        for s in range(steps):
            D.flush(s)
            evs[s][0].record(D.stream)
            r.step()
            evs[s][1].record(D.stream)
        D.sync()
        clocks = sampler.stop() if sampler else None
        ms = sum(a.elapsed_time(b) for a, b in evs)
        launches, graph_steps = r.b.launches - l0, r.b.graph_steps - g0
        r.b.observables(0)                          # raises on Inf/NaN
        ms_all, units_all = combine_over_ranks(ms, r.gp * steps, ws, D.dev) if p == "fp64" else (ms, r.gp * steps)
        prof = profile_rows(D, [r])
        e2e = e2e_rows(D, [r], 3, None) if not args.no_e2e else None
        out[p] = {"value": units_all / (ms_all * 1e-3), "ms_per_step": ms_all / steps, "steps": steps,
                  "warmup": args.warmup, "gp_per_step": r.gp, "gpu_launches": launches,
                  "launches_per_step": launches / steps, "graph_replayed_steps": graph_steps,
                  "roofline": dominant_roofline(D, prof, p), "e2e": e2e, "schedule": r.schedule,
                  "clocks": clocks,
                  "kernel_ms_share": {f"{k[2]}": round(v[0] / sum(x[0] for x in prof.values()), 4)
                                      for k, v in prof.items()}}
        r.close()
    return out


def run_scale(D, args, precision):
    """Config 2 (FP64) or config 3 (mixed): the three propagators on the
    at-scale grid, one step each per benchmark step."""
    psi0 = start_state()
    meths = [(m, o, dt) for m, o, dt in (("taylor", 12, CFG.dt_stable), ("rk4", 4, CFG.dt_stable),
                                         ("lanczos", 12, CFG.dt)) if args.method in ("all", m)]
    rows = [HandleRow(m, o, dt, precision, D.sptr, psi0) for m, o, dt in meths]
    steps = max(5, args.steps // 2)
    row_ms = time_rows(D, rows, steps, max(3, args.warmup // 2))
    for r in rows:
        r.h.sync()                                       # raises on Inf/NaN
    prof = profile_rows(D, rows)
    e2e = e2e_rows(D, rows, 2, psi0) if not args.no_e2e else None
    total = sum(row_ms.values())
    out = {"value": sum(r.gp for r in rows) * steps / (total * 1e-3), "ms_per_step": total / steps,
           "steps": steps, "rows_gp_steps_per_s": {r.name: r.gp * steps / (row_ms[r.name] * 1e-3) for r in rows},
           "rows_ms_per_step": {k: v / steps for k, v in row_ms.items()},
           "roofline": dominant_roofline(D, prof, precision), "e2e": e2e,
           "kernel_rooflines": {k[2]: roofline_of(D, k, prof) for k in prof
                                if (k[2] in KERNEL_FLOPS_PER_GP if precision == "fp64" else k[2] in MIXED_BYTES_PER_GP)}}
    for r in rows:
        r.close()
    return out


def run_hpsi(D, args, reps=20):
    """The operator alone (tdse_apply_h) on the at-scale grid: y = H(E) x on
    device buffers, L2 flushed before every launch, CUDA events around it."""
    torch = D.torch
    x = torch.from_numpy(start_state()).to(D.dev)
    y = torch.empty_like(x)
    out = {}
    for prec in ("fp64", "mixed"):
        h = make_handle(D.sptr, prec)
        for _ in range(3):
            h.apply_h(0.03, x.data_ptr(), y.data_ptr())
        D.sync()
        evs = D.events(reps)
        for k in range(reps):
            D.flush(k)
            evs[k][0].record(D.stream)
            h.apply_h(0.03, x.data_ptr(), y.data_ptr())
            evs[k][1].record(D.stream)
        D.sync()
        ms = sum(a.elapsed_time(b) for a, b in evs) / reps
        gbs = FP64_BYTES_PER_GP["apply_h"] * CFG.G / (ms * 1e-3) / 1e9 if prec == "fp64" else \
            MIXED_BYTES_PER_GP["apply_h"] * CFG.G / (ms * 1e-3) / 1e9
        o = {"us_per_call": 1e3 * ms, "gp_per_s": CFG.G / (ms * 1e-3), "hbm_gbs": gbs,
             "hbm_frac": gbs / HBM_PEAK_GBS}
        if prec == "fp64":
            tf = H5_FLOPS * CFG.G / (ms * 1e-3) / 1e12
            o.update({"tflops": tf, "alu_frac": tf / D.fp64_peak, "bound": "alu",
                      "algorithmic": f"{H5_FLOPS} flop and {FP64_BYTES_PER_GP['apply_h']} B per grid point"})
        else:
            o.update({"bound": "hbm", "algorithmic": f"{MIXED_BYTES_PER_GP['apply_h']} B per grid point "
                                                     "(x, FP32 diagonal, y); the call splits x into FP32 parts "
                                                     "first (a second launch)"})
        out[prec] = o
        h.close()
    out["workload"] = (f"at-scale grid (N={CFG.N} dr={CFG.dr} lmax={CFG.lmax} 5-point, {CFG.G} points), "
                       f"length gauge, {reps} calls, L2 flushed before each")
    return out


def run_small_config(D, nsteps=200, reps=3):
    """Config 1 (N=500, dr=0.2, lmax=4, 3-point; 2,500 grid points): us per
    step of each FP64 propagator, nsteps steps per call (one call timed by
    CUDA events, best of reps, L2 flushed before each), on the cluster path
    (the default for this size) and on the multi-launch path."""
    from paper_1308_1856_gb300 import TDSE
    c = W.SMALL
    psi0 = W.hydrogen_1s(c.N, c.dr, c.lmax)
    out = {"workload": f"small configuration N={c.N} dr={c.dr} lmax={c.lmax} {c.stencil}-point, FP64, "
                       f"{nsteps} steps per timed call, best of {reps}"}
    for path in ("cluster", "multi_launch"):
        res = {}
        for method, order, dt in (("taylor", 8, 0.01), ("rk4", 4, 0.01), ("lanczos", 12, 0.05)):
            t = TDSE(c.N, c.dr, c.lmax, stencil=c.stencil)
            t.set_pulse(c.E0, c.omega, c.ncycles)
            t.set_stream(D.sptr)
            t.set_small_grid_path("force" if path == "cluster" else "off")
            t.set_state(psi0)
            t.propagate(method, order, dt, 20)
            best = float("inf")
            l0 = t.launches
            for k in range(reps):
                D.flush(k)
                a, b = D.events(1)[0]
                a.record(D.stream)
                t.propagate(method, order, dt, nsteps)
                b.record(D.stream)
                D.sync()
                best = min(best, a.elapsed_time(b))
            assert t.small_grid_path_used == (path == "cluster")
            res[f"{method}-{order}"] = {"us_per_step": 1e3 * best / nsteps,
                                        "gp_steps_per_s": c.G * nsteps / (best * 1e-3),
                                        "launches_per_call": (t.launches - l0) / reps}
            t.close()
        out[path] = res
    return out


def _oracle_observables_series(args):
    """(oracle) d(t), populations and norm after each of nsteps Lanczos steps
    of one instance from a given state and time."""
    N, dr, L, m, dt, nsteps, t0, E0, omega, nc, ra, psi = args
    import oracle
    g = oracle.Grid(N=N, h=dr, L=L, stencil=5)
    pulse = oracle.Pulse(E0=E0, omega=omega, ncycles=nc)
    mask = oracle.Mask(ra) if ra is not None else None
    series = []
    x = psi
    for n in range(nsteps):
        x, _ = oracle.propagate(g, x, "lanczos", m, dt, 1, t0=t0 + n * dt, pulse=pulse, mask=mask)
        ob = oracle.observables(g, x, r_b=10.0)
        series.append((ob["norm"], ob["dipole"], ob["l_pop"]))
    return x, series


def _errors(gpu_series, gpu_state, ora_state, ora_series):
    """Errors of one run against the oracle: final state (relative L2), norm,
    populations (relative where P_l >= 1e-8, absolute below) and the dipole
    series d(t) (absolute, and relative to its largest value)."""
    dmax = max(abs(o[1]) for o in ora_series) or 1.0
    d_abs = max(abs(g[1] - o[1]) for g, o in zip(gpu_series, ora_series))
    pl_g, pl_o = gpu_series[-1][2], ora_series[-1][2]
    big = pl_o >= 1e-8
    return {"state_rel_l2": float(np.linalg.norm(gpu_state - ora_state) / np.linalg.norm(ora_state)),
            "norm_abs": max(abs(g[0] - o[0]) for g, o in zip(gpu_series, ora_series)),
            "l_pop_max_rel": float(np.max(np.abs(pl_g[big] - pl_o[big]) / pl_o[big])) if big.any() else 0.0,
            "l_pop_small_max_abs": float(np.max(np.abs(pl_g[~big] - pl_o[~big]))) if (~big).any() else 0.0,
            "dipole_series_max_abs": d_abs, "dipole_series_max_rel": d_abs / dmax, "steps": len(ora_series)}


def run_scale_accuracy(D, nsteps=6):
    """Config 3's error against the FP64 oracle: Lanczos-12 on the at-scale
    grid at a converging step (rho(H) dt = m/2), from the benchmark's start
    state at 0.3 T, mixed and FP64 GPU runs against the oracle after every
    step (norm, populations, dipole d(t))."""
    dt = W.converging_dt(CFG.N, CFG.dr, CFG.lmax, 12, CFG.stencil, CFG.E0)
    psi0 = start_state()
    t0 = 0.3 * CFG.duration
    ora_state, ora_series = _oracle_observables_series(
        (CFG.N, CFG.dr, CFG.lmax, 12, dt, nsteps, t0, CFG.E0, CFG.omega, CFG.ncycles, CFG.R - CFG.absorber_width,
         psi0))
    out = {"workload": f"at-scale grid, Lanczos-12, dt={dt:.4g} (rho(H) dt = m/2), {nsteps} steps from the "
                       "start state at 0.3 T; errors against the FP64 oracle after every step"}
    for prec in ("mixed", "fp64"):
        h = make_handle(D.sptr, prec)
        h.set_state(psi0)
        h.time = t0
        ser = []
        for n in range(nsteps):
            h.propagate("lanczos", 12, dt, 1)
            ob = h.observables()
            ser.append((ob["norm"], ob["dipole"], ob["l_pop"]))
        out[prec] = _errors(ser, h.get_state(), ora_state, ora_series)
        h.close()
    return out


def run_batched_converged(D, args, nsteps_acc=8, timed_steps=5):
    """Config 4 at a converging step: every instance's dt with rho(H) dt = m/2
    (W.converging_dt).  Throughput of the 256-instance batch in FP64 and mixed
    precision, and the errors of both against the FP64 oracle on sampled
    instances (the 4 smallest and 4 seeded others of at most 5e5 points)
    advanced from smooth states at 0.37 of their pulse (the same launches
    whatever else is in the batch: an instance's result is the same alone and
    in the mix, bitwise)."""
    specs = W.batched_specs(BATCH_COUNT, BATCH_SEED)
    dts = [W.converging_dt(x.N, x.dr, x.lmax, x.krylov, 5, x.E0) for x in specs]
    out = {"workload": "batched configuration, per-instance dt with rho(H) dt = m/2 "
                       f"({min(dts):.3g}..{max(dts):.3g})"}
    for prec in ("fp64", "mixed"):
        r = BatchRow(prec, D.sptr, count=args.batch_count, schedule=args.schedule.get(prec), dts=dts)
        ms = time_rows(D, [r], timed_steps, 3)[r.name]
        out[prec] = {"value": r.gp * timed_steps / (ms * 1e-3), "ms_per_step": ms / timed_steps}
        r.close()
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    # accuracy on sampled instances
    G = [x.N * (x.lmax + 1) for x in specs]
    order = sorted(range(len(specs)), key=lambda i: G[i])
    rng = np.random.default_rng(1311)
    pool = [i for i in order[4:] if G[i] <= 500_000]
    sample = order[:4] + [int(i) for i in rng.choice(pool, 4, replace=False)]
    jobs, t0s, psis = [], [], []
    for i in sample:
        x = specs[i]
        T = 2 * math.pi * x.ncycles / x.omega
        t0s.append(0.37 * T)
        psis.append(W.smooth_state(x.N, x.dr, x.lmax, seed=50 + i, lmax_populated=20))
        jobs.append((x.N, x.dr, x.lmax, x.krylov, dts[i], nsteps_acc, t0s[-1], x.E0, x.omega, x.ncycles,
                     x.N * x.dr - BATCH_ABSORBER, psis[-1]))
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(len(jobs)) as pool_:
        ora = pool_.map(_oracle_observables_series, jobs)
    from paper_1308_1856_gb300 import Batch
    acc = {"instances": sample, "steps": nsteps_acc}
    for prec in ("fp64", "mixed"):
        b = Batch([batched_request_spec(specs[i], dts[i]) for i in sample], stencil=5, precision=prec)
        b.set_stream(D.sptr)
        for k in range(len(sample)):
            b.set_state(k, psis[k])
            b.set_time(k, t0s[k])
        sers = [[] for _ in sample]
        for n in range(nsteps_acc):
            b.propagate(1)
            for k in range(len(sample)):
                ob = b.observables(k)
                sers[k].append((ob["norm"], ob["dipole"], ob["l_pop"]))
        errs = [_errors(sers[k], b.get_state(k), ora[k][0], ora[k][1]) for k in range(len(sample))]
        b.close()
        acc[prec] = {key: max(e[key] for e in errs) for key in errs[0] if key != "steps"}
    out["errors_vs_oracle"] = acc
    return out


def serve_trace(sptr, precision, rate, count, horizon, kbatch, budget, seed):
    """Continuous batching of a finite Poisson trace through the server: each
    request is one instance of the batched configuration (seeded draws) run for
    `horizon` Lanczos steps from t = 0; the loop admits what has arrived and
    fits, runs one step batch of `kbatch` steps over every running request,
    waits for it, and retires what finished.  Time-to-completion = the end of
    the step batch in which a request took its last step minus its arrival."""
    from paper_1308_1856_gb300 import Server
    specs = [batched_request_spec(x) for x in W.batched_specs(count, seed)]
    arrivals = W.poisson_arrivals(count, rate, seed + 1)
    srv = Server(budget, max_resident=count, stencil=5, precision=precision)
    srv.set_stream(sptr)
    st0 = srv.stats()
    arrived, lat, resident_peak, batches = {}, [], 0, 0
    nxt = 0
    t0 = time.perf_counter()
    while len(lat) < count:
        now = time.perf_counter() - t0
        while nxt < count and arrivals[nxt] <= now:
            arrived[srv.submit(specs[nxt], horizon)] = arrivals[nxt]
            nxt += 1
        st = srv.stats()
        if st["running"] == 0 and st["queued"] == 0:
            time.sleep(max(0.0, arrivals[nxt] - now))
            continue
        srv.step(kbatch)
        srv.sync()
        batches += 1
        done = time.perf_counter() - t0
        resident_peak = max(resident_peak, srv.stats()["resident"])
        for rid in srv.poll():
            lat.append(done - arrived.pop(rid))
            srv.observables(rid)                 # the result a client reads (raises on Inf/NaN)
            srv.release(rid)
    makespan = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat = np.array(lat)
    return {"rate_req_per_s": rate, "requests": count, "horizon_steps": horizon, "step_batch": kbatch,
            "precision": precision, "hbm_budget_bytes": budget,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "makespan_s": makespan,
            "gp_steps_per_s": (st["gp_steps"] - st0["gp_steps"]) / makespan,
            "resident_peak": resident_peak, "step_batches": batches,
            "gpu_launches": st["launches"] - st0["launches"]}


def run_served(args, sptr):
    """Config 5: an overloaded trace (mean 50 req/s) and one at a rate the GPU
    sustains, both through the same server."""
    budget = int(args.serve_budget_gb * (1 << 30))
    out = {"workload": "served: Poisson arrivals, specs drawn as in the batched configuration "
                       f"(seed {args.serve_seed}), each request {args.serve_horizon} Lanczos steps "
                       f"(dt {BATCH_DT}) from t = 0, step batches of {args.serve_batch}, HBM budget "
                       f"{args.serve_budget_gb:g} GB, FIFO admission"}
    precs = ["fp64", "mixed"] if args.serve_precision == "both" else [args.serve_precision]
    for prec in precs:
        for name, rate, count in (("overload", args.serve_rate, args.serve_requests),
                                  ("sustained", args.serve_sustained_rate, args.serve_sustained_requests)):
            if count > 0:
                out[f"{name}_{prec}"] = serve_trace(sptr, prec, rate, count, args.serve_horizon, args.serve_batch,
                                                    budget, args.serve_seed)
    return out


# Stage counts of the explicit Runge-Kutta tableaus (appendix "Runge-Kutta"),
# and the first-same-as-last one (its last stage's argument is the new state).
RK_STAGES = {"euler": 1, "classic": 4, "fehlberg": 6, "cash_karp": 6, "dormand_prince": 7, "merson": 5}
RK_FSAL = ("dormand_prince",)


def rk_step_flops_per_gp(s: int, fsal: bool = False) -> int:
    """Algorithmic FP64 flops per grid point of one step of an s-stage explicit
    RK method through the general stage kernel (5-point stencil, FMA = 2):
    stage i < s-1 applies H and forms g_{i+1} from psi and i+1 slopes
    (4 (i+1)); the last applies H, forms psi (unless first-same-as-last) and
    Delta from s slopes (4 s each) and adds |Delta|^2 (4)."""
    return s * H5_FLOPS + sum(4 * (i + 1) for i in range(s - 1)) + (4 if fsal else 8) * s + 4


def run_rk_pairs(D, steps=5, warmup=3, tableaus=("dormand_prince", "fehlberg")):
    """Embedded RK pairs on the at-scale grid (FP64, dt = the explicit
    propagators' stable step): per-step time with L2 flushed before every
    step, and the general stage kernel against the FP64 peak."""
    psi0 = start_state()
    out = {"workload": "scale grid (N=8000 dr=0.05 lmax=63 5-point, mask), FP64, "
                       f"dt={CFG.dt_stable:g}, L2 flushed before every step"}
    for tb in tableaus:
        s = RK_STAGES[tb]
        h = make_handle(D.sptr, "fp64")
        h.set_state(psi0)
        h.time = 0.3 * CFG.duration
        for _ in range(warmup):
            h.propagate_rk(tb, CFG.dt_stable, 1)
        evs = D.events(steps)
        sigma = 0.0
        for k in range(steps):
            D.flush(k)
            evs[k][0].record(D.stream)
            sigma += h.propagate_rk(tb, CFG.dt_stable, 1)
            evs[k][1].record(D.stream)
        D.sync()
        ms = sum(a.elapsed_time(b) for a, b in evs) / steps
        h.profile(True)
        for k in range(steps):
            D.flush(k)
            h.propagate_rk(tb, CFG.dt_stable, 1)
        kms, n = h.profile_read().get("rk_stage", (0.0, 0))
        h.profile(False)
        h.close()
        flops = rk_step_flops_per_gp(s, tb in RK_FSAL) * CFG.G * steps
        achieved = flops / (kms * 1e-3) / 1e12 if kms > 0 else None
        out[tb] = {"stages": s, "ms_per_step": ms, "gp_steps_per_s": CFG.G / (ms * 1e-3),
                   "sigma_per_step": sigma / steps,
                   "roofline": {"bound": "alu", "kernel": "rk_general_stage (single, fp64)", "achieved": achieved,
                                "peak": D.fp64_peak, "unit": "TFLOP/s",
                                "frac": None if achieved is None else achieved / D.fp64_peak,
                                "flops_per_launch": flops / max(n, 1), "avg_launch_ms": kms / max(n, 1),
                                "launches": n}}
    return out


def run_step_observables(D, steps=5, warmup=3, ntheta=180, r_b=10.0):
    """Sec. 4 observables recorded after every step on the at-scale grid
    (FP64 Lanczos-12, dt = 0.02): the dipole series and the flux through r_b
    with its density at ntheta angles and their time integrals.  Per-step time
    with and without them, and the dipole kernel against the FP64 peak."""
    psi0 = start_state()
    ct = np.cos((np.arange(ntheta) + 0.5) * np.pi / ntheta)
    out = {"workload": f"scale grid, FP64 Lanczos-12 dt={CFG.dt:g}; dipole series + flux at r_b={r_b:g} with "
                       f"{ntheta} angles after every step; L2 flushed before every step"}
    for label, hooks in (("without", False), ("with", True)):
        h = make_handle(D.sptr, "fp64")
        h.set_state(psi0)
        h.time = 0.3 * CFG.duration
        if hooks:
            h.record_dipole(steps + warmup + 8)
            h.flux_setup(r_b, ct)
        for _ in range(warmup):
            h.propagate("lanczos", 12, CFG.dt, 1)
        evs = D.events(steps)
        for k in range(steps):
            D.flush(k)
            evs[k][0].record(D.stream)
            h.propagate("lanczos", 12, CFG.dt, 1)
            evs[k][1].record(D.stream)
        D.sync()
        out[f"ms_per_step_{label}"] = sum(a.elapsed_time(b) for a, b in evs) / steps
        if hooks:
            h.profile(True)
            for k in range(3):
                D.flush(k)
                h.propagate("lanczos", 12, CFG.dt, 1)
            prof = h.profile_read()
            h.profile(False)
            dms, dn = prof.get("dipole", (0.0, 0))
            fms, fn = prof.get("flux", (0.0, 0))
            flops = DIPOLE_FLOPS_PER_GP * CFG.G
            ach = flops / (dms / dn * 1e-3) / 1e12 if dn else None
            out["dipole_kernel"] = {"bound": "alu", "achieved": ach, "peak": D.fp64_peak, "unit": "TFLOP/s",
                                    "frac": None if ach is None else ach / D.fp64_peak,
                                    "avg_launch_ms": dms / max(dn, 1), "launches": dn}
            out["flux_kernel_avg_ms"] = fms / max(fn, 1)
        h.close()
    out["overhead_frac"] = out["ms_per_step_with"] / out["ms_per_step_without"] - 1.0
    return out


def run_batched_observables(D, args, steps=5, warmup=3, ntheta=180):
    """The batched configuration (FP64) with the Sec. 4 output of every
    instance after every step (the dipole series and the flux through each
    instance's r_b with ntheta angles), against the same steps without it;
    and imaginary-time steps of the whole batch (dtau = each instance's dt,
    Sec. 3).  L2 flushed before every step."""
    r = BatchRow("fp64", D.sptr, count=args.batch_count, schedule=args.schedule.get("fp64"))
    b = r.b
    ct = np.cos((np.arange(ntheta) + 0.5) * np.pi / ntheta)
    out = {"workload": f"batched configuration, FP64; dipole series + flux at each r_b with {ntheta} angles "
                       f"after every step; imaginary-time steps of the same batch; L2 flushed before every step",
           "gp_per_step": r.gp}

    def timed(call):
        for _ in range(warmup):
            D.flush()
            call()
        D.sync()
        evs = D.events(steps)
        for k in range(steps):
            D.flush(k)
            evs[k][0].record(D.stream)
            call()
            evs[k][1].record(D.stream)
        D.sync()
        return sum(a.elapsed_time(c) for a, c in evs) / steps

    out["ms_per_step_without"] = timed(r.step)
    b.record_dipole(2 * (steps + warmup) + 8)
    b.flux_setup(ct)
    out["ms_per_step_with"] = timed(r.step)
    out["overhead_frac"] = out["ms_per_step_with"] / out["ms_per_step_without"] - 1.0
    b.profile(True)
    for k in range(2):
        D.flush(k)
        r.step()
    prof = b.profile_read()
    b.profile(False)
    dms, dn = prof.get("dipole", (0.0, 0))
    fms, fn = prof.get("flux", (0.0, 0))
    if dn:
        ach = DIPOLE_FLOPS_PER_GP * r.gp / (dms / dn * 1e-3) / 1e12
        out["dipole_kernel"] = {"bound": "alu", "kernel": "bt_dipole (batched, fp64)", "achieved": ach,
                                "peak": D.fp64_peak, "unit": "TFLOP/s", "frac": ach / D.fp64_peak,
                                "avg_launch_ms": dms / dn, "launches": dn}
    out["flux_kernel_avg_ms"] = fms / max(fn, 1)
    ser = b.dipole_series(0)
    out["series_entries_instance0"] = int(ser.shape[0])
    b.record_dipole(0)
    b.flux_setup(enable=False)
    from paper_1308_1856_gb300 import _binding as C
    ms_imag = timed(lambda: C.tdse_batch_propagate_imag(b.h, 1, None))   # asynchronous: no energies read
    e = b.propagate_imag(1)
    out["imag"] = {"ms_per_step": ms_imag, "gp_steps_per_s": r.gp / (ms_imag * 1e-3),
                   "energy_range": [float(np.nanmin(e)), float(np.nanmax(e))]}
    r.close()
    return out


def run_probe(D):
    """FP64 and FP32 FMA throughput of this GPU (tdse_fma_throughput)."""
    from paper_1308_1856_gb300 import fma_throughput
    sampler = ClockSampler(gpu_uuid(D.dev.index))
    sampler.start()
    f64 = max(fma_throughput(True, D.sptr) for _ in range(5)) / 1e12
    f32 = max(fma_throughput(False, D.sptr) for _ in range(3)) / 1e12
    clocks = sampler.stop()
    clk = SM_MAX_MHZ * 1e6
    return {"fp64_tflops": f64, "fp32_tflops": f32, "clocks": clocks,
            "fp64_fma_per_clk_per_sm_at_max_clock": f64 * 1e12 / 2 / D.sms / clk,
            "fp32_fma_per_clk_per_sm_at_max_clock": f32 * 1e12 / 2 / D.sms / clk,
            "fp64_peak_derived_tflops": D.fp64_peak, "sms": D.sms}


def compact(res):
    """The per-configuration summary printed last on the line (short enough
    to survive a truncated log)."""
    def roof(r):
        if not r:
            return None
        o = {"k": r["kernel"], "bound": r["bound"], "frac": sig(r["frac"], 3)}
        if "hbm_frac" in r:
            o["hbm_frac"] = sig(r["hbm_frac"], 3)
        return o
    out = {}
    hl = res.get("batched", {})
    if "fp64" in hl:
        b = hl["fp64"]
        out["c4_batched_f64"] = {"gps": sig(b["value"]), "ms": sig(b["ms_per_step"]), "roof": roof(b["roofline"]),
                                 "e2e_gps": sig((b["e2e"] or {}).get("value")),
                                 "launches_per_step": sig(b["launches_per_step"], 3),
                                 "graph_steps": b["graph_replayed_steps"]}
    if "mixed" in hl:
        b = hl["mixed"]
        out["c4_batched_mixed"] = {"gps": sig(b["value"]), "ms": sig(b["ms_per_step"]),
                                   "roof": roof(b["roofline"]), "e2e_gps": sig((b["e2e"] or {}).get("value"))}
    if "batched_converged" in res:
        c = res["batched_converged"]
        e = c["errors_vs_oracle"]
        out["c4_converged"] = {"f64_gps": sig(c["fp64"]["value"]), "mixed_gps": sig(c["mixed"]["value"]),
                               "mixed_over_f64": sig(c["mixed_over_fp64"], 3),
                               "mixed_err": {k: sig(v, 2) for k, v in e["mixed"].items()},
                               "f64_err_state": sig(e["fp64"]["state_rel_l2"], 2)}
    for key, name in (("scale_fp64", "c2_scale_f64"), ("scale_mixed", "c3_scale_mixed")):
        if key in res:
            s = res[key]
            out[name] = {"gps": sig(s["value"]), "rows_gps": {k.split("/")[0]: sig(v) for k, v in
                                                              s["rows_gp_steps_per_s"].items()},
                         "roof": roof(s["roofline"]), "e2e_gps": sig((s["e2e"] or {}).get("value"))}
    if "scale_accuracy" in res:
        out.setdefault("c3_scale_mixed", {})["err_vs_oracle"] = {
            k: sig(v, 2) for k, v in res["scale_accuracy"]["mixed"].items() if k != "steps"}
    if "small_config" in res:
        s = res["small_config"]
        out["c1_small_us"] = {p: {k: sig(v["us_per_step"], 3) for k, v in s[p].items()}
                              for p in ("cluster", "multi_launch") if p in s}
    if "served" in res:
        out["c5_served"] = {k: {"p50": sig(v["p50_s"], 3), "p99": sig(v["p99_s"], 3),
                                "gps": sig(v["gp_steps_per_s"], 3)}
                            for k, v in res["served"].items() if isinstance(v, dict)}
    if "hpsi" in res:
        h = res["hpsi"]
        out["hpsi"] = {"f64": {"us": sig(h["fp64"]["us_per_call"], 3), "alu_frac": sig(h["fp64"]["alu_frac"], 3),
                               "hbm_frac": sig(h["fp64"]["hbm_frac"], 3)},
                       "mixed": {"us": sig(h["mixed"]["us_per_call"], 3), "hbm_frac": sig(h["mixed"]["hbm_frac"], 3)}}
    if "batched_observables" in res:
        o = res["batched_observables"]
        out["c4_batched_obs"] = {"overhead_frac": sig(o["overhead_frac"], 3),
                                 "dipole_frac": sig((o.get("dipole_kernel") or {}).get("frac"), 3),
                                 "imag_gps": sig(o["imag"]["gp_steps_per_s"])}
    if "fp64_probe" in res:
        out["fp64_probe_tflops"] = sig(res["fp64_probe"]["fp64_tflops"], 4)
    if "cpu_baselines" in res:
        out["cpu_oracle"] = {k: sig(v["value"], 3) for k, v in res["cpu_baselines"].items()}
    return out


def run_ours(args, ws, rank, local):
    D = Device(local)
    res = {}
    legs = args.rows
    if legs in ("all", "probe"):
        res["fp64_probe"] = run_probe(D)
    if legs in ("all", "headline", "batched"):
        res["batched"] = run_headline(D, args, ws)
    if legs == "headline":
        return D, res
    if legs in ("all", "single"):
        if args.precision in ("all", "fp64"):
            res["scale_fp64"] = run_scale(D, args, "fp64")
        if args.precision in ("all", "mixed"):
            res["scale_mixed"] = run_scale(D, args, "mixed")
    if legs in ("all", "hpsi"):
        res["hpsi"] = run_hpsi(D, args)
    if legs in ("all", "small"):
        res["small_config"] = run_small_config(D)
    if legs in ("all", "accuracy"):
        res["scale_accuracy"] = run_scale_accuracy(D)
    if legs in ("all", "converged"):
        res["batched_converged"] = run_batched_converged(D, args)
    if legs in ("all", "rk"):
        res["rk_pairs"] = run_rk_pairs(D)
    if legs in ("all", "obs"):
        res["step_observables"] = run_step_observables(D)
    if legs in ("all", "batch_obs"):
        res["batched_observables"] = run_batched_observables(D, args)
    if legs in ("all", "served") and not args.no_serve:
        res["served"] = run_served(args, D.sptr)
    return D, res


def reference_line(args, ws):
    """The reference arm: the serial oracle (the paper's algorithms as
    written) on the host cores, on the headline's workload."""
    cores = host_cores()
    warm = max(0, args.warmup)
    v, el, used = oracle_batched(cores, args.steps, warm)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": warm, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": headline_workload(), "grid_points_per_step": batched_points()},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": f"a seeded sample of {ORACLE_SAMPLE} of the {BATCH_COUNT} instances (seed "
                                       f"{ORACLE_SAMPLE_SEED}; {sample_points()} grid points), one Lanczos step "
                                       f"of each per step, spread over {used} serial oracle processes, {warm} "
                                       f"untimed + {args.steps} timed steps, {el:.1f} s for the timed ones"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


def sample_points():
    specs = W.batched_specs(BATCH_COUNT, BATCH_SEED)
    return sum(specs[i].N * (specs[i].lmax + 1) for i in oracle_sample_ids())


def batched_points():
    return sum(x.N * (x.lmax + 1) for x in W.batched_specs(BATCH_COUNT, BATCH_SEED))


def headline_workload():
    return (f"batched FP64: {BATCH_COUNT} instances (seed {BATCH_SEED}, N 2000-16000, dr 0.1, lmax 15-127, "
            f"Krylov 8-16, 5-point, dt {BATCH_DT}, cos^(1/8) mask over the last {BATCH_ABSORBER:g} a.u.), "
            "one Lanczos step of every instance per step")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end legs (profiling runs)")
    ap.add_argument("--e2e-groups", type=int, default=None,
                    help="instance groups of the batched rows' pipelined copies in the end-to-end leg")
    ap.add_argument("--method", default="all", choices=["all", "taylor", "rk4", "lanczos"],
                    help="restrict the at-scale rows to one propagator (profiling runs)")
    ap.add_argument("--precision", default="all", choices=["all", "fp64", "mixed"],
                    help="restrict the batched and at-scale rows to one precision (profiling runs)")
    ap.add_argument("--rows", default="all",
                    choices=["all", "headline", "batched", "single", "hpsi", "small", "accuracy", "converged",
                             "served", "rk", "obs", "batch_obs", "probe"],
                    help="run one leg only (headline: the batched FP64 and mixed rows without the other legs)")
    ap.add_argument("--batch-count", type=int, default=BATCH_COUNT,
                    help="instances of the batched rows (smaller only for profiling captures)")
    ap.add_argument("--schedule", action="append", default=[], metavar="PREC=PF,RING,SB,EB",
                    help="fixed launch schedule of a batched row instead of autotuning (profiling runs): "
                         "prefetch rows, ring rows, stencil and elementwise blocks per SM")
    ap.add_argument("--no-serve", action="store_true", help="skip the served traces")
    ap.add_argument("--serve-precision", default="both", choices=["fp64", "mixed", "both"])
    ap.add_argument("--serve-rate", type=float, default=50.0, help="overloaded trace: mean req/s")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-sustained-rate", type=float, default=2.0)
    ap.add_argument("--serve-sustained-requests", type=int, default=32)
    ap.add_argument("--serve-horizon", type=int, default=500, help="Lanczos steps per request")
    ap.add_argument("--serve-batch", type=int, default=100, help="steps per step batch")
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-seed", type=int, default=1309)
    args = ap.parse_args()
    if args.e2e_groups is not None:
        globals()["E2E_GROUPS"] = max(1, args.e2e_groups)
    sched = {}
    for item in args.schedule:
        prec, vals = item.split("=")
        sched[prec] = tuple(int(v) for v in vals.split(","))
    args.schedule = sched
    ws, rank, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(reference_line(args, ws)))
        return 0
    if ws > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    from oracle import build as ob
    D, res = run_ours(args, ws, rank, local)
    if rank == 0:
        cpu = {}
        if not args.no_cpu_baseline and args.rows in ("all", "headline", "batched"):
            ob.build()
            cores = host_cores()
            v, el, used = oracle_batched(cores, 1, 0)
            cpu["c4_batched_f64"] = {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
                                     "sample": f"one Lanczos step of a seeded sample of {ORACLE_SAMPLE} of the "
                                               f"{BATCH_COUNT} instances ({sample_points()} grid points) spread "
                                               f"over {used} serial oracle processes, {el:.1f} s"}
            if args.rows == "all":
                v2, st2, el2 = oracle_scale_sample()
                cpu["c2_scale_f64"] = {"value": v2, "unit": UNIT, "cores": 1, "kind": "oracle",
                                       "sample": f"{st2} steps each of Taylor-12, RK4 and Lanczos-12 on the "
                                                 f"at-scale grid in {el2:.1f} s, serial"}
                us = oracle_small_us()
                cpu["c1_small"] = {"value": W.SMALL.G / (1e-6 * us["lanczos-12"]), "unit": UNIT, "cores": 1,
                                   "kind": "oracle", "us_per_step": us,
                                   "sample": "100 steps of each method on the small configuration, serial"}
        res["cpu_baselines"] = cpu
        head = res.get("batched", {}).get("fp64")
        line = {"metric": METRIC}
        if head:
            line.update({
                "value": head["value"], "unit": UNIT, "n_gpus": ws, "steps": head["steps"],
                "warmup": head["warmup"], "ms_per_step": head["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": headline_workload(), "grid_points_per_step": head["gp_per_step"],
                           "path": "tdse_batch_propagate(1) per step: a replay of the captured step graph",
                           "parallelism": f"replicas x{ws}",
                           "l2": "flushed (256 MB write) before every timed step; the states (36 GB) exceed L2"},
                "roofline": head["roofline"], "cpu_baseline": cpu.get("c4_batched_f64"),
                "clocks": head["clocks"], "e2e": head["e2e"], "gpu_launches": head["gpu_launches"]})
        line.update({k: v for k, v in res.items() if k not in ("cpu_baselines",)})
        line["cpu_baselines"] = cpu
        line["configs"] = compact(res)
        print(json.dumps(line))
    if ws > 1:
        import torch
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
