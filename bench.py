"""Throughput benchmark of the FD-TDSE hot path.

One benchmark step advances every row by one time step:
- six at-scale single-instance rows: hydrogen, N = 8000 radial points,
  dr = 0.05 a.u. (box 400), lmax = 63, 5-point stencil, complex128 state,
  sin^2 pulse (E0 = 0.0534, omega = 0.057, 4 cycles), cos^(1/8) mask over the
  last 50 a.u.; Taylor order 12, classic RK4 and Lanczos with Krylov
  dimension 12, each in FP64 and in mixed precision (FP32 stencil, FP64
  state/dots/norms/expm).  Lanczos runs at dt = 0.02; the explicit Taylor/RK4
  propagators are unstable at that dt on this grid (rho(H) dt ~ 1.6e4), so
  they run at their stable dt = 4e-6 -- the work per step does not depend on dt;
- two batched rows: 256 seeded uneven instances (N 2000-16000, dr = 0.1,
  lmax 15-127, Krylov dimension 8-16, dt = 0.02), one Lanczos step each, in
  FP64 and in mixed precision, with an autotuned launch schedule.
Metric: grid-point * steps per second summed over the rows (335.5 M grid
points per benchmark step).  Further legs: end to end through the C ABI with
host buffers, the served traces, the embedded RK pairs, the per-step
observables, the small configuration and the serial oracle on the host cores.

L2 (129 MB) is flushed before every timed row by writing a 256 MB buffer;
each row is timed by CUDA events on the library's stream (the flush sits
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
ALL_METHODS = [(m, o, dt, p) for p in ("fp64", "mixed")
               for m, o, dt in (("taylor", 12, CFG.dt_stable), ("rk4", 4, CFG.dt_stable),
                                ("lanczos", 12, CFG.dt))]
METHODS = list(ALL_METHODS)
HBM_PEAK_GBS = 6783.1       # measured copy bandwidth of this GB300 pool (MEASURED_PEAKS.json)
METRIC = "grid-point*steps/s"
BATCH_DT = 0.02            # the batched configuration states no step; that of the at-scale one
BATCH_ABSORBER = 50.0      # nor an absorber; the same cos^(1/8) mask over the last 50 a.u.
E2E_GROUPS = 4             # instance groups whose copies overlap the others' compute (e2e leg)
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
# Dipole moments kernel, per grid point: |f|^2 (4), w Re(f_l^* f_{l+1}) (5),
# the unscaled first derivative (8), w Im(f_{l+1}^* D1 f_l) (5) and
# w (l+1) Im(f_{l+1}^* f_l) (5).
DIPOLE_FLOPS_PER_GP = 27
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


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per algorithmic
# grid point of one launch, from the ncu captures summarised under profiles/:
# the batched kernels on the first 16 instances of the batched configuration
# (phases where all 16 are active, 10.66M points per launch), scaled here to a
# full launch by its points; the single-instance kernels on the at-scale grid
# (512000 points).  An entry is removed when its kernel changes after capture.
MEASURED_TRAFFIC_PER_POINT = {
    ("batched", "fp64", "lanczos_a"): (537.5e6 + 165.8e6) / 10664737,
    ("batched", "fp64", "lanczos_b"): (343.0e6 + 138.5e6) / 10664737,
    ("batched", "mixed", "lanczos_a"): (296.7e6 + 66.7e6) / 10664737,
    ("batched", "mixed", "lanczos_b"): (171.2e6 + 52.7e6) / 10664737,
    ("single", "fp64", "taylor_stage"): 20.6e6 / 512000,
}


def make_handle(stream_ptr: int, precision: str = "fp64"):
    from paper_1308_1856_gb300 import TDSE
    t = TDSE(CFG.N, CFG.dr, CFG.lmax, stencil=CFG.stencil)
    t.set_options(absorber=True, absorber_r=CFG.R - CFG.absorber_width, r_b=10.0,
                  precision=precision)
    t.set_pulse(CFG.E0, CFG.omega, CFG.ncycles)
    t.set_stream(stream_ptr)
    return t


class HandleRow:
    """One single-instance propagator on the at-scale grid."""
    kind = "single"

    def __init__(self, method, order, dt, prec, stream_ptr, psi0):
        self.method, self.order, self.dt, self.prec = method, order, dt, prec
        self.name = f"{method}-{order}/{prec}"
        self.h = make_handle(stream_ptr, prec)
        self.h.set_state(psi0)
        self.h.time = 0.3 * CFG.duration
        self.gp = CFG.G
        self.e2e_bytes = (CFG.G * 16, CFG.G * 16 + 8 * (CFG.lmax + 5))

    def step(self):
        self.h.propagate(self.method, self.order, self.dt, 1)

    # algorithmic grid points processed by each launch of a kernel kind, per step
    def kernel_points(self, kind):
        if kind in ("lanczos_a",):
            return self.order * self.gp
        if kind == "lanczos_b":
            return (self.order - 1) * self.gp
        if kind in ("taylor_stage",):
            return self.order * self.gp
        if kind == "rk_stage":
            return 4 * self.gp
        return self.gp

    def e2e_step(self, pin_in, pin_out, times):
        t0 = time.perf_counter()
        self.h.set_state_ptr(pin_in[0].data_ptr())
        t1 = time.perf_counter()
        self.step()
        self.h.get_state_ptr(pin_out[0].data_ptr())
        t2 = time.perf_counter()
        obs = self.h.observables()
        times += np.array([t1 - t0, t2 - t1, time.perf_counter() - t2])
        return obs


class BatchRow:
    """The batched configuration: 256 uneven instances (seed 1308), one Lanczos
    step of every instance per benchmark step."""
    kind = "batched"

    def __init__(self, prec, stream_ptr, count=256, schedule=None):
        from paper_1308_1856_gb300 import Batch
        self.specs = W.batched_specs(count, 1308)
        self.prec = prec
        self.name = f"batched-{count}/{prec}"
        d = [dict(N=x.N, dr=x.dr, lmax=x.lmax, krylov=x.krylov, dt=BATCH_DT, E0=x.E0, omega=x.omega,
                  ncycles=x.ncycles, absorber_r=x.N * x.dr - BATCH_ABSORBER) for x in self.specs]
        self.b = Batch(d, stencil=5, precision=prec)
        self.b.set_stream(stream_ptr)
        if schedule is None:
            self.schedule = self.b.autotune()     # before the warm-up; not timed
        else:                                     # a fixed schedule (profiling runs)
            pf, ring, sb, eb = schedule
            self.b.set_schedule(pf, sb, eb, ring_rows=ring)
            self.schedule = self.b.schedule()
        self.gp = self.b.points
        self.G = [x.N * (x.lmax + 1) for x in self.specs]
        self.e2e_bytes = (self.gp * 16, self.gp * 16)

    def step(self):
        self.b.propagate(1)

    def kernel_points(self, kind):
        m = [x.krylov for x in self.specs]
        if kind == "lanczos_a":
            return sum(g * mi for g, mi in zip(self.G, m))
        if kind == "lanczos_b":
            return sum(g * (mi - 1) for g, mi in zip(self.G, m))
        return self.gp

    @property
    def h(self):
        return self.b

    def e2e_step(self, pin_in, pin_out, times):
        # every state in, one step, every state out, the copies of one group of
        # instances overlapping the compute of another (tdse_batch_propagate_io)
        t0 = time.perf_counter()
        self.b.propagate_io(pin_in[0].data_ptr(), pin_out[0].data_ptr(), 1, groups=E2E_GROUPS)
        t1 = time.perf_counter()
        obs = self.b.observables(0)
        times += np.array([0.0, t1 - t0, time.perf_counter() - t1])
        return obs


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


def batched_request_spec(x, dt=BATCH_DT):
    return dict(N=x.N, dr=x.dr, lmax=x.lmax, krylov=x.krylov, dt=dt, E0=x.E0, omega=x.omega,
                ncycles=x.ncycles, absorber_r=x.N * x.dr - BATCH_ABSORBER)


def serve_trace(stream_ptr, precision, rate, count, horizon, kbatch, budget, seed):
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
    srv.set_stream(stream_ptr)
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


def run_served(args, stream_ptr):
    """Config 'served': an overloaded trace (mean 50 req/s) and one at a rate
    the GPU sustains, both through the same server."""
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
                key = name if len(precs) == 1 else f"{name}_{prec}"
                out[key] = serve_trace(stream_ptr, prec, rate, count, args.serve_horizon, args.serve_batch,
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


def run_rk_pairs(stream_ptr, psi0, steps=5, warmup=3, tableaus=("dormand_prince", "fehlberg")):
    """Embedded RK pairs on the at-scale grid (FP64, dt = the explicit
    propagators' stable step): per-step time by CUDA events on the library's
    stream with L2 flushed (256 MB write) before every step (the flush outside
    the events), and the general stage kernel against the FP64 ALU peak from a
    separate profiled pass."""
    import torch
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {"workload": "scale grid (N=8000 dr=0.05 lmax=63 5-point, mask), FP64, "
                       f"dt={CFG.dt_stable:g}, L2 flushed before every step"}
    for tb in tableaus:
        s = RK_STAGES[tb]
        h = make_handle(stream_ptr, "fp64")
        h.set_state(psi0)
        h.time = 0.3 * CFG.duration
        for _ in range(warmup):
            h.propagate_rk(tb, CFG.dt_stable, 1)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        sigma = 0.0
        for k in range(steps):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            sigma += h.propagate_rk(tb, CFG.dt_stable, 1)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / steps
        h.profile(True)
        for k in range(steps):
            flush.fill_(float(k))
            h.propagate_rk(tb, CFG.dt_stable, 1)
        kms, n = h.profile_read().get("rk_stage", (0.0, 0))
        h.profile(False)
        h.close()
        flops = rk_step_flops_per_gp(s, tb in RK_FSAL) * CFG.G * steps
        achieved = flops / (kms * 1e-3) / 1e12 if kms > 0 else None
        out[tb] = {
            "stages": s, "ms_per_step": ms, "gp_steps_per_s": CFG.G / (ms * 1e-3),
            "sigma_per_step": sigma / steps,
            "roofline": {"bound": "alu", "kernel": "rk_general_stage (single, fp64)", "achieved": achieved,
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": None if achieved is None else achieved / FP64_PEAK_TFLOPS,
                         "traffic": None, "flops_per_launch": flops / max(n, 1),
                         "avg_launch_ms": kms / max(n, 1), "launches": n},
        }
    return out


def run_step_observables(stream_ptr, psi0, steps=5, warmup=3, ntheta=180, r_b=10.0):
    """Sec. 4 observables recorded after every step on the at-scale grid
    (FP64 Lanczos-12, dt = 0.02): the dipole series (<z>, <zdot>, <zddot>)
    and the flux through r_b with its density at ntheta angles and their time
    integrals.  Per-step time with and without them (CUDA events, L2 flushed
    before every step), and the dipole kernel against the FP64 peak (it reads
    the state once, 16 B per grid point, and is FP64-instruction bound)."""
    import torch
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ct = np.cos((np.arange(ntheta) + 0.5) * np.pi / ntheta)
    out = {"workload": f"scale grid, FP64 Lanczos-12 dt={CFG.dt:g}; dipole series + flux at r_b={r_b:g} with "
                       f"{ntheta} angles after every step; L2 flushed before every step"}
    for label, hooks in (("without", False), ("with", True)):
        h = make_handle(stream_ptr, "fp64")
        h.set_state(psi0)
        h.time = 0.3 * CFG.duration
        if hooks:
            h.record_dipole(steps + warmup + 8)
            h.flux_setup(r_b, ct)
        for _ in range(warmup):
            h.propagate("lanczos", 12, CFG.dt, 1)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            h.propagate("lanczos", 12, CFG.dt, 1)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        out[f"ms_per_step_{label}"] = sum(a.elapsed_time(b) for a, b in evs) / steps
        if hooks:
            h.profile(True)
            for k in range(3):
                flush.fill_(float(k))
                h.propagate("lanczos", 12, CFG.dt, 1)
            prof = h.profile_read()
            h.profile(False)
            dms, dn = prof.get("dipole", (0.0, 0))
            fms, fn = prof.get("flux", (0.0, 0))
            flops = DIPOLE_FLOPS_PER_GP * CFG.G
            ach = flops / (dms / dn * 1e-3) / 1e12 if dn else None
            out["dipole_kernel"] = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                    "frac": None if ach is None else ach / FP64_PEAK_TFLOPS,
                                    "flops_per_launch": flops, "bytes_per_launch": 16.0 * CFG.G,
                                    "avg_launch_ms": dms / max(dn, 1), "launches": dn}
            out["flux_kernel_avg_ms"] = fms / max(fn, 1)
            f = h.flux()
            out["flux_now"], out["flux_yield"] = f["flux"], f["yield"]
        h.close()
    out["overhead_frac"] = out["ms_per_step_with"] / out["ms_per_step_without"] - 1.0
    return out


def run_small_config(stream_ptr, nsteps=200, reps=3):
    """The small configuration (N=500, dr=0.2, lmax=4, 3-point; 2,500 grid
    points), where a step is a few microseconds of arithmetic and the launch
    and grid-reduction latency decide: us per step of each FP64 propagator,
    nsteps steps per call (one call timed by CUDA events, best of reps, L2
    flushed before each)."""
    import torch
    from paper_1308_1856_gb300 import TDSE
    c = W.SMALL
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    psi0 = W.hydrogen_1s(c.N, c.dr, c.lmax)
    out = {"workload": f"small configuration N={c.N} dr={c.dr} lmax={c.lmax} {c.stencil}-point, FP64, "
                       f"{nsteps} steps per timed call, best of {reps}"}
    for method, order, dt in (("taylor", 8, 0.01), ("rk4", 4, 0.01), ("lanczos", 12, 0.05)):
        t = TDSE(c.N, c.dr, c.lmax, stencil=c.stencil)
        t.set_pulse(c.E0, c.omega, c.ncycles)
        t.set_stream(stream_ptr)
        t.set_state(psi0)
        t.propagate(method, order, dt, 20)
        best = float("inf")
        for k in range(reps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            t.propagate(method, order, dt, nsteps)
            b.record(stream)
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        t.close()
        out[f"{method}-{order}"] = {"us_per_step": 1e3 * best / nsteps, "gp_steps_per_s": c.G * nsteps / (best * 1e-3)}
    return out


def mixed_error(stream_ptr, psi0, nsteps=10):
    """The mixed-precision path's error against the FP64 path on the at-scale
    grid: Lanczos-12 from the benchmark's start state, at a step where the
    propagator converges (dt = 5e-6) and at the stated dt = 0.02, where
    rounding is amplified (compare with the FP64 floor: tests/test_gpu_floor.py).
    The FP64 path itself matches the oracle to 1e-12 per step (tests)."""
    out = {}
    for dt in (5e-6, CFG.dt):
        res = {}
        for prec in ("fp64", "mixed"):
            h = make_handle(stream_ptr, prec)
            h.set_state(psi0)
            h.time = 0.3 * CFG.duration
            h.propagate("lanczos", 12, dt, nsteps)
            res[prec] = (h.get_state(), h.observables())
            h.close()
        (a, oa), (b, ob) = res["fp64"], res["mixed"]
        big = oa["l_pop"] >= 1e-8
        out[f"dt={dt:g}"] = {
            "steps": nsteps,
            "state_rel_l2": float(np.linalg.norm(b - a) / np.linalg.norm(a)),
            "l_pop_max_rel_err": float(np.max(np.abs(ob["l_pop"][big] - oa["l_pop"][big]) / oa["l_pop"][big])),
            "norm_abs_err": abs(ob["norm"] - oa["norm"]),
            "dipole_abs_err": abs(ob["dipole"] - oa["dipole"]),
        }
    return out


def run_ours(args, ws, rank, local):
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)              # a real stream (not the legacy default stream)
    torch.cuda.set_stream(stream)
    psi0 = start_state()
    rows = []
    if args.rows == "served":
        return {"metric": METRIC, "served": run_served(args, stream.cuda_stream)}
    if args.rows == "rk":
        return {"metric": METRIC, "rk_pairs": run_rk_pairs(stream.cuda_stream, psi0, steps=args.steps,
                                                           warmup=args.warmup)}
    if args.rows == "small":
        return {"metric": METRIC, "small_config": run_small_config(stream.cuda_stream)}
    if args.rows == "obs":
        return {"metric": METRIC, "step_observables": run_step_observables(stream.cuda_stream, psi0,
                                                                           steps=args.steps, warmup=args.warmup)}
    if args.rows in ("all", "single"):
        rows += [HandleRow(m, o, dt, p, stream.cuda_stream, psi0) for m, o, dt, p in METHODS]
    if args.rows in ("all", "batched"):
        rows += [BatchRow(p, stream.cuda_stream, count=args.batch_count, schedule=args.schedule.get(p))
                 for p in ("fp64", "mixed")
                 if args.precision in ("all", p) and args.method in ("all", "lanczos")]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one_step(events=None):
        for idx, row in enumerate(rows):
            flush.fill_(float(idx))
            if events is not None:
                events[idx][0].record(stream)
            row.step()
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
    launches0 = sum(r.h.launches for r in rows)
    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
            for _ in rows] for _ in range(args.steps)]
    wall0 = time.perf_counter()
    for k in range(args.steps):
        one_step(evs[k])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    launches = sum(r.h.launches for r in rows) - launches0
    row_ms = {r.name: sum(evs[k][i][0].elapsed_time(evs[k][i][1]) for k in range(args.steps))
              for i, r in enumerate(rows)}
    total_ms = sum(row_ms.values())
    gp_step = sum(r.gp for r in rows)
    total_ms, units_all = combine_over_ranks(total_ms, gp_step * args.steps, ws, dev)
    if ws > 1:
        torch.distributed.barrier()
    for r in rows:
        r.h.sync() if hasattr(r.h, "sync") else r.b.observables(0)   # raises on Inf/NaN
    # ---- per-kernel durations (a separate profiled pass over the same steps) ----
    for r in rows:
        r.h.profile(True)
    prof_steps = 2
    for _ in range(prof_steps):
        one_step()
    prof = {}          # (row kind, precision, kernel) -> [ms, launches, algorithmic points]
    for r in rows:
        for kname, (ms, n) in r.h.profile_read().items():
            if n:
                a = prof.setdefault((r.kind, r.prec, kname), [0.0, 0, 0])
                a[0] += ms
                a[1] += n
                a[2] += prof_steps * r.kernel_points(kname)
        r.h.profile(False)
    kernel_share = {f"{k}/{p}/{kind}": v[0] for (kind, p, k), v in prof.items()}
    tot_k = sum(kernel_share.values())

    def traffic_of(key, points_per_launch):
        per = MEASURED_TRAFFIC_PER_POINT.get((key[0], key[1], key[2]))
        return None if per is None else per * points_per_launch

    def roof_fp64(key):
        ms, n, pts = prof[key]
        flops = KERNEL_FLOPS_PER_GP.get(key[2], H5_FLOPS) * pts
        achieved = flops / (ms * 1e-3) / 1e12
        return {"bound": "alu", "kernel": f"{key[2]} ({key[0]}, fp64)", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": traffic_of(key, pts / n),
                "flops_per_launch": flops / n, "avg_launch_ms": ms / n,
                "peak_source": "FP64: 152 SMs x 2 FMA/clk/SM x 2 flop x 2070 MHz (derived)"}

    def roof_mixed(key):
        ms, n, pts = prof[key]
        nbytes = MIXED_BYTES_PER_GP[key[2]] * pts
        achieved = nbytes / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "kernel": f"{key[2]} ({key[0]}, mixed)", "achieved": achieved,
                "peak": HBM_PEAK_GBS, "unit": "GB/s", "frac": achieved / HBM_PEAK_GBS,
                "traffic": traffic_of(key, pts / n),
                "bytes_per_launch": nbytes / n, "avg_launch_ms": ms / n,
                "peak_source": "HBM copy bandwidth of measured (MEASURED_PEAKS.json)"}

    f64 = [k for k in prof if k[1] == "fp64" and k[2] in KERNEL_FLOPS_PER_GP]
    mix = [k for k in prof if k[1] == "mixed" and k[2] in MIXED_BYTES_PER_GP]
    top_all = max(prof, key=lambda k: prof[k][0])
    roofline = roof_fp64(top_all) if top_all in f64 else (roof_mixed(top_all) if top_all in mix else None)
    roofline_fp64 = roof_fp64(max(f64, key=lambda k: prof[k][0])) if f64 else None
    roofline_mixed = roof_mixed(max(mix, key=lambda k: prof[k][0])) if mix else None
    # ---- end-to-end through the C ABI with host buffers ----
    e2e_steps = 0 if args.no_e2e else 2
    pins = []
    for r in rows:
        if r.kind == "single":
            pin_in = [torch.from_numpy(psi0.view(np.float64).copy()).pin_memory()]
            pin_out = [torch.empty_like(pin_in[0]).pin_memory()]
        else:
            pin_in = [torch.from_numpy(r.b.get_states().view(np.float64)).pin_memory()] if e2e_steps else []
            pin_out = [torch.empty_like(p).pin_memory() for p in pin_in]
        pins.append((pin_in, pin_out))
    # one untimed pass first: the first copies through freshly pinned buffers
    # pay one-off mapping costs that no later step sees
    e2e_times = [np.zeros(3) for _ in rows]
    if e2e_steps:
        for r, (pin_in, pin_out), tm in zip(rows, pins, e2e_times):
            r.e2e_step(pin_in, pin_out, tm)
    e2e_times = [np.zeros(3) for _ in rows]
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    obs = None
    for _ in range(e2e_steps):
        for r, (pin_in, pin_out), tm in zip(rows, pins, e2e_times):
            obs = r.e2e_step(pin_in, pin_out, tm)
    e2e_s = time.perf_counter() - e0
    e2e_s_max, e2e_units = combine_over_ranks(e2e_s, gp_step * e2e_steps, ws, dev)
    value = units_all / (total_ms * 1e-3)
    e2e_value = e2e_units / e2e_s_max if e2e_steps else None
    result = {
        "metric": METRIC, "value": value, "unit": "grid-point*steps/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        # the FP64 rows compute in f64, the mixed rows in f32 (stencil) + f64
        "dtype": ",".join(t for t in ("f64", "f32+f64")
                          if t in {"f64" if r.prec == "fp64" else "f32+f64" for r in rows}),
        "data": "synthetic",
        "config": {"workload": "scale (hydrogen N=8000 dr=0.05 lmax=63 5-point, cos^(1/8) mask): one step each of "
                               "Taylor-12 and RK4 (dt=4e-6) and Lanczos-12 (dt=0.02) in FP64 and mixed; "
                               "batched: 256 instances (seed 1308, N 2000-16000, dr 0.1, lmax 15-127, "
                               "Krylov 8-16, dt 0.02), one Lanczos step each, FP64 and mixed",
                   "grid_points_per_step": gp_step, "rows": [r.name for r in rows],
                   "parallelism": f"replicas x{ws}",
                   "l2": "flushed (256 MB write) before every timed row"},
        "rows_ms_per_step": {k: v / args.steps for k, v in row_ms.items()},
        "rows_gp_steps_per_s": {r.name: r.gp * args.steps / (row_ms[r.name] * 1e-3) for r in rows},
        "roofline": roofline, "roofline_fp64": roofline_fp64, "roofline_mixed": roofline_mixed,
        "kernel_ms_share": {k: round(v / tot_k, 4) for k, v in kernel_share.items()},
        "batched_schedules": {r.name: r.schedule for r in rows if r.kind == "batched"},
        "e2e": {"value": e2e_value, "unit": "grid-point*steps/s",
                "h2d_bytes_per_step": sum(r.e2e_bytes[0] for r in rows),
                "d2h_bytes_per_step": sum(r.e2e_bytes[1] for r in rows), "steps": e2e_steps,
                "warmup": 1 if e2e_steps else 0,
                "ms_per_step_by_row": {r.name: {"h2d": 1e3 * tm[0] / max(e2e_steps, 1),
                                                "step_and_d2h": 1e3 * tm[1] / max(e2e_steps, 1),
                                                "observables": 1e3 * tm[2] / max(e2e_steps, 1)}
                                       for r, tm in zip(rows, e2e_times)},
                "batched_io": f"tdse_batch_propagate_io, {E2E_GROUPS} instance groups (h2d counted in "
                              "step_and_d2h)"},
        "gpu_launches": launches, "wall_s": wall, "clocks": clocks,
    }
    for r in rows:
        if hasattr(r.h, "close"):
            r.h.close()
    if args.rows == "all":
        result["mixed_error"] = mixed_error(stream.cuda_stream, psi0)
        result["rk_pairs"] = run_rk_pairs(stream.cuda_stream, psi0)
        result["step_observables"] = run_step_observables(stream.cuda_stream, psi0)
        result["small_config"] = run_small_config(stream.cuda_stream)
    if args.rows == "all" and not args.no_serve:
        result["served"] = run_served(args, stream.cuda_stream)
    return result


def _oracle_worker(budget_s: float):
    """One serial oracle replica (a process of its own): (grid-point steps, seconds)."""
    v, steps, el = cpu_oracle_sample(budget_s)
    return v * el, el, steps


def cpu_oracle_throughput(budget_s: float, workers: int):
    """The serial oracle on `workers` host cores: independent replicas, one per
    process (spawned: the parent may already hold a CUDA context), each on its
    own copy of the workload; grid-point steps summed over the replicas divided
    by the slowest replica's time."""
    if workers <= 1:
        v, steps, el = cpu_oracle_sample(budget_s)
        return v, steps, el, 1
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        res = pool.map(_oracle_worker, [budget_s] * workers)
    gp = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    return gp / el, sum(r[2] for r in res), el, workers


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--e2e-groups", type=int, default=None,
                    help="instance groups of the batched rows' pipelined copies in the end-to-end leg")
    ap.add_argument("--method", default="all", choices=["all", "taylor", "rk4", "lanczos"],
                    help="restrict to one propagator (profiling runs)")
    ap.add_argument("--precision", default="all", choices=["all", "fp64", "mixed"],
                    help="restrict to one precision (profiling runs)")
    ap.add_argument("--rows", default="all", choices=["all", "single", "batched", "served", "rk", "obs", "small"],
                    help="restrict to one group of rows (single-instance, batched, served, embedded RK, "
                         "step observables, small configuration)")
    ap.add_argument("--batch-count", type=int, default=256,
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
    METHODS[:] = [m for m in ALL_METHODS if (args.method in ("all", m[0]))
                  and (args.precision in ("all", m[3]))]
    ws, rank, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return 0
        cores = host_cores()
        v, steps, el, used = cpu_oracle_throughput(min(60.0, 12.0 * max(1, args.steps) / 4), cores)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "grid-point*steps/s",
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * el / steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "scale (same as ours)", "grid_points": CFG.G},
                "cpu_baseline": {"value": v, "unit": "grid-point*steps/s", "cores": used, "kind": "oracle",
                                 "sample": f"{used} independent serial oracle replicas, {steps} full benchmark "
                                           f"steps (Taylor-12 + RK4 + Lanczos-12 on the at-scale grid) in "
                                           f"{el:.1f} s"},
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
            cores = host_cores()
            va, stepsa, ela, used = cpu_oracle_throughput(12.0, cores)
            res["cpu_baseline_all_cores"] = {
                "value": va, "unit": "grid-point*steps/s", "cores": used, "kind": "oracle",
                "sample": f"{used} independent serial oracle replicas (one process per core), {stepsa} full "
                          f"benchmark steps in {ela:.1f} s"}
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
