"""Throughput benchmark of the polar-coordinate FDLB step on GB300.

Default workload: the Kelvin-Helmholtz annulus, N_r x N_theta = 4096 x 4096,
33 velocities, FP32 (float-float moments, temperature and weights).  One "step"
is one time step of the combined scheme over the whole grid (one fused kernel
launch).  The distribution (2 x 2.2 GB) is far larger than L2, so no flush is
needed between steps.

Prints ONE JSON line.  Keys beyond the base contract:
  roofline      dominant kernel (the fused step) against measured HBM bandwidth
  cpu_baseline  the FP64 CPU oracle timed on this host on a bounded sample
  fp64          the same workload through the FP64 path (value + roofline)
  adjoint       the FP32 adjoint step on the same workload, its ratio to the
                forward step, and one reverse step with recompute
  noneq         the non-equilibrium moments and departures of Sec. IV (all
                four groups, 48 fields) on the same workload
  e2e           the metric through pclb_run_host with page-locked host buffers
  clocks        SM clocks / throttle reasons sampled during the timed region

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload kh|rm|rm_adj|shock|rot] [--no-cpu-baseline]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell·velocity updates/s + %HBM roofline: FP32 vs FP64 step; adjoint/forward"
UNIT = "cell·velocity updates/s"
Q = 33
FALLBACK_HBM_GBS = 6800.0
# FP64 step: algorithmic flops per cell-velocity update (equilibrium 13,
# relaxation 3, MWB in r 8 and theta 11, combination 2, per-node moments,
# temperature and weights 9 amortised over the 33 velocities)
FP64_FLOPS_PER_UPDATE = 46.0
# 152 SMs x 2 FP64 FMA lanes per SM per clock x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def _workload(name: str, size: str = ""):
    """The named workload; ``size`` = "N_rxN_theta" replaces its grid (the
    same fields sampled on another grid, e.g. for a profile that must stay
    small)."""
    from paper_1302_7104_gb300 import inputs as I
    kw = {}
    if size:
        n_r, n_t = (int(x) for x in size.lower().split("x"))
        kw = {"n_r": n_r, "n_theta": n_t}
    return {
        "kh": lambda: I.kh(**kw),
        "rm": lambda: I.rm(**kw),
        "rm_adj": lambda: I.rm_adj(**kw),
        "shock": lambda: I.shock(**kw),
        "rot": lambda: I.rot(**kw),
    }[name]()


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


_KERNEL_SOURCES = {
    "fp32": ("paper_1302_7104_gb300/csrc/step_kernel_f32.cu", "paper_1302_7104_gb300/csrc/f32_eq2.cuh",
             "paper_1302_7104_gb300/csrc/f32_state.cuh", "paper_1302_7104_gb300/csrc/f32x2.cuh",
             "paper_1302_7104_gb300/csrc/device_common.cuh", "paper_1302_7104_gb300/csrc/pclb_internal.h"),
    "fp64": ("paper_1302_7104_gb300/csrc/step_kernel.cu", "paper_1302_7104_gb300/csrc/ghost_cols.cuh",
             "paper_1302_7104_gb300/csrc/device_common.cuh", "paper_1302_7104_gb300/csrc/pclb_internal.h"),
}


def _kernel_hash(tag: str = "fp32") -> str:
    """Hash of the sources of the FP32 ("fp32") or FP64 ("fp64") step kernel."""
    h = hashlib.sha256()
    for rel in _KERNEL_SOURCES[tag]:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(kernel_tag: str, cells: int):
    """DRAM bytes per launch from the committed ncu summary for this kernel,
    scaled to `cells`, or None if the kernel changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        line = line.strip()
        if line.startswith("#") or ":" not in line:
            continue
        k, v = line.split(":", 1)
        rec[k.strip()] = v.strip()
    if rec.get(f"{kernel_tag}_source_hash") != _kernel_hash(kernel_tag):
        return None
    key = f"{kernel_tag}_bytes_per_cell"
    if key not in rec:
        return None
    return float(rec[key]) * cells


def _alu_peaks(stream) -> dict:
    """Measured packed FP32x2 and FP64 multiply-add rates of this GPU in
    TFLOP/s, from the benchmark's own helper library (libpclb_bench.so, built
    beside the product library; not part of its C ABI)."""
    import ctypes
    from paper_1302_7104_gb300 import build as B
    L = ctypes.CDLL(B.BENCH_LIB)
    L.bench_alu_peaks.restype = ctypes.c_int
    L.bench_alu_peaks.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    out = (ctypes.c_double * 2)()
    rc = L.bench_alu_peaks(ctypes.c_void_p(stream.cuda_stream), out)
    if rc != 0:
        raise RuntimeError(f"bench_alu_peaks failed ({rc})")
    return {"ffma2_tflops": out[0], "dfma_tflops": out[1]}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons in the background."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # wait for the first sample so that the timed region is covered
        t_end = time.perf_counter() + 5.0
        while not self.lines and time.perf_counter() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self, begin: bool):
        if begin:
            self.t_begin = time.perf_counter()
        else:
            self.t_end = time.perf_counter()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.05)   # let the sample taken at the end of the region arrive
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        t0 = getattr(self, "t_begin", None)
        t1 = getattr(self, "t_end", None)
        lines = self.lines
        if t0 is not None and t1 is not None:
            inside = [(t, ln) for t, ln in lines if t0 <= t <= t1 + 0.04]
            lines = inside
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for _, ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, p in zip(names, parts[3:7]):
                if p.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "interval_ms": 20}


def max_over_ranks(secs: float, device=None) -> float:
    """The job's time: the longest of the ranks' timed regions (one value per
    rank, all-reduced with MAX when a process group is up)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return secs
    t = torch.tensor([secs], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(updates_per_step: int, steps: int, world_size: int, secs: float) -> float:
    """Whole-job rate of `world_size` independent replicas, each doing
    `steps` steps of `updates_per_step` updates in at most `secs` (weak
    scaling: the work per GPU is fixed)."""
    return updates_per_step * steps * world_size / secs


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def time_steps(g, steps: int, warmup: int, torch, clocks=None):
    """Warm up, then time exactly `steps` steps with CUDA events on the
    context's stream.  Returns seconds."""
    g.step(warmup)
    g.sync()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    if clocks is not None:
        clocks.mark(True)
    start.record(g.stream)
    for _ in range(steps):
        g.step(1)
    end.record(g.stream)
    end.synchronize()
    if clocks is not None:
        clocks.mark(False)
    return start.elapsed_time(end) / 1e3


def cpu_baseline(wname: str, n_theta: int = 2048, steps: int = 12):
    """The FP64 oracle as it stands, on a radial band of the workload: the full
    radial resolution with `n_theta` azimuthal nodes, `steps` steps."""
    import oracle as O
    from paper_1302_7104_gb300 import inputs as I
    full = {"kh": I.kh, "rm": I.rm, "rm_adj": I.rm_adj, "shock": I.shock, "rot": I.rot}[wname]
    w = full(n_theta=min(n_theta, full().n_theta)) if wname != "rot" else full()
    f = O.set_state(w)
    t0 = time.perf_counter()
    O.run(w, f, steps)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    ups = w.n_r * w.n_theta * Q * steps / dt
    return {"value": ups, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{wname} radial band {w.n_r}x{w.n_theta} (full radial resolution), {steps} steps, "
                      f"FP64, OpenMP over theta rows, {dt:.1f} s"}


def run_ours(args):
    import torch
    from paper_1302_7104_gb300 import pclb as P

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = _workload(args.workload, args.size)
    cells = w.n_r * w.n_theta
    updates = cells * Q
    hbm, peak_src = _peaks()

    g = P.PCLB(w, precision="fp32", device=f"cuda:{local}")
    g.set_state()
    g.sync()
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    secs = time_steps(g, args.steps, args.warmup, torch, clocks)
    clk = clocks.stop()
    flags = g.status_flags()
    secs = max_over_ranks(secs, device=f"cuda:{local}")
    value = job_throughput(updates, args.steps, ws, secs)
    per_launch = secs / args.steps
    alg_bytes = updates * 8.0
    achieved = alg_bytes / per_launch / 1e9
    traffic = _profiled_traffic("fp32", cells)

    # e2e: the same metric through the host-buffer C ABI call, copies included
    pinned = [torch.as_tensor(x, dtype=torch.float32).pin_memory() for x in w.fields()]
    outs = [torch.empty((w.n_theta, w.n_r), dtype=torch.float32).pin_memory() for _ in range(4)]
    for _ in range(max(1, min(args.warmup, 2))):
        g.run_host(*pinned, 1, outs)
    e2e_steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.run_host(*pinned, 1, outs)
    e2e_secs = time.perf_counter() - t0
    e2e_value = updates * e2e_steps * ws / e2e_secs
    io_bytes = 4 * cells * 4
    del pinned, outs

    # adjoint step on the same workload (lam <- J(f)^T lam for a saved state),
    # and one reverse step as the checkpointed backward pass runs it
    # (recompute one forward step into a state buffer, one adjoint step)
    adjoint = None
    if not args.no_adjoint:
        g.set_state()
        state = g.save_state()
        g.moments_vjp(g_rho=torch.ones((w.n_theta, w.n_r), dtype=torch.float32, device=f"cuda:{local}"))
        ka = max(3, min(args.steps, 10))
        for _ in range(2):
            g.adjoint_state(state)
        g.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(g.stream)
        for _ in range(ka):
            g.adjoint_state(state)
        e1.record(g.stream)
        e1.synchronize()
        t_adj = e0.elapsed_time(e1) / 1e3 / ka
        # a reverse step as the checkpointed backward pass runs it: recompute
        # one step straight into the next state buffer, then one adjoint step
        nxt = g.new_state()
        bufs = (state, nxt)
        e0.record(g.stream)
        for i in range(ka):
            g.step_states(bufs[i & 1], bufs[(i + 1) & 1])
            g.adjoint_state(bufs[i & 1])
        e1.record(g.stream)
        e1.synchronize()
        t_rev = e0.elapsed_time(e1) / 1e3 / ka
        del nxt, bufs
        alg = updates * 12.0   # read f and lam, write lam
        adjoint = {"ms_per_step": t_adj * 1e3, "value": updates / t_adj, "unit": UNIT,
                   "ratio_to_forward": t_adj / per_launch,
                   "reverse_step_ms": t_rev * 1e3, "reverse_ratio_to_forward": t_rev / per_launch,
                   "roofline": {"bound": "hbm", "achieved": alg / t_adj / 1e9, "peak": hbm, "unit": "GB/s",
                                "frac": alg / t_adj / 1e9 / hbm, "alg_bytes_per_launch": alg,
                                "kernel": "pclb::adjoint_pair_f32x2 (+ adjoint_wall_kernel on a side stream)"}}
        del state

    # non-equilibrium manifestations (Sec. IV), all four groups, on the same state
    noneq = None
    if not args.no_noneq:
        g.set_state()
        g.step(1)
        out = g.noneq(15)
        g.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        kn = max(3, min(args.steps, 10))
        e0.record(g.stream)
        for _ in range(kn):
            g.noneq(15, out=out)
        e1.record(g.stream)
        e1.synchronize()
        t_n = e0.elapsed_time(e1) / 1e3 / kn
        nbytes = cells * (Q + 48) * 4.0     # read f, write 4 groups x 12 fields
        noneq = {"ms": t_n * 1e3, "groups": 4, "fields": 48,
                 "roofline": {"bound": "hbm", "achieved": nbytes / t_n / 1e9, "peak": hbm, "unit": "GB/s",
                              "frac": nbytes / t_n / 1e9 / hbm, "alg_bytes_per_launch": nbytes,
                              "kernel": "pclb::noneq_kernel<float>"}}
        del out
    g.close()

    # FP64 step on the same workload
    fp64 = None
    if not args.no_fp64:
        g64 = P.PCLB(w, precision="fp64", device=f"cuda:{local}")
        g64.set_state()
        g64.sync()
        k64 = max(3, min(args.steps, 10))
        s64 = time_steps(g64, k64, 2, torch)
        g64.close()
        t64 = s64 / k64
        tflops = updates * FP64_FLOPS_PER_UPDATE / t64 / 1e12
        # the FP64 multiply-add rate measured on this GPU, as context for the derived peak
        try:
            measured = _alu_peaks(torch.cuda.current_stream(local))
        except Exception:   # context only; the derived peak stands
            measured = None
        fp64 = {"value": updates * k64 / s64, "unit": UNIT, "steps": k64, "ms_per_step": t64 * 1e3,
                "alu_measured_tflops": measured,
                "roofline": {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": tflops / FP64_PEAK_TFLOPS, "flops_per_update": FP64_FLOPS_PER_UPDATE,
                             "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                             "hbm_frac": updates * 16.0 / t64 / 1e9 / hbm,
                             "traffic": _profiled_traffic("fp64", cells),
                             "kernel": "pclb::step_kernel<double>"}}

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_launch * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.workload}_{w.n_r}x{w.n_theta}_q33_fp32", "n_r": w.n_r,
                   "n_theta": w.n_theta, "velocities": Q, "cells": cells, "tau": w.tau, "dt": w.dt,
                   "parallelism": f"replicas{ws}" if ws > 1 else "single",
                   "l2": "state 2 x %.2f GB > 129 MB L2, no flush needed" % (updates * 4 / 1e9),
                   "T_recovery": "float-float"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_source": peak_src,
                     "kernel": "pclb::step_kernel_f32", "alg_bytes_per_launch": alg_bytes},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": io_bytes,
                "d2h_bytes_per_step": io_bytes, "steps": e2e_steps},
        "gpu_launches": args.steps,
        "status_flags": flags,
    }
    if fp64 is not None:
        line["fp64"] = fp64
    if adjoint is not None:
        line["adjoint"] = adjoint
    if noneq is not None:
        line["noneq"] = noneq
    if clk is not None:
        line["clocks"] = clk
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle as O
    from paper_1302_7104_gb300 import inputs as I
    full = _workload(args.workload)
    w = {"kh": I.kh, "rm": I.rm, "rm_adj": I.rm_adj, "shock": I.shock, "rot": I.rot}[args.workload](
        n_theta=min(128, full.n_theta)) if args.workload != "rot" else full
    f = O.set_state(w)
    prob = O.Problem(w)
    f = O.run(w, f, args.warmup, prob=prob)
    t0 = time.perf_counter()
    O.run(w, f, args.steps, prob=prob)
    secs = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    value = w.n_r * w.n_theta * Q * args.steps / secs
    sample = (f"{args.workload} radial band {w.n_r}x{w.n_theta} (full radial resolution), FP64 oracle, "
              f"OpenMP over theta rows")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}_{full.n_r}x{full.n_theta}_q33_fp32",
                       "sample_n_theta": w.n_theta},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kh", choices=["kh", "rm", "rm_adj", "shock", "rot"])
    ap.add_argument("--size", default="", help="N_rxN_theta: the workload's fields on another grid")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-noneq", action="store_true")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
