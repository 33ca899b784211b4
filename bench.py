#!/usr/bin/env python
"""Throughput benchmark of the GBEES propagation on one GB300 (cell-updates/s).

One timed "step" of the measurement contract is one whole run of the workload
through the hot path: the initial Gaussian, then every propagate segment
(grow, flux update, prune) and measurement update up to t_end. (A time step
of the method is called a time step here.) The default workload is Lorenz '96
in 6-D with h = 0.25, threshold 1e-6 and t_end = 1.0 (7.0e6 initial cells,
7.0e7 at the end, 1.8e10 cell updates per run), FP64 as `value` and FP32
storage beside it; the Lorenz '63 h = 0.25 workload with eight measurements is
reported as an extra key. `value` is device time (CUDA events on the
library's stream) with the inputs resident; `e2e` runs the same through the C
ABI with host buffers and reads the final density back to the host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f64|f32]
  python bench.py --impl reference ...   # the CPU oracle as the reference arm

With N > 1 (torchrun) every rank runs its own replica: the path has no data
exchange between grids, so scaling is weak and no collective is used except
the barrier and the max/sum of the timings.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s"
DEFAULT_WORKLOAD = "lorenz96_6d"
SECONDARY_WORKLOAD = "lorenz63_h0.25"

# DRAM traffic per cell update of the roofline kernel, from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of the launch divided by the
# cell updates it made), keyed by workload/precision; valid only while the
# device sources have the recorded hash (null otherwise).
TRAFFIC_BYTES_PER_CELL = {
    # k_persistent, third launch of `bench.py --workload lorenz63_h0.25 --steps 1 --warmup 1
    # --no-secondary --no-extras --cpu-budget 0 --max-cells 1048576 --no-tune --block-threads 256`
    # (segment t = 0.5..0.75: 2118979 cell updates, counted by the oracle): 6.493 MB read + 0.803 MB
    # written (the grid stays in L2)
    "lorenz63_h0.25/f64/k_persistent": {"bytes_per_cell": (6493184 + 802816) / 2118979, "src": "5c6420cf21eedbce"},
    # k_faces, all 539 launches of the profiled run of `bench.py --precision f64|f32 --steps 1 --warmup 0
    # --no-secondary --no-extras --cpu-budget 0 --e2e-runs 1 --no-tune --block-threads 256`
    # (17,611,960,218 cell updates in FP64, 17,611,960,553 in FP32):
    # FP64 10743.123 GB read + 1139.365 GB written; FP32 6651.750 GB read + 612.772 GB written
    "lorenz96_6d_h0.25/f64/k_faces": {"bytes_per_cell": (10743122864128 + 1139365122560) / 17611960218,
                                      "src": "5c6420cf21eedbce"},
    "lorenz96_6d_h0.25/f32/k_faces": {"bytes_per_cell": (6651749612288 + 612772230144) / 17611960553,
                                      "src": "5c6420cf21eedbce"},
}
# The paper's own throughput on its two cases, in this benchmark's unit (cells
# per second, total cell computations over the runtime): the fastest GPU row of
# its Lorenz '63 table (Table 3, H100) and of its Lorenz '96 table (Table 4,
# H200). vs_baseline divides by them on those workloads only; another machine's
# number, context rather than a target.
PAPER_CELLS_PER_S = {
    "paper_e1": (28.8e6, "Table 3, NVIDIA H100: 226 ms, 28.8 M cells/s"),
    "paper_e2": (40.6e6, "Table 4, NVIDIA H200: 739 s, 40.6 M cells/s"),
}
# Workloads whose paper number is quoted as context only (none at present: both
# cases run at the threshold that reproduces the burden of Table 2).
PAPER_CONTEXT = {}
DEVICE_SOURCES = [os.path.join(ROOT, "paper_2508_13986_gb300", "csrc", f)
                  for f in ("gbees_keys.cuh", "gbees_device.cuh", "gbees_phases.cuh", "gbees_kernels.cuh",
                            "gbees_misc_kernels.cuh", "gbees_persistent.cuh")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--precision", choices=["f64", "f32"], default="f64")
    ap.add_argument("--no-secondary", action="store_true", help="skip the other precision's line")
    ap.add_argument("--cpu-budget", type=float, default=12.0,
                    help="seconds of timed oracle work for cpu_baseline (0: skip)")
    ap.add_argument("--e2e-runs", type=int, default=3,
                    help="whole runs timed end to end through the C ABI (at most --steps)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra keys (the Lorenz '63 workload and the served stream)")
    ap.add_argument("--block-threads", type=int, default=0,
                    help="threads per block of the step kernels (0: tuned by timing 128 and 256)")
    ap.add_argument("--no-tune", dest="tune", action="store_false", help="skip the launch-shape tuning")
    ap.add_argument("--max-cells", type=int, default=0,
                    help="pool capacity of a single-grid workload (0: sized from the workload, see auto_max_cells)")
    ap.add_argument("--launch-mode", choices=["auto", "persistent", "graph", "direct"], default="auto")
    ap.add_argument("--requests", type=int, default=100, help="requests of the serving stream (--workload serving)")
    ap.add_argument("--rate", type=float, default=50.0, help="arrival rate per second of the serving stream")
    ap.add_argument("--t-end", type=float, default=None,
                    help="stop the workload at this time (large-grid runs); the default is its own t_end")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
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
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        out_dir = os.environ.get("BENCH_CLOCKS_DIR")  # keep the raw samples there when set
        if out_dir and os.path.isdir(out_dir):
            with open(os.path.join(out_dir, "clocks.csv"), "a") as f:
                f.write("\n".join(self.lines) + "\n")
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ runs

def auto_max_cells(w, precision, dev) -> int:
    """Pool capacity for a single-grid workload: its pool growth times its
    initial set (24 by default: the pool of the 6-D h = 0.25 horizon peaks at
    18x; 48 for the paper's Lorenz '96 case, which peaks at 38x), a power of
    two, at least 2^24 (coarser grids grow more in relative terms), and halved
    while the workspace would take more than 80 % of the device memory."""
    import torch

    from paper_2508_13986_gb300 import gbees, workloads

    cap = 1 << 24
    while cap < w.pool_growth * workloads.initial_cells_estimate(w):
        cap <<= 1
    total = torch.cuda.get_device_properties(dev).total_memory
    while cap > (1 << 24):
        cfg = gbees.make_config(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, precision,
                                w.limiter, cap)
        if gbees.gbees_workspace_bytes(cfg) <= 0.8 * total:
            break
        cap >>= 1
    return cap


def run_workload(grid, w, with_readout=False):
    """One whole run through the public API. Returns (cell updates, steps, bytes in, bytes out, peak cells)."""
    grid.init_gaussian(w.mean, w.cov)
    h2d = 8 * w.n + 8 * w.n * w.n
    updates = steps = 0
    peak = grid.count() if with_readout else 0
    for t_target, meas in w.segments():
        st = grid.propagate(t_target)
        updates += st.cell_updates
        steps += st.steps
        peak = max(peak, st.n_cells)
        if meas is not None:
            grid.correct_gaussian(meas.y, meas.R, meas.H_idx)
            h2d += 8 * meas.y.size + 8 * meas.R.size + 4 * meas.H_idx.size
    d2h = 0
    if with_readout:
        idx, p = grid.read_cells(sorted_=False)
        mean, cov = grid.moments()
        d2h = idx.nbytes + p.nbytes + mean.nbytes + cov.nbytes
    return updates, steps, h2d, d2h, peak


def bytes_per_update(n: int, precision: str) -> int:
    """Algorithmic HBM bytes of one cell update (one active cell advanced one
    step, grow included): the update pass reads the packed key (8), the value
    (S) and the 2n int32 links (8 n) and writes the new value (S); the grow
    scan reads the value and the links again (S + 8 n). Neighbour values are
    L2 hits. B = 8 + 3 S + 16 n."""
    S = 8 if precision == "f64" else 4
    return 8 + 3 * S + 16 * n


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def device_source_hash() -> str:
    h = hashlib.sha256()
    for path in DEVICE_SOURCES:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def fp64_peak():
    """FP64 arithmetic peak of the GPU from its unit counts and clock: SMs x 2
    FP64 FMA lanes per SM per clock (ncu's sm__sass_thread_inst_executed_op_dfma
    peak_sustained on GB300: 304 per cycle for 152 SMs) x 2 flops x the
    maximum SM clock of MEASURED_PEAKS.json (2070 MHz). Returns (TFLOP/s, how)."""
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    tf = sms * 2 * 2 * mhz * 1e6 / 1e12
    return tf, f"derived: {sms} SMs x 2 FP64 FMA lanes/clock x 2 flops x {mhz:.0f} MHz"


def fp64_flops_per_update(kernel: str, n: int) -> int:
    """Algorithmic FP64 flops of one cell update in a step kernel (an FMA counts
    two): the flux pass evaluates the n lower faces of the cell, 11 flops each
    (the transverse sum, donor cell and corrections: 2 + 2 + 1; the limited
    high-resolution term: 1 + 2 + 1 + 2); the wave pass 7 per dimension (two
    jumps, the entering wave 1 + 2, its share of tg 2); the update pass 3 per
    dimension plus 3 (difference and FMA per face, then the rescale)."""
    return {"k_faces": 11 * n, "k_waves_list": 7 * n, "k_apply": 3 * n + 3}[kernel]


def time_precision(args, w, precision, dev, rank, world, steps=None, warmup=None):
    import torch

    from paper_2508_13986_gb300 import gbees

    prec = gbees.GBEES_FP64 if precision == "f64" else gbees.GBEES_FP32
    mode = {"auto": gbees.GBEES_LAUNCH_AUTO, "persistent": gbees.GBEES_LAUNCH_PERSISTENT,
            "graph": gbees.GBEES_LAUNCH_GRAPH, "direct": gbees.GBEES_LAUNCH_DIRECT}[args.launch_mode]
    max_cells = args.max_cells or auto_max_cells(w, prec, dev)
    # launch shape: threads per block of the step kernels, chosen by timing a
    # short stretch of this workload with each candidate (results do not
    # depend on it)
    tuned = {"block_threads": args.block_threads or 256, "tuned": False}
    if not args.block_threads and args.tune:
        from paper_2508_13986_gb300.autotune import tune_grid

        t_probe = min(w.t_end, 0.05)
        best, times = tune_grid(w, prec, t_probe=t_probe, probe_widths=(1,), launch_modes=(mode,),
                                device=f"cuda:{dev}", max_cells=max_cells, block_threads=(128, 256), repeats=1)
        tuned = {"block_threads": best.block_threads or 256, "tuned": True, "probe_t_end": t_probe,
                 "ns_per_cell_update": {str(k.block_threads): round(v * 1e6, 4) for k, v in times.items()}}
    grid = gbees.grid_for_workload(w, precision=prec, max_cells=max_cells, device=f"cuda:{dev}",
                                   launch_mode=mode, block_threads=tuned["block_threads"])
    stream = grid.stream
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=f"cuda:{dev}")
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    for _ in range(warmup):
        run_workload(grid, w)
    barrier(world)
    torch.cuda.synchronize(dev)
    grid.profile(enable=False, reset=True)
    clocks = ClockSampler(dev)
    clocks.start()
    total_ms, total_updates, total_steps, peak = 0.0, 0, 0, 0
    for _ in range(steps):
        flush.zero_()  # L2 flush between timed runs (outside the events)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        u, s, _, _, pk = run_workload(grid, w)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        total_updates += u
        total_steps += s
        peak = max(peak, pk)
    clk = clocks.stop()
    pt = grid.profile()
    launches = pt["total_launches"]
    persist_split = ({k: v / pt["persist_steps"] for k, v in pt["persist_us"].items()}
                     if pt["persist_steps"] else None)
    barrier(world)
    torch.cuda.synchronize(dev)

    # profiled pass: the same runs with one launch per kernel and CUDA events
    # around every phase on the library's stream (per-kernel durations)
    grid.profile(enable=True, reset=True)
    prof_updates = 0
    for _ in range(1):
        flush.zero_()
        torch.cuda.synchronize(dev)
        u, _, _, _, _ = run_workload(grid, w)
        prof_updates += u
    prof = grid.profile(enable=False)

    # end to end through the C ABI with host buffers: inputs from host memory,
    # final density and moments read back to host memory, wall clock
    e2e_ms, e2e_updates, h2d, d2h = 0.0, 0, 0, 0
    e2e_runs = max(1, min(steps, args.e2e_runs))
    for _ in range(e2e_runs):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        u, _, bi, bo, _ = run_workload(grid, w, with_readout=True)
        torch.cuda.synchronize(dev)
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_updates += u
        h2d, d2h = bi, bo
    grid.close()

    ms_max = reduce_max(total_ms, world)
    upd_sum = reduce_sum(total_updates, world)
    e2e_max = reduce_max(e2e_ms, world)
    e2e_sum = reduce_sum(e2e_updates, world)
    steps_sum = reduce_sum(total_steps, world)

    peak_gbs, peak_src = load_peaks()
    bpc = bytes_per_update(w.n, precision)
    args_steps = steps
    # the dominant kernel of the timed region: the persistent step-loop kernel
    # when the launch mode used it (its launches are event-timed inside the
    # library on its stream), otherwise the slowest per-cell step kernel of the
    # profiled pass (one launch per kernel, events around each)
    if pt["persist_launches"] and pt["persist_updates"] >= 0.5 * total_updates:
        kernel = "k_persistent (whole step loop, one cooperative launch per propagate segment)"
        timing = "CUDA events around every persistent launch on the library stream, timed region"
        launches_k = pt["persist_launches"]
        units = pt["persist_updates"]
        avg_us = pt["persist_ms"] * 1e3 / max(launches_k, 1)
    else:
        per_cell = {k: prof["ms"][k] for k in ("grow", "faces", "apply")}
        top = max(per_cell, key=per_cell.get)
        kernel = {"grow": "k_waves_list", "faces": "k_faces", "apply": "k_apply"}[top]
        timing = "CUDA events around each launch of that kernel in a profiled pass of the same runs"
        launches_k = max(prof["timed"][top], 1)
        units = prof_updates
        avg_us = per_cell[top] * 1e3 / launches_k
    units_per_launch = units / max(launches_k, 1)
    achieved = bpc * units_per_launch / (avg_us * 1e-6) / 1e9 if avg_us > 0 else None
    traffic = None
    rec = TRAFFIC_BYTES_PER_CELL.get(f"{w.name}/{precision}/{kernel.split(' ')[0]}")
    if rec and rec.get("src") == device_source_hash():
        traffic = rec["bytes_per_cell"] * units_per_launch
    roof = {
        "bound": "hbm",
        "kernel": kernel,
        "timing": timing,
        "achieved": achieved,
        "peak": peak_gbs,
        "peak_source": peak_src,
        "unit": "GB/s",
        "frac": (achieved / peak_gbs) if achieved else None,
        "traffic": traffic,
        "algorithmic_bytes_per_cell_update": bpc,
        "cell_updates_per_launch": units_per_launch,
        "avg_launch_us": avg_us,
    }
    kname = kernel.split(" ")[0]
    if precision == "f64" and kname in ("k_faces", "k_waves_list", "k_apply"):
        # FP64 step kernels are bound by the FP64 pipe on this chip (ncu: the
        # flux pass keeps it 64 % busy at 29 % of DRAM bandwidth):
        # the roofline is the FP64 arithmetic peak; the HBM figures stay beside it
        tf, how = fp64_peak()
        fpc = fp64_flops_per_update(kname, w.n)
        ach = fpc * units_per_launch / (avg_us * 1e-6) / 1e12 if avg_us > 0 else None
        roof = {"bound": "alu", "kernel": kernel, "timing": timing, "achieved": ach, "peak": tf,
                "peak_source": how, "unit": "TFLOP/s", "frac": (ach / tf) if ach else None, "traffic": traffic,
                "algorithmic_fp64_flops_per_cell_update": fpc, "cell_updates_per_launch": units_per_launch,
                "avg_launch_us": avg_us,
                "hbm": {"achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                        "frac": (achieved / peak_gbs) if achieved else None,
                        "algorithmic_bytes_per_cell_update": bpc}}
    tot_ms = sum(prof["ms"].values())
    phase_share = {k: (v / tot_ms if tot_ms > 0 else 0.0) for k, v in prof["ms"].items()}
    return {
        "value": upd_sum / (ms_max / 1e3),
        "ms_per_step": ms_max / args_steps,
        "steps": args_steps,
        "warmup": warmup,
        "updates_per_run": total_updates / args_steps,
        "time_steps_per_run": total_steps / args_steps,
        "time_steps_per_s": steps_sum / (ms_max / 1e3),
        "peak_cells": peak,
        "e2e": {"value": e2e_sum / (e2e_max / 1e3), "unit": METRIC, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_run": e2e_max / e2e_runs, "runs": e2e_runs},
        "roofline": roof,
        "profiled_phase_share": phase_share,
        "profiled_phase_ms": {k: v for k, v in prof["ms"].items()},
        "launch_shape": tuned,
        "persistent_us_per_step": persist_split,
        "gpu_launches": launches,
        "clocks": clk,
    }


def time_batch(args, ws, precision, dev, rank, world):
    """Many independent grids per step: the initial Gaussians of all grids and
    one batched propagation of all of them to their own end times."""
    import torch

    from paper_2508_13986_gb300 import gbees, workloads

    prec = gbees.GBEES_FP64 if precision == "f64" else gbees.GBEES_FP32
    grids = [gbees.grid_for_workload(w, precision=prec, max_cells=workloads.capacity_for(w), device=f"cuda:{dev}")
             for w in ws]
    stream = grids[0].stream
    t_ends = [w.t_end for w in ws]
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=f"cuda:{dev}")

    def run(with_readout=False):
        for g, w in zip(grids, ws):
            g.init_gaussian(w.mean, w.cov)
        st = gbees.propagate_batch(grids, t_ends)
        h2d = sum(8 * w.n + 8 * w.n * w.n for w in ws) + 8 * len(ws)
        d2h = 0
        if with_readout:
            for g in grids:
                idx, p = g.read_cells(sorted_=False)
                mean, cov = g.moments()
                d2h += idx.nbytes + p.nbytes + mean.nbytes + cov.nbytes
        return (sum(x.cell_updates for x in st), sum(x.steps for x in st), max(x.n_pool for x in st), h2d, d2h)

    for _ in range(args.warmup):
        run()
    barrier(world)
    torch.cuda.synchronize(dev)
    grids[0].profile(enable=False, reset=True)
    clocks = ClockSampler(dev)
    clocks.start()
    total_ms = total_updates = total_steps = peak = 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        u, nst, pk, _, _ = run()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        total_updates += u
        total_steps += nst
        peak = max(peak, pk)
    clk = clocks.stop()
    pt = grids[0].profile()
    launches = sum(g.profile()["total_launches"] for g in grids)
    e2e_ms = e2e_updates = 0
    h2d = d2h = 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        u, _, _, h2d, d2h = run(with_readout=True)
        torch.cuda.synchronize(dev)
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_updates += u
    for g in grids:
        g.close()
    del grids
    torch.cuda.empty_cache()
    ms_max = reduce_max(total_ms, world)
    upd_sum = reduce_sum(total_updates, world)
    e2e_max = reduce_max(e2e_ms, world)
    e2e_sum = reduce_sum(e2e_updates, world)
    steps_sum = reduce_sum(total_steps, world)
    peak_gbs, peak_src = load_peaks()
    bpc = bytes_per_update(ws[0].n, precision)
    launches_k = max(pt["persist_launches"], 1)
    avg_us = pt["persist_ms"] * 1e3 / launches_k
    units_per_launch = pt["persist_updates"] / launches_k
    achieved = bpc * units_per_launch / (avg_us * 1e-6) / 1e9 if avg_us > 0 else None
    return {
        "value": upd_sum / (ms_max / 1e3),
        "ms_per_step": ms_max / args.steps,
        "updates_per_run": total_updates / args.steps,
        "time_steps_per_run": total_steps / args.steps,
        "time_steps_per_s": steps_sum / (ms_max / 1e3),
        "peak_cells": peak,
        "e2e": {"value": e2e_sum / (e2e_max / 1e3), "unit": METRIC, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_run": e2e_max / args.steps, "runs": args.steps},
        "roofline": {
            "bound": "hbm",
            "kernel": "k_batch (one block per grid, all grids' step loops in one launch)",
            "timing": "CUDA events around every batch launch on the library stream, timed region",
            "achieved": achieved,
            "peak": peak_gbs,
            "peak_source": peak_src,
            "unit": "GB/s",
            "frac": (achieved / peak_gbs) if achieved else None,
            "traffic": None,
            "algorithmic_bytes_per_cell_update": bpc,
            "cell_updates_per_launch": units_per_launch,
            "avg_launch_us": avg_us,
        },
        "profiled_phase_share": None,
        "persistent_us_per_step": None,
        "gpu_launches": launches,
        "clocks": clk,
    }


def serving_forms(args, local, block_threads=0):
    """The request stream served three ways on one GPU: batched FP32, batched
    FP64 (continuous batching, model families overlapping on the device), and
    the plain FP64 form (one request at a time, gbees_propagate)."""
    import torch

    from paper_2508_13986_gb300 import gbees, workloads
    from paper_2508_13986_gb300.serving import Server

    stream = workloads.serving_stream(count=args.requests, rate=args.rate)
    warm = workloads.serving_stream(count=8, rate=1000.0, seed=7)
    out = {}
    for tag, prec, mode in (("batched_f32", gbees.GBEES_FP32, "batched"), ("batched_f64", gbees.GBEES_FP64, "batched"),
                            ("single_f64", gbees.GBEES_FP64, "single")):
        Server(precision=prec, device=f"cuda:{local}", mode=mode, realtime=False,
               block_threads=block_threads).run(warm)
        clocks = ClockSampler(local)
        clocks.start()
        srv = Server(precision=prec, device=f"cuda:{local}", mode=mode, realtime=True, block_threads=block_threads)
        srv.run(stream)
        st = dict(srv.stats)
        st["clocks"] = clocks.stop()
        out[tag] = st
        torch.cuda.empty_cache()
    return out


def main_serving(args):
    import torch

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    out = serving_forms(args, local)
    main = out["batched_f32"]
    print(json.dumps({
        "metric": METRIC, "value": main["cell_updates_per_s"], "unit": METRIC, "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": main["wall_s"] * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serving", "requests": args.requests, "rate_per_s": args.rate,
                   "mix": "70 % Lorenz '63 (batch distributions), 30 % Lorenz '96 6-D; 0-3 corrections each",
                   "pool_bytes": 120 << 30, "round_steps": 64,
                   "timing": "wall clock from the first arrival to the last completion (arrivals in real time)"},
        "serving": out,
    }))


SAMPLE_CELLS = 150_000


def oracle_sample_cells(w):
    """The oracle's initial density of w (untimed); for a grid of more than
    SAMPLE_CELLS cells only the central cube of cells max_j |i_j| <= r around
    the mean's cell (the largest r within that size). Returns (idx, p, label)."""
    import numpy as np

    from oracle.oracle import Oracle

    o = Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, w.limiter)
    o.init_gaussian(w.mean, w.cov)
    idx, p = o.read_cells()
    if len(p) <= SAMPLE_CELLS:
        return idx, p, f"{w.name}: the whole initial density ({len(p)} cells)"
    r = 1
    while (2 * (r + 1) + 1) ** w.n <= SAMPLE_CELLS:
        r += 1
    keep = np.abs(idx).max(axis=1) <= r
    return idx[keep], p[keep], (f"{w.name}: the central cube |i_j| <= {r} of the initial density "
                                f"({int(keep.sum())} of {len(p)} cells)")


def oracle_sample_step(w, idx, p):
    """One oracle time step (grow, dt, flux update, normalisation) from the
    sample cells; returns (cell updates, seconds), the loading untimed."""
    from oracle.oracle import Oracle

    o = Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, w.limiter)
    o.init_cells(idx, p)
    t0 = time.perf_counter()
    st = o.propagate(w.t_end, max_steps=1)
    return st.cell_updates, time.perf_counter() - t0


def cpu_baseline(w, budget_s):
    """The oracle as it stands on the host cores (all of them through its
    OpenMP loops, and one), on a bounded sample of the same workload: time
    steps from the sample cells, repeated for about budget_s seconds of timed
    work."""
    from oracle import oracle as O

    idx, p, label = oracle_sample_cells(w)
    out = {}
    for tag, threads in (("all", 0), ("one", 1)):
        cores = O.set_threads(threads)
        upd, el, reps = 0, 0.0, 0
        while reps == 0 or (tag == "all" and el < budget_s):
            u, dt = oracle_sample_step(w, idx, p)
            upd += u
            el += dt
            reps += 1
        out[tag] = {"value": upd / el, "unit": METRIC, "cores": cores, "kind": "oracle",
                    "sample": f"{label}; one time step from it, {reps}x, {upd} cell updates in {el:.1f} s "
                              f"(loading excluded)"}
    O.set_threads(0)
    return out["all"], out["one"]


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def _reduce(x, world, op_name):
    """All-reduce one number over the replicas (a CUDA tensor under NCCL, a CPU
    tensor under gloo)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def reduce_max(x, world):
    return _reduce(x, world, "MAX")


def reduce_sum(x, world):
    return _reduce(x, world, "SUM")


def main_ours(args):
    import torch

    from paper_2508_13986_gb300 import workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    if args.workload.startswith("lorenz63_batch"):
        count = int(args.workload[len("lorenz63_batch"):] or 256)
        ws = workloads.lorenz63_batch(count=count)
        if args.t_end is not None:
            ws = [x.with_(t_end=min(x.t_end, args.t_end)) for x in ws]
        w = ws[0]
        cfg_extra = {"grids": count, "t_end": "per grid, uniform in [0.25, 1.0]" if args.t_end is None
                     else f"per grid, uniform in [0.25, 1.0], capped at {args.t_end}",
                     "grid_sizes": "ragged, 1.7e3-2.7e5 initial cells"}
        timer = lambda prec, st=None, wu=None: time_batch(args, ws, prec, local, rank, world)  # noqa: E731
    else:
        w = workloads.config(args.workload)
        if args.t_end is not None:
            w = w.with_(t_end=args.t_end, measurements=[m for m in w.measurements if m.t < args.t_end])
        cfg_extra = {"t_end": w.t_end}
        timer = lambda prec, st=None, wu=None: time_precision(args, w, prec, local, rank, world, st, wu)  # noqa: E731
    main = timer(args.precision)
    other = None
    if not args.no_secondary:
        # the other precision beside the headline, on fewer runs (stated in the line)
        other_prec = "f32" if args.precision == "f64" else "f64"
        other = timer(other_prec, min(args.steps, 5), min(args.warmup, 3))
    extras = {}
    if not args.no_extras and args.workload == DEFAULT_WORKLOAD and args.t_end is None:
        # the Lorenz '63 workload with measurements (small grid: the persistent
        # kernel) in both precisions, timed the same way
        w2 = workloads.config(SECONDARY_WORKLOAD)
        for prec in ("f64", "f32"):
            r = time_precision(args, w2, prec, local, rank, world, min(args.steps, 10), min(args.warmup, 3))
            extras.setdefault(SECONDARY_WORKLOAD, {})[prec] = {
                "value": r["value"], "unit": METRIC, "ms_per_run": r["ms_per_step"],
                "time_steps_per_run": r["time_steps_per_run"], "cell_updates_per_run": r["updates_per_run"],
                "e2e": r["e2e"], "roofline": r["roofline"], "persistent_us_per_step": r["persistent_us_per_step"],
                "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}
        if rank == 0:
            bt = (main.get("launch_shape") or {}).get("block_threads", 0)
            sv = serving_forms(args, local, bt)
            extras["serving"] = {"requests": args.requests, "rate_per_s": args.rate, "block_threads": bt,
                                 "mix": "70 % Lorenz '63, 30 % Lorenz '96 6-D; 0-3 corrections each",
                                 "forms": {k: {x: v[x] for x in ("cell_updates_per_s", "requests_per_s", "latency_p50_s",
                                                                 "latency_p99_s", "wall_s", "failed", "clocks")}
                                           for k, v in sv.items()}}
    if rank == 0:
        cpu = cpu1 = None
        if world == 1 and args.cpu_budget > 0:
            cpu, cpu1 = cpu_baseline(w, args.cpu_budget)
        line = {
            "metric": METRIC,
            "value": main["value"],
            "unit": METRIC,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": main["ms_per_step"],
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": (main["value"] / PAPER_CELLS_PER_S[args.workload][0]
                            if args.workload in PAPER_CELLS_PER_S else None),
            "dtype": args.precision,
            "data": "synthetic",
            "config": {"workload": args.workload, **cfg_extra, "parallelism": f"replicas{world}",
                       "step": "one whole run: init + propagate/correct to t_end (ms_per_step is per run)",
                       "l2": "flushed between timed runs (256 MiB write)",
                       "launch_mode": args.launch_mode,
                       "cell_updates_per_run": main["updates_per_run"],
                       "time_steps_per_run": main["time_steps_per_run"],
                       "time_steps_per_s": main["time_steps_per_s"],
                       "peak_cells": main["peak_cells"],
                       "e2e_runs": main["e2e"]["runs"], "profiled_runs": 1,
                       "launch_shape": main.get("launch_shape"),
                       **({"paper_baseline": PAPER_CELLS_PER_S[args.workload][1]}
                          if args.workload in PAPER_CELLS_PER_S else {}),
                       **({"paper_context": PAPER_CONTEXT[args.workload]}
                          if args.workload in PAPER_CONTEXT else {})},
            "e2e": main["e2e"],
            "roofline": main["roofline"],
            "cpu_baseline": cpu,
            "cpu_baseline_1core": cpu1,
            "gpu_launches": main["gpu_launches"],
            "clocks": main["clocks"],
            "profiled_phase_share": main["profiled_phase_share"],
            "persistent_us_per_step": main["persistent_us_per_step"],
        }
        if other is not None:
            line["other_precision"] = {
                "dtype": "f32" if args.precision == "f64" else "f64",
                "value": other["value"], "ms_per_step": other["ms_per_step"],
                "steps": other.get("steps"), "warmup": other.get("warmup"), "e2e": other["e2e"],
                "launch_shape": other.get("launch_shape"),
                "roofline": other["roofline"], "gpu_launches": other["gpu_launches"], "clocks": other["clocks"],
                "profiled_phase_share": other["profiled_phase_share"],
                "persistent_us_per_step": other["persistent_us_per_step"]}
        line.update(extras)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def main_reference(args):
    """The reference arm: the CPU oracle (plain FP64 GBEES) on its host cores,
    one bounded sample of the same workload per step (one oracle time step
    from the sample cells of oracle_sample_cells, the loading untimed)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2508_13986_gb300 import workloads

    w = workloads.config(args.workload)
    cores = O.set_threads(0)
    idx, p, label = oracle_sample_cells(w)
    for _ in range(args.warmup):
        oracle_sample_step(w, idx, p)
    upd, el = 0, 0.0
    for _ in range(args.steps):
        u, dt = oracle_sample_step(w, idx, p)
        upd += u
        el += dt
    val = upd / el
    sample = f"{label}; one time step from it per step ({upd // max(args.steps, 1)} cell updates), loading excluded"
    print(json.dumps({
        "metric": METRIC, "value": val, "unit": METRIC, "impl": "reference", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "parallelism": f"cpu oracle, {cores} threads"},
        "cpu_baseline": {"value": val, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        main_reference(a)
    elif a.workload == "serving":
        main_serving(a)
    else:
        main_ours(a)
