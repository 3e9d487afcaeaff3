#!/usr/bin/env python3
"""Benchmark: cell-updates/s of the fused finite-volume step on one GB300.

Headline workload (N=1): 2D shallow-water radial dam break, Clawpack-classic
(Roe + Harten-Hyman, MC limiter, transverse corrections), 1024 x 1024 cells,
FP64.  One step = one fused step attempt (ghost remap, Riemann solves,
limiting, corrections, transverse propagation, update, CFL reduction and
controller).  The same JSON line also carries the FP32 form of that workload,
the FP32 batched 1D elasticity ensemble against FP64 one-at-a-time, and the
serving stream's p50/p99 latency.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs its own replica (the step does not
shard: replicas only); value = all ranks' cell updates / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s & % HBM peak, FP64 plain vs FP32 batched; p50/p99 solve latency"
UNIT = "cell-updates/s"
L2_FLUSH_BYTES = 512 << 20

# Algorithmic work per cell update, counted on the oracle's own arithmetic by
# oracle/flop_count.cpp (FP add/sub/mul/div/sqrt/exp; min, max, abs and
# compares not counted; a CPU test pins these constants to its output):
# - headline 2D SW classic (Roe + HH, MC, transverse 2): the oracle's step on
#   smooth data with every wave non-zero (904.95 per cell at 1024^2) less the
#   four Roe averages (20 each) its transverse solver re-derives per cell,
#   which the kernel takes from the normal solve;
# - SharpClaw 2D Euler, WENO5 characteristic-wise: one L(Q) evaluation per
#   stage (three per SSP-RK3 step);
# - 1D elasticity f-wave classic step;
# - 1D acoustics classic step (MC): the oracle's step (95 per cell) less the
#   medium constants it re-derives at every interface (c = sqrt(K/rho): one
#   division and one square root; Z = rho c and 2 Z twice: three products),
#   which the kernel takes as constants.
# Bytes: one read and one write of the conserved fields (plus aux reads).
SW2D_FLOPS_PER_CELL = 825.0
EULER2D_WENO5_FLOPS_PER_CELL_STAGE = 3032.4
ELAST1D_FLOPS_PER_CELL = 96.0
ACOU1D_FLOPS_PER_CELL = 90.0
SW2D_BYTES_PER_CELL = {"fp64": 48.0, "fp32": 24.0}
ELAST1D_BYTES_PER_CELL = {"fp64": 48.0, "fp32": 24.0}  # q read+write, aux read
ACOU1D_BYTES_PER_CELL = {"fp64": 32.0, "fp32": 16.0}   # q read+write
# 3D acoustics (4 fields, w bytes per value), per cell and step: the x sweep
# reads the state and stores five face records (6 m w); the y and z sweeps
# read the state, store two records and reduce into three, a read and a write
# each at the DRAM (9 m w each); the update reads the state and nine records
# and writes the state (11 m w): 35 m w in all
ACOU3D_BYTES_PER_CELL = {"fp32": 35 * 4 * 4, "fp64": 35 * 4 * 8}
# ALU peaks from unit counts and clocks (for comparison with the measured FMA
# rate the roofline uses): 152 SMs x 2.07 GHz x 2 FLOP per FMA x FMA lanes per
# SM per clock (FP64: 2; FP32: 128)
FP64_PEAK_DERIVED_TFLOPS = 152 * 2.07e9 * 2 * 2 / 1e12
FP32_PEAK_DERIVED_TFLOPS = 152 * 2.07e9 * 2 * 128 / 1e12


TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "traffic_classic2d_sw_fp64_1024.json")
KERNEL_SOURCES = ["claw_common.cuh", "riemann.cuh", "classic.cuh", "launch.cuh", "kernels.h",
                  "k_sw.cu"]


def kernel_sha():
    """Hash of the sources that define the headline kernel."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1111_6583_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(tile):
    """DRAM bytes per launch of the headline kernel from the last ncu capture,
    or None when the kernel sources changed since it was taken or the capture
    ran another tile shape."""
    if not os.path.exists(TRAFFIC_RECORD):
        return None
    rec = json.load(open(TRAFFIC_RECORD))
    if rec.get("sources_sha256") != kernel_sha() or rec.get("tile") != list(tile):
        return None
    return rec["dram_bytes_per_launch"]


def record_traffic(csv_path, tile):
    """Write the traffic record from an ncu --csv launch list of the bench
    command (metrics dram__bytes_read.sum, dram__bytes_write.sum; the last
    four classic2d launches of `--case sw2d1024` are its four steps; ncu
    flushes the caches before each launch it captures, so these are the
    bytes of a launch that starts with a cold L2, as the timed steps do)."""
    import csv
    rows = list(csv.reader(open(csv_path)))
    hi = [i for i, r in enumerate(rows) if "Kernel Name" in r][0]
    hdr = rows[hi]
    mi, vi, ii = hdr.index("Metric Name"), hdr.index("Metric Value"), hdr.index("ID")
    by = {}
    for r in rows[hi + 1:]:
        if len(r) > vi:
            by.setdefault(r[ii], {})[r[mi]] = float(r[vi].replace(",", ""))
    timed = list(by.values())[-4:]
    b = sum(v["dram__bytes_read.sum"] + v["dram__bytes_write.sum"] for v in timed) / len(timed)
    t = "%d,%d" % tuple(tile)
    rec = {"kernel": "classic2d_kernel<RpSW<double,2>>", "workload": "dam break 1024x1024 FP64",
           "tile": list(tile), "dram_bytes_per_launch": b, "sources_sha256": kernel_sha(),
           "command": "python bench.py --case sw2d1024 --tile %s > plain.log 2>&1 && "
                      "ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,"
                      "dram__bytes_write.sum --clock-control none -k regex:classic2d --csv "
                      "--log-file traffic_sw2d.csv python bench.py --case sw2d1024 "
                      "--tile %s" % (t, t)}
    json.dump(rec, open(TRAFFIC_RECORD, "w"), indent=1)
    print(json.dumps(rec))


def copy_rate_gbs(nbytes=1 << 30, reps=5):
    """A device-to-device copy of nbytes (read + write bytes over the best of
    `reps` CUDA-event timings): the copy rate of this run, beside the
    measured one in MEASURED_PEAKS.json."""
    import torch
    a = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for _ in range(reps + 1):
        e0.record()
        b.copy_(a)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None or ms < best else best
    del a, b
    return 2.0 * nbytes / (best * 1e-3) / 1e9


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def peaks_file():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(p)) if os.path.exists(p) else {}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index=0):
        self.samples = []
        self.index = index
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if len(s) > 8 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) > 8 and s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            if len(s) > 8:
                for k, nm in enumerate(names):
                    if s[5 + k].lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def dist_setup(gpus, backend=None):
    """One process per GPU (torchrun environment).  Replicas only: the ranks
    share no data; the process group carries the barrier and the max of the
    timings.  backend defaults to NCCL with a GPU, gloo without."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank, total_ms_max, world):
    """Whole-job throughput of N replicas: every rank processes the same
    units; the job takes the slowest rank's time."""
    return units_per_rank * world / (total_ms_max * 1e-3)


def timed_steps(solver, stream, steps, flush):
    """Per-step CUDA events on the launching stream; the L2 is flushed between
    steps outside the timed intervals.  Returns the per-step durations (ms)."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    with torch.cuda.stream(stream):
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            solver.advance(1)
            b.record(stream)
    stream.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def bench_sw2d(prec, steps, warmup, n=1024, tile=None):
    """Timed step attempts of the dam break; also returns how many of them the
    controller accepted (the headline counts accepted steps only).  The tile
    is the autotuner's pick, or `tile` (bw, h) when given."""
    import torch
    from paper_1111_6583_gb300 import claw
    from paper_1111_6583_gb300 import workloads as wl
    spec = wl.sw_dambreak_2d(n=n)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = claw.Solver(spec, prec, stream=stream.cuda_stream)
        bw, h = s.tune(*tile) if tile else s.tune()
        s.set_t_end(1.5)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        s.advance(warmup)
    stream.synchronize()
    before = s.info()["steps"]
    ms = timed_steps(s, stream, steps, flush)
    info = s.info()
    info["accepted_in_timed"] = info["steps"] - before
    s.close()
    return spec, ms, info, (bw, h)


def e2e_sw2d(prec, steps, warmup, n=1024):
    """Same metric through the C ABI from host memory: each step copies the
    state in from pinned host memory, steps, and copies it back."""
    import torch
    from paper_1111_6583_gb300 import claw
    from paper_1111_6583_gb300 import workloads as wl
    spec = wl.sw_dambreak_2d(n=n)
    dt = torch.float64 if prec == "fp64" else torch.float32
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = claw.Solver(spec, prec, stream=stream.cuda_stream)
        s.tune()
        s.set_t_end(1.5)
    hin = torch.as_tensor(spec["q0"], dtype=dt).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    for _ in range(warmup):
        s.step_host(hin, hout, 1)
        hin, hout = hout, hin
    stream.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        st = s.step_host(hin, hout, 1)
        hin, hout = hout, hin
    t1 = time.perf_counter()
    s.close()
    nbytes = hin.numel() * hin.element_size()
    cells = n * n
    return {"value": cells * steps / (t1 - t0), "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes}


def bench_elasticity(members, steps, fp64_sample):
    """FP32 batched ensemble (one fused launch per step over all members) vs
    FP64 one-at-a-time on a sample of the same members."""
    import torch
    from paper_1111_6583_gb300 import claw
    from paper_1111_6583_gb300 import workloads as wl
    ens = wl.elasticity_ensemble(members)
    specs = [wl.elasticity_member(e["n"], e["amp"], e["width"], t_end=e["t_end"]) for e in ens]
    cells = sum(e["n"] for e in ens)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = claw.Batch(specs, "fp32", stream=stream.cuda_stream)
        shape = b.tune()  # how warps take work, timed on the bound members
        b.advance(3)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        b.advance(steps)
        e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    out = {"members": members, "cells": cells, "steps": steps,
           "fp32_batched": cells * steps / (ms * 1e-3), "fp32_ms_per_step": ms / steps,
           "work_mode": {1: "whole tiles", 2: "single units"}.get(shape[1], "automatic")}
    b.close()
    # FP64, one grid at a time (each member its own solver and launches)
    sample = specs[:fp64_sample]
    scells = sum(sp["q0"].shape[1] for sp in sample)
    solvers = []
    with torch.cuda.stream(stream):
        for sp in sample:
            solvers.append(claw.Solver(sp, "fp64", stream=stream.cuda_stream))
        for sv in solvers:
            sv.advance(2)
    stream.synchronize()
    k = max(1, steps // 10)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(k):
            for sv in solvers:
                sv.advance(1)
        e1.record(stream)
    stream.synchronize()
    ms64 = e0.elapsed_time(e1)
    for sv in solvers:
        sv.close()
    out["fp64_one_at_a_time"] = scells * k / (ms64 * 1e-3)
    out["fp64_sample_members"] = len(sample)
    return out


def bench_serving(nreq, prec, rate=200.0, budget=120 << 30, policy="srw", min_cells=1 << 23,
                  tune_at=32):
    """Poisson stream of 2D shallow-water solves through the continuous-
    batching server; latency = completion - arrival (server clock).  policy:
    the server's schedule ('srw': shortest remaining work first, min_cells
    cells per attempt; 'all': every running request in every attempt).  The
    server tunes its tile shape once, on the live mix, when tune_at requests
    are running (0: never)."""
    from paper_1111_6583_gb300 import claw
    from paper_1111_6583_gb300 import workloads as wl
    stream_reqs = wl.serving_stream(nreq, rate)
    sv = claw.Server(wl.sw_humps_2d(64, [], 1.0), prec, budget_bytes=budget, max_slots=512)
    sv.schedule(policy, min_cells)
    specs = [wl.sw_humps_2d(r["n"], r["humps"], r["t_end"]) for r in stream_reqs]
    t0 = claw.clock()
    pending = {}
    nxt = 0
    lat = []
    cell_updates = 0
    tile = None
    while nxt < nreq or pending:
        now = claw.clock() - t0
        while nxt < nreq and stream_reqs[nxt]["arrival"] <= now:
            tk = sv.submit(specs[nxt])
            pending[tk] = nxt
            nxt += 1
        if pending:
            running, _ = sv.pump(8)
            if tile is None and tune_at and running >= tune_at:
                tile = sv.tune()
            for tk in sv.take_done():
                r = sv.poll(tk, want_state=False)
                i = pending.pop(tk)
                lat.append(r["t_done"] - (t0 + stream_reqs[i]["arrival"]))
                n = specs[i]["n"][0]
                cell_updates += n * n * r["steps"]
        elif nxt < nreq:
            time.sleep(max(0.0, min(0.002, stream_reqs[nxt]["arrival"] - now)))
    wall = claw.clock() - t0
    sv.close()
    lat = np.array(lat)
    return {"requests": nreq, "rate_per_s": rate, "prec": prec, "schedule": policy,
            "min_cells": min_cells if policy == "srw" else None,
            "tile": list(tile) if tile else "fixed 64 x 21 (not tuned)",
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "throughput_cell_updates_per_s": cell_updates / wall, "wall_s": wall}


def bench_shockbubble(prec, steps, warmup, nx=2048, ny=1024, weno_order=5,
                      integrator="ssp_rk3", tile=None):
    """2D Euler shock-bubble, SharpClaw WENO-char: one step = three fused
    stage launches (SSP-RK3, CFL 0.8) or ten (SSP(10,4), CFL 2.0).  The
    stage tile is the autotuner's pick (WENO5), or `tile` when given."""
    import torch
    from paper_1111_6583_gb300 import claw
    from paper_1111_6583_gb300 import workloads as wl
    spec = wl.shock_bubble_2d(nx=nx, ny=ny)
    spec["weno_order"] = weno_order
    spec["time_integrator"] = integrator
    if integrator == "ssp104":
        spec.update(cfl_desired=2.0, cfl_max=2.5)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = claw.Solver(spec, prec, stream=stream.cuda_stream)
        shape = s.tune(*tile) if tile else s.tune()
        s.set_t_end(0.2)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        s.advance(warmup)
    stream.synchronize()
    ms = timed_steps(s, stream, steps, flush)
    s.close()
    avg = sum(ms) / len(ms)
    return {"value": nx * ny * len(ms) / (sum(ms) * 1e-3), "unit": UNIT, "ms_per_step": avg,
            "tile": list(shape),
            "workload": "2D Euler shock-bubble %dx%d, SharpClaw WENO%d-char + %s, %s"
                        % (nx, ny, weno_order,
                           "SSP-RK3" if integrator == "ssp_rk3" else "SSP(10,4)",
                           prec.upper())}


def bench_axisym(prec, steps, warmup, nx=1280, ny=320, dim_split=0, source_split="godunov"):
    """The axisymmetric shock-bubble of Sec. 7.2 at the paper's 1280 x 320:
    Euler + tracer, classic unsplit with full transverse corrections (or
    dimensionally split), geometric source by Godunov (or Strang) splitting;
    one step = the step kernel (two when split) + the source kernel (two for
    Strang) + its marker."""
    import torch
    from paper_1111_6583_gb300 import claw
    from paper_1111_6583_gb300 import workloads as wl
    spec = wl.shock_bubble_axisym(nx=nx, ny=ny, dim_split=dim_split, source_split=source_split)
    if dim_split:
        spec["transverse"] = 0
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = claw.Solver(spec, prec, stream=stream.cuda_stream)
        tile = s.tune()
        s.set_t_end(spec["t_end"])
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        s.advance(warmup)
    stream.synchronize()
    ms = timed_steps(s, stream, steps, flush)
    s.close()
    avg = sum(ms) / len(ms)
    return {"value": nx * ny * len(ms) / (sum(ms) * 1e-3), "unit": UNIT, "ms_per_step": avg,
            "tile": list(tile) if tile else None,
            "workload": "axisymmetric shock-bubble %dx%d, Euler + tracer, classic %s, "
                        "geometric source (%s), %s"
                        % (nx, ny, "dimensionally split" if dim_split else "unsplit full "
                           "transverse", source_split.capitalize(), prec.upper())}


def bench_acoustics_vc(prec, steps, warmup, n=1024):
    """2D acoustics in a heterogeneous medium on a stretched grid (capacity):
    classic with full transverse corrections on the per-face path (two face
    sweeps + the update per step)."""
    import torch
    from paper_1111_6583_gb300 import claw
    from paper_1111_6583_gb300 import workloads as wl
    spec = wl.acoustics_vc_2d(n=n)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = claw.Solver(spec, prec, stream=stream.cuda_stream)
        s.set_t_end(spec["t_end"])
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        s.advance(warmup)
    stream.synchronize()
    ms = timed_steps(s, stream, steps, flush)
    s.close()
    avg = sum(ms) / len(ms)
    return {"value": n * n * len(ms) / (sum(ms) * 1e-3), "unit": UNIT, "ms_per_step": avg,
            "workload": "2D acoustics, varying medium + capacity %dx%d, classic full "
                        "transverse (per-face path), %s" % (n, n, prec.upper())}


def bench_acoustics_table1(prec, steps, warmup, nd, n):
    """The paper's Table 1 acoustics system, constant medium: 2D on n^2 (row
    kernel, autotuned tiles) or 3D on n^3 (a memset, three face sweeps with
    transverse and double-transverse terms, the update)."""
    import torch
    from paper_1111_6583_gb300 import claw
    from paper_1111_6583_gb300 import workloads as wl
    spec = wl.acoustics_2d(n=n) if nd == 2 else wl.acoustics_3d(n=n)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = claw.Solver(spec, prec, stream=stream.cuda_stream)
        tile = s.tune() if nd == 2 else None
        s.set_t_end(spec["t_end"])
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        s.advance(warmup)
    stream.synchronize()
    ms = timed_steps(s, stream, steps, flush)
    s.close()
    avg = sum(ms) / len(ms)
    cells = n ** nd
    out = {"value": cells * len(ms) / (sum(ms) * 1e-3), "unit": UNIT, "ms_per_step": avg,
           "workload": "%dD acoustics, constant medium %s, classic MC full transverse%s, %s"
                       % (nd, "x".join([str(n)] * nd),
                          " + double transverse" if nd == 3 else "", prec.upper())}
    if tile:
        out["tile"] = list(tile)
    return out


def bench_psystem(prec, steps, warmup, periods=32, cells_per_period=64):
    """2D p-system in the checkerboard medium (Sec. 7.3), SharpClaw WENO5
    component-wise + SSP(10,4): one step = ten fused stage launches."""
    import torch
    from paper_1111_6583_gb300 import claw
    from paper_1111_6583_gb300 import workloads as wl
    spec = wl.psystem_checkerboard_2d(periods=periods, cells_per_period=cells_per_period)
    n = spec["n"][0]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = claw.Solver(spec, prec, stream=stream.cuda_stream)
        s.set_t_end(spec["t_end"])
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        s.advance(warmup)
    stream.synchronize()
    ms = timed_steps(s, stream, steps, flush)
    s.close()
    avg = sum(ms) / len(ms)
    return {"value": n * n * len(ms) / (sum(ms) * 1e-3), "unit": UNIT, "ms_per_step": avg,
            "workload": "2D p-system checkerboard %dx%d (%d periods, dx = 1/%d), SharpClaw "
                        "WENO5 + SSP(10,4), %s" % (n, n, periods, cells_per_period,
                                                   prec.upper())}


def _sig(x, d=4):
    """x rounded to d significant digits (None and non-numbers pass through)."""
    if isinstance(x, bool) or not isinstance(x, (int, float)) or x == 0 or x != x:
        return x
    import math
    return round(x, d - 1 - int(math.floor(math.log10(abs(x)))))


def _compact(o):
    if isinstance(o, dict):
        return {k: _compact(v) for k, v in o.items()}
    if isinstance(o, (list, tuple)):
        return [_compact(v) for v in o]
    return _sig(o)


def bench_acoustics_1d(prec="fp64", n=2000, t_end=2.0):
    """The 1D acoustics pulse (2000 cells, periodic, MC, CFL 0.9) run to t = 2
    with the controller from replayed CUDA graphs of step attempts: time per
    accepted step and steps per second (the state is 32 KB: latency-bound)."""
    import torch
    from paper_1111_6583_gb300 import claw
    from paper_1111_6583_gb300 import workloads as wl
    spec = wl.acoustics_1d(n=n, t_end=t_end)
    out = {}
    for rep in range(2):  # the first run builds and uploads the graphs
        s = claw.Solver(spec, prec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        info = s.evolve(t_end, use_graph=True)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        s.close()
        out = {"steps": info["steps"], "t": info["t"], "us_per_step": ms * 1e3 / info["steps"],
               "steps_per_s": info["steps"] / (ms * 1e-3),
               "value": n * info["steps"] / (ms * 1e-3), "unit": UNIT}
    return out


def bench_acoustics_1d_hbm(prec, steps, warmup, log2n=26):
    """Roofline form of the 1D acoustics step: 2^26 cells (same physics, the
    pulse on a longer periodic line), one fused step kernel + controller per
    step; algorithmic bytes = one read and one write of the two fields."""
    import torch
    from paper_1111_6583_gb300 import claw
    from paper_1111_6583_gb300 import workloads as wl
    n = 1 << log2n
    spec = wl.acoustics_1d(n=n, t_end=1e9)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = claw.Solver(spec, prec, stream=stream.cuda_stream)
        s.set_t_end(1e9)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        s.advance(warmup)
    stream.synchronize()
    ms = timed_steps(s, stream, steps, flush)
    s.close()
    avg = sum(ms) / len(ms)
    gbs = ACOU1D_BYTES_PER_CELL[prec] * n / (avg * 1e-3) / 1e9
    return {"cells": n, "ms_per_step": avg, "value": n / (avg * 1e-3), "unit": UNIT,
            "hbm_gbs": gbs}


def err_vs_oracle(q, ref):
    """max-norm relative (per field, maximised) and L1 relative errors of q
    against the FP64 oracle's result ref."""
    q = np.asarray(q, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    big = np.abs(ref).max()
    mx = 0.0
    for k in range(ref.shape[0]):
        den = np.abs(ref[k]).max()
        den = big if den < 1e-12 * big else den
        mx = max(mx, float(np.abs(q[k] - ref[k]).max() / den))
    return {"max_rel": mx, "l1_rel": float(np.abs(q - ref).sum() / np.abs(ref).sum())}


def errors_vs_oracle():
    """Outside every timed region: the FP32 (and FP64) GPU results of the
    workloads at the oracle's sizes, run to their final times, against the
    FP64 oracle: dam break 256^2 to t = 1.5, shock-bubble 256 x 128 to t =
    0.2, sampled ensemble members to t = 50 (batched FP32 launch), and one
    served FP32 request."""
    import torch
    import oracle
    from paper_1111_6583_gb300 import claw
    from paper_1111_6583_gb300 import workloads as wl
    oracle.build()
    out = {}

    def gpu_run(spec, prec, t_end):
        s = claw.Solver(spec, prec)
        info = s.evolve(t_end)
        torch.cuda.synchronize()
        q = s.q.double().cpu().numpy()
        s.close()
        return q, info

    for name, spec, t_end in (("dambreak_256", wl.sw_dambreak_2d(n=256), 1.5),
                              ("shock_bubble_256x128", wl.shock_bubble_2d(nx=256, ny=128), 0.2)):
        qo, io = oracle.evolve(oracle.make_problem(spec), spec["q0"], spec.get("aux"),
                               t_end=t_end)
        row = {"t": t_end, "oracle_steps": io["steps"]}
        for prec in ("fp64", "fp32"):
            q, info = gpu_run(spec, prec, t_end)
            row[prec] = err_vs_oracle(q, qo)
            row[prec]["steps"] = info["steps"]
        out[name] = row
    # ensemble members: three of the smaller grids (spread over 2^12..2^14)
    ens = wl.elasticity_ensemble(4096)
    small = sorted((e["n"], k) for k, e in enumerate(ens) if e["n"] <= (1 << 14))
    pick = [small[0][1], small[len(small) // 2][1], small[-1][1]]
    specs = [wl.elasticity_member(ens[k]["n"], ens[k]["amp"], ens[k]["width"], t_end=50.0)
             for k in pick]
    b = claw.Batch(specs, "fp32")
    binfo = b.evolve()
    qs = [t.double().cpu().numpy() for t in b.sync()]
    b.close()
    rows = []
    for k, sp, q, bi in zip(pick, specs, qs, binfo):
        qo, io = oracle.evolve(oracle.make_problem(sp), sp["q0"], sp["aux"], t_end=50.0)
        e = err_vs_oracle(q, qo)
        e.update(member=k, cells=sp["n"][0], steps=bi["steps"], oracle_steps=io["steps"])
        rows.append(e)
    out["ensemble_members_t50"] = rows
    # one served FP32 request against the oracle: the smallest of the first 20
    # of the benchmark's stream
    req = min(wl.serving_stream(400, 200.0)[:20], key=lambda r: r["n"])
    sp = wl.sw_humps_2d(req["n"], req["humps"], req["t_end"])
    sv = claw.Server(sp, "fp32", budget_bytes=1 << 30, max_slots=4)
    tk = sv.submit(sp)
    res = None
    while res is None:
        sv.pump(64)
        res = sv.poll(tk)
    sv.close()
    qo, io = oracle.evolve(oracle.make_problem(sp), sp["q0"], None, t_end=req["t_end"])
    e = err_vs_oracle(res["q"], qo)
    e.update(cells=req["n"] ** 2, t=req["t_end"], steps=res["steps"], oracle_steps=io["steps"])
    out["served_request"] = e
    return out


def cpu_single_thread(budget_s=3.0):
    """The oracle on one host thread at its parity sizes (run in a child
    process with OMP_NUM_THREADS=1): cell-updates/s per workload."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-single",
                        str(budget_s)], capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr[-300:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def _cpu_single_child(budget_s):
    import oracle
    from paper_1111_6583_gb300 import workloads as wl
    oracle.build()
    out = {"threads": oracle.threads()}

    def rate(spec, cells):
        # the first dt from the controller, then steps of that size
        P = oracle.make_problem(spec)
        q, info = oracle.evolve(P, spec["q0"], spec.get("aux"), t0=0.0, t_end=1e9, max_steps=1)
        dt = info["dt_next"]
        steps = 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < budget_s:
            q, _ = oracle.step(P, q, spec.get("aux"), dt)
            steps += 1
        return cells * steps / (time.perf_counter() - t0)

    out["acoustics_1d_2000"] = rate(wl.acoustics_1d(2000), 2000)
    out["dambreak_256"] = rate(wl.sw_dambreak_2d(n=256), 256 * 256)
    out["shock_bubble_256x128"] = rate(wl.shock_bubble_2d(nx=256, ny=128), 256 * 128)
    # a 64-member subset of the ensemble, two steps per member per round
    ens = wl.elasticity_ensemble(64)
    members = []
    for e in ens:
        sp = wl.elasticity_member(e["n"], e["amp"], e["width"])
        P = oracle.make_problem(sp)
        q, info = oracle.evolve(P, sp["q0"], sp["aux"], t0=0.0, t_end=1e9, max_steps=1)
        members.append((P, q, sp["aux"], info["dt_next"], e["n"]))
    tot, el = 0, 0.0
    while el < budget_s:
        for P, q, aux, dt, n in members:
            t0 = time.perf_counter()
            oracle.step(P, q, aux, dt)
            el += time.perf_counter() - t0
            tot += n
    out["ensemble_64_members"] = tot / el
    out["serving_64sq"] = rate(wl.sw_humps_2d(64, [(0.5, 0.5, 0.5, 0.1)], 1.0), 64 * 64)
    print(json.dumps(out))


def summary(line):
    """Short digest of the line's results (the last key, so that a record that
    keeps only the end of the output still has it)."""
    g = lambda *ks: _dig(line, ks)
    s = {
        "headline_fp64_1024": {"ms": g("ms_per_step"), "cu_s": g("value"),
                               "alu_frac": g("roofline", "frac"),
                               "peak_fp64_tf": g("roofline", "peak"),
                               "frac_of_measured": g("roofline", "frac_of_measured")},
        "peaks_measured": {k: g("peaks", k) for k in ("fp64_fma_tflops_measured",
                                                      "fp32_fma_tflops_measured", "hbm_gbs")},
        "dambreak_fp32_1024": {"ms": g("fp32", "ms_per_step"), "cu_s": g("fp32", "value"),
                               "alu_frac": g("fp32", "alu_frac")},
        "dambreak_8192": {p: {"ms": g("dambreak_8192", p, "ms_per_step"),
                              "alu_frac": g("dambreak_8192", p, "alu_frac")}
                          for p in ("fp64", "fp32")},
        "dambreak_4096": {p: {"ms": g("dambreak_4096", p, "ms_per_step"),
                              "hbm_frac": g("dambreak_4096", p, "hbm_frac"),
                              "alu_frac": g("dambreak_4096", p, "alu_frac")}
                          for p in ("fp64", "fp32")},
        "acoustics_1d_2000": {"us_step": g("acoustics_1d", "us_per_step"),
                              "steps_s": g("acoustics_1d", "steps_per_s")},
        "acoustics_1d_2p26": {p: {"ms": g("acoustics_1d_2p26", p, "ms_per_step"),
                                  "hbm_frac": g("acoustics_1d_2p26", p, "hbm_frac"),
                                  "alu_frac": g("acoustics_1d_2p26", p, "alu_frac")}
                              for p in ("fp64", "fp32")},
        "acoustics_3d_256": {"fp64_ms": g("acoustics_table1", "3d_fp64", "ms_per_step"),
                             "fp32_ms": g("acoustics_table1", "3d_fp32", "ms_per_step"),
                             "fp32_hbm_frac": g("acoustics_table1", "3d_fp32", "hbm_frac")},
        "shock_bubble_2048x1024": {p: {"ms": g("shock_bubble", p, "ms_per_step"),
                                       "alu_frac": g("shock_bubble", p, "alu_frac")}
                                   for p in ("fp64", "fp32")},
        "ensemble_4096": {"fp32_ms": g("batched_elasticity", "fp32_ms_per_step"),
                          "fp32_hbm_frac": g("batched_elasticity", "fp32_hbm_frac"),
                          "fp32_cu_s": g("batched_elasticity", "fp32_batched"),
                          "fp64_1at_cu_s": g("batched_elasticity", "fp64_one_at_a_time")},
        "serving": {p: {k: g(key, k) for k in ("p50_s", "p99_s",
                                                "throughput_cell_updates_per_s", "requests")}
                    for p, key in (("fp32", "serving"), ("fp64", "serving_fp64"))},
        "fp32_err_vs_oracle": {
            "dambreak_256_t1.5": g("errors_vs_oracle", "dambreak_256", "fp32", "l1_rel"),
            "shock_bubble_256x128_t0.2": g("errors_vs_oracle", "shock_bubble_256x128", "fp32",
                                           "l1_rel"),
            "ensemble_t50_max": max([r.get("l1_rel", 0) for r in
                                     g("errors_vs_oracle", "ensemble_members_t50") or []] or
                                    [None], key=lambda v: -1 if v is None else v),
            "served": g("errors_vs_oracle", "served_request", "l1_rel")},
        "fp64_err_vs_oracle_max": {
            "dambreak_256": g("errors_vs_oracle", "dambreak_256", "fp64", "max_rel"),
            "shock_bubble": g("errors_vs_oracle", "shock_bubble_256x128", "fp64", "max_rel")},
    }
    return _compact(s)


def _dig(d, ks):
    for k in ks:
        if not isinstance(d, dict) or k not in d:
            return None
        d = d[k]
    return d


def cpu_baseline_sw2d(n=1024, budget_s=12.0):
    """The oracle as it stands on the host cores: steps of the headline
    workload until about budget_s of CPU time."""
    import oracle
    from paper_1111_6583_gb300 import workloads as wl
    oracle.build()
    spec = wl.sw_dambreak_2d(n=n)
    P = oracle.make_problem(spec)
    q = spec["q0"]
    dt = 0.9 * P.dx / 2.0
    steps = 0
    t0 = time.perf_counter()
    while True:
        q, _ = oracle.step(P, q, None, dt)
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": n * n * steps / el, "unit": UNIT, "cores": oracle.threads(),
            "cpu_model": cpu_model(), "kind": "oracle",
            "sample": "%d steps of the %dx%d FP64 dam break (dt = 0.9 dx / 2)" % (steps, n, n)}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cb = cpu_baseline_sw2d(budget_s=max(5.0, 60.0 / max(1, args.steps + args.warmup)))
    # each timed step of the reference arm: one oracle step of the workload
    import oracle
    from paper_1111_6583_gb300 import workloads as wl
    spec = wl.sw_dambreak_2d(n=1024)
    P = oracle.make_problem(spec)
    q = spec["q0"]
    dt = 0.9 * P.dx / 2.0
    for _ in range(args.warmup):
        q, _ = oracle.step(P, q, None, dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q, _ = oracle.step(P, q, None, dt)
    el = time.perf_counter() - t0
    value = 1024 * 1024 * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "2D shallow-water dam break 1024x1024, classic Roe+HH, MC, "
                                   "transverse 2, FP64", "global_batch": 1, "seq_len": 0,
                       "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cb["cores"],
                             "cpu_model": cb.get("cpu_model"), "kind": "oracle",
                             "sample": "%d timed oracle steps of the 1024x1024 workload"
                                       % args.steps},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def profile_case(case, tile=None):
    """A short fixed launch sequence of one kernel for ncu captures (untimed):
    sw2d64/sw2d32 -- 2048^2 dam break, autotune (40 launches) then 3 steps;
    elast -- 1024-member FP32 elasticity batch, 5 fused steps;
    sharp, sharp_f32 -- 1024x512 shock-bubble FP64 / FP32, 2 SharpClaw steps (6
    stage launches, default tile);
    sw2d1024 -- the headline 1024^2 FP64 dam break, autotune (or --tile) then 4 steps;
    axisym -- 1280x320 axisymmetric shock-bubble FP64, tune then 3 steps;
    vc -- 1024^2 varying-medium acoustics with capacity FP64, 3 steps;
    acou2d -- 1024^2 constant-medium acoustics FP64, tile 128 x 32, 3 steps;
    psystem -- 1024^2 p-system checkerboard FP64, one SSP(10,4) step (10 stages);
    weno7 -- 1024x512 shock-bubble FP64, WENO7 + SSP(10,4), one step;
    acou3d -- 256^3 constant-medium acoustics FP64, 3 steps (acou3d128: 128^3,
    small enough for a multi-pass capture; acou3d_f32, acou3d128_f32: FP32);
    acou1d, acou1d_f32 -- 2^25-cell 1D acoustics, 3 steps (FP64, FP32);
    acou2000 -- the 2000-cell 1D acoustics of the latency workload, FP64, 20
    step attempts."""
    import torch
    from paper_1111_6583_gb300 import claw
    from paper_1111_6583_gb300 import workloads as wl
    if case in ("sw2d64", "sw2d32"):
        s = claw.Solver(wl.sw_dambreak_2d(n=2048), "fp64" if case == "sw2d64" else "fp32")
        print("tile", s.tune())
        s.set_t_end(1.5)
        s.advance(3)
    elif case == "sw2d1024":
        s = claw.Solver(wl.sw_dambreak_2d(n=1024), "fp64")
        print("tile", s.tune(*tile) if tile else s.tune())
        s.set_t_end(1.5)
        s.advance(4)
    elif case == "axisym":
        sp = wl.shock_bubble_axisym()
        s = claw.Solver(sp, "fp64")
        print("tile", s.tune())
        s.set_t_end(sp["t_end"])
        s.advance(3)
    elif case == "acou2d":
        sp = wl.acoustics_2d(n=1024)
        s = claw.Solver(sp, "fp64")
        s.tune(128, 32)
        s.set_t_end(sp["t_end"])
        s.advance(3)
    elif case == "psystem":
        sp = wl.psystem_checkerboard_2d(periods=16, cells_per_period=64)
        s = claw.Solver(sp, "fp64")
        s.set_t_end(sp["t_end"])
        s.advance(1)
    elif case == "weno7":
        sp = wl.shock_bubble_2d(nx=1024, ny=512)
        sp.update(weno_order=7, time_integrator="ssp104", cfl_desired=2.0, cfl_max=2.5)
        s = claw.Solver(sp, "fp64")
        s.set_t_end(0.2)
        s.advance(1)
    elif case in ("acou3d", "acou3d128", "acou3d_f32", "acou3d128_f32"):
        sp = wl.acoustics_3d(n=128 if "128" in case else 256)
        s = claw.Solver(sp, "fp32" if case.endswith("f32") else "fp64")
        s.set_t_end(sp["t_end"])
        s.advance(3)
    elif case == "acou2000":
        s = claw.Solver(wl.acoustics_1d(n=2000), "fp64")
        s.set_t_end(2.0)
        s.advance(20)
    elif case in ("acou1d", "acou1d_f32"):
        s = claw.Solver(wl.acoustics_1d(n=1 << 25, t_end=1e9),
                        "fp32" if case.endswith("f32") else "fp64")
        s.set_t_end(1e9)
        s.advance(3)
    elif case == "vc":
        sp = wl.acoustics_vc_2d(n=1024)
        s = claw.Solver(sp, "fp64")
        s.set_t_end(sp["t_end"])
        s.advance(3)
    elif case == "elast":
        ens = wl.elasticity_ensemble(1024)
        b = claw.Batch([wl.elasticity_member(e["n"], e["amp"], e["width"]) for e in ens], "fp32")
        b.advance(5)
    elif case in ("sharp", "sharp_f32"):
        s = claw.Solver(wl.shock_bubble_2d(nx=1024, ny=512),
                        "fp32" if case.endswith("f32") else "fp64")
        s.set_t_end(0.2)
        s.advance(2)
    else:
        raise SystemExit("unknown case " + case)
    torch.cuda.synchronize()
    print("ok")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-requests-fp64", type=int, default=60)
    ap.add_argument("--members", type=int, default=4096)
    ap.add_argument("--record-traffic", default=None,
                    help="write the headline kernel's traffic record from an ncu csv")
    ap.add_argument("--tile", default=None,
                    help="BW,H: fixed 2D tile shape for --case sw2d1024 and --record-traffic")
    ap.add_argument("--case", default=None,
                    help="run one short launch sequence for a profiler (sw2d64, sw2d32, sw2d1024, "
                         "elast, sharp, axisym, vc, acou2d, psystem, weno7, acou3d, acou3d128, "
                         "acou3d_f32, acou3d128_f32)")
    ap.add_argument("--cpu-single", type=float, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_single is not None:
        _cpu_single_child(args.cpu_single)
        return
    if args.record_traffic:
        if not args.tile:
            raise SystemExit("--record-traffic needs the --tile the capture ran")
        record_traffic(args.record_traffic, [int(v) for v in args.tile.split(",")])
        return
    if args.case:
        import __graft_entry__
        __graft_entry__.build()
        profile_case(args.case, [int(v) for v in args.tile.split(",")] if args.tile else None)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_6583_gb300 import claw
    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    hbm, hbm_kind = peaks()
    # measured ALU denominators (FMA probes, before the timed region: rate
    # and the SM clock it ran at) and the device's SM count and L2 size
    fp64_raw, fp64_mhz = claw.fma_peak("fp64", with_clock=True)
    fp32_raw, fp32_mhz = claw.fma_peak("fp32", with_clock=True)
    props = torch.cuda.get_device_properties(local)
    device = {"name": props.name, "sms": props.multi_processor_count,
              "l2_bytes": getattr(props, "L2_cache_size", None),
              "hbm_bytes": props.total_memory}
    copy_gbs = copy_rate_gbs()

    barrier(world)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        spec, ms, info, shape = bench_sw2d("fp64", args.steps, args.warmup, args.n)
    torch.cuda.synchronize()
    barrier(world)
    # ALU roofline denominators: the peaks derived from unit counts and the
    # maximum SM clock; the probes' rates, per SM clock and scaled to that
    # clock, are reported beside them (they vary from box to box by up to
    # ~15 % at the same clock, FP64 more than FP32)
    max_mhz = clk.summary().get("sm_max_mhz") or peaks_file().get("sm_max_mhz") or 2070.0
    fp64_tf, fp32_tf = FP64_PEAK_DERIVED_TFLOPS, FP32_PEAK_DERIVED_TFLOPS
    fp64_meas = fp64_raw * max_mhz / fp64_mhz if fp64_mhz > 0 else fp64_raw
    fp32_meas = fp32_raw * max_mhz / fp32_mhz if fp32_mhz > 0 else fp32_raw
    total_ms = max_over_ranks(sum(ms), world)
    cells = args.n * args.n
    accepted = info["accepted_in_timed"]
    value = replica_value(cells * accepted, total_ms, world)
    avg_ms = sum(ms) / len(ms)
    achieved_tf = SW2D_FLOPS_PER_CELL * cells / (avg_ms * 1e-3) / 1e12
    hbm_gbs = SW2D_BYTES_PER_CELL["fp64"] * cells / (avg_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "2D shallow-water dam break %dx%d, classic Roe+HH, MC, "
                               "transverse 2, FP64" % (args.n, args.n),
                   "global_batch": world, "seq_len": 0, "parallelism": "replicas",
                   "l2": "flushed between timed steps (512 MB write, untimed)"},
        # launch shape and accepted steps beside the workload (the workload
        # keys are the ones both arms share)
        "tile": {"bw": shape[0], "h": shape[1]},
        "accepted_steps": accepted,
        "gpu_launches": args.steps,
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": fp64_tf,
                     "unit": "TFLOP/s", "frac": achieved_tf / fp64_tf,
                     "traffic": recorded_traffic(shape),
                     "peak_kind": "derived: 152 SMs x 2.07 GHz x 2 FP64 FMA lanes x 2 FLOP",
                     "peak_measured": fp64_meas,
                     "frac_of_measured": achieved_tf / fp64_meas,
                     "peak_derived": FP64_PEAK_DERIVED_TFLOPS,
                     "flops_per_cell": SW2D_FLOPS_PER_CELL,
                     "hbm_gbs": hbm_gbs, "hbm_frac": hbm_gbs / hbm, "hbm_peak": hbm,
                     "hbm_peak_kind": hbm_kind},
        "peaks": {"fp64_fma_tflops_measured": fp64_meas, "fp32_fma_tflops_measured": fp32_meas,
                  "probe_raw": {"fp64_tflops": fp64_raw, "fp64_sm_mhz": fp64_mhz,
                                "fp32_tflops": fp32_raw, "fp32_sm_mhz": fp32_mhz,
                                "scaled_to_mhz": max_mhz},
                  "hbm_gbs": hbm, "hbm_copy_gbs_this_run": copy_gbs,
                  "hbm_nominal_gbs": 7900.0,
                  "hbm_kind": hbm_kind, "fp64_derived_tflops": FP64_PEAK_DERIVED_TFLOPS,
                  "fp32_derived_tflops": FP32_PEAK_DERIVED_TFLOPS},
        "device": device,
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_extras:
        ex = {}
        spec32, ms32, info32, shape32 = bench_sw2d("fp32", args.steps, args.warmup, args.n)
        avg32 = sum(ms32) / len(ms32)
        gbs32 = SW2D_BYTES_PER_CELL["fp32"] * cells / (avg32 * 1e-3) / 1e9
        ex["fp32"] = {"value": cells * info32["accepted_in_timed"] / (sum(ms32) * 1e-3),
                      "unit": UNIT, "ms_per_step": avg32, "hbm_gbs": gbs32,
                      "hbm_frac": gbs32 / hbm,
                      "alu_frac": SW2D_FLOPS_PER_CELL * cells / (avg32 * 1e-3) / 1e12 / fp32_tf,
                      "tile": list(shape32)}
        line["e2e"] = e2e_sw2d("fp64", max(5, args.steps // 4), 3, args.n)
        big = {}
        for p in ("fp64", "fp32"):
            _, msb, ib, shb = bench_sw2d(p, 10, 3, 4096)
            ab = sum(msb) / len(msb)
            gb = SW2D_BYTES_PER_CELL[p] * 4096 * 4096 / (ab * 1e-3) / 1e9
            big[p] = {"ms_per_step": ab, "value": 4096 * 4096 / (ab * 1e-3), "hbm_gbs": gb,
                      "hbm_frac": gb / hbm, "tile": list(shb),
                      "alu_frac": SW2D_FLOPS_PER_CELL * 4096 * 4096 / (ab * 1e-3) / 1e12
                      / (fp64_tf if p == "fp64" else fp32_tf)}
        ex["dambreak_4096"] = big
        # 8192^2 (1.6 GB per FP64 state copy), on the 4096^2 tile (no tuning
        # trials at this size)
        huge = {}
        for p in ("fp64", "fp32"):
            _, msh, _, shh = bench_sw2d(p, 3, 2, 8192, tile=big[p]["tile"])
            ah = sum(msh) / len(msh)
            gh = SW2D_BYTES_PER_CELL[p] * 8192 * 8192 / (ah * 1e-3) / 1e9
            huge[p] = {"ms_per_step": ah, "value": 8192 * 8192 / (ah * 1e-3), "hbm_gbs": gh,
                       "hbm_frac": gh / hbm, "tile": list(shh),
                       "alu_frac": SW2D_FLOPS_PER_CELL * 8192 * 8192 / (ah * 1e-3) / 1e12
                       / (fp64_tf if p == "fp64" else fp32_tf)}
        ex["dambreak_8192"] = huge
        ex["acoustics_1d"] = bench_acoustics_1d("fp64")
        a26 = {}
        for p in ("fp64", "fp32"):
            r = bench_acoustics_1d_hbm(p, 10, 3)
            r["hbm_frac"] = r["hbm_gbs"] / hbm
            r["alu_frac"] = (ACOU1D_FLOPS_PER_CELL * r["cells"] / (r["ms_per_step"] * 1e-3)
                             / 1e12 / (fp64_tf if p == "fp64" else fp32_tf))
            a26[p] = r
        ex["acoustics_1d_2p26"] = a26
        sb = {p: bench_shockbubble(p, 5, 3) for p in ("fp64", "fp32")}
        for p in ("fp64", "fp32"):
            fl = 3 * EULER2D_WENO5_FLOPS_PER_CELL_STAGE * 2048 * 1024
            sb[p]["alu_frac"] = fl / (sb[p]["ms_per_step"] * 1e-3) / 1e12 / (
                fp64_tf if p == "fp64" else fp32_tf)
        sb["fp64_weno7_ssp104"] = bench_shockbubble("fp64", 3, 3, weno_order=7,
                                                    integrator="ssp104")
        ex["shock_bubble"] = sb
        ex["psystem_checkerboard"] = {p: bench_psystem(p, 3, 3) for p in ("fp64", "fp32")}
        ax = {p: bench_axisym(p, 20, 3) for p in ("fp64", "fp32")}
        ax["fp64_split"] = bench_axisym("fp64", 20, 3, dim_split=1)
        ax["fp64_strang"] = bench_axisym("fp64", 20, 3, source_split="strang")
        ex["axisym_shock_bubble"] = ax
        at = {"2d_" + p: bench_acoustics_table1(p, 20, 3, 2, 1024) for p in ("fp64", "fp32")}
        at.update({"3d_" + p: bench_acoustics_table1(p, 5, 3, 3, 256) for p in ("fp64", "fp32")})
        # 3D: algorithmic bytes per cell and step over the four launches
        g3 = ACOU3D_BYTES_PER_CELL["fp32"] * 256 ** 3 / (at["3d_fp32"]["ms_per_step"] * 1e-3)
        at["3d_fp32"]["hbm_gbs"] = g3 / 1e9
        at["3d_fp32"]["hbm_frac"] = g3 / 1e9 / hbm
        ex["acoustics_table1"] = at
        ex["acoustics_vc_capacity"] = {p: bench_acoustics_vc(p, 10, 3) for p in ("fp64", "fp32")}
        try:
            be = bench_elasticity(args.members, 100, 16)
            gbe = ELAST1D_BYTES_PER_CELL["fp32"] * be["cells"] / (be["fp32_ms_per_step"] * 1e-3)
            be["fp32_hbm_gbs"] = gbe / 1e9
            be["fp32_hbm_frac"] = gbe / 1e9 / hbm
            be["fp32_alu_frac"] = (ELAST1D_FLOPS_PER_CELL * be["cells"] /
                                   (be["fp32_ms_per_step"] * 1e-3) / 1e12 / fp32_tf)
            ex["batched_elasticity"] = be
        except Exception as e:  # reported, not hidden
            ex["batched_elasticity"] = {"error": repr(e)}
        try:
            ex["serving"] = bench_serving(args.serve_requests, "fp32")
            ex["serving_every_request_per_attempt"] = bench_serving(
                args.serve_requests, "fp32", policy="all")
            ex["serving_fp64"] = bench_serving(args.serve_requests_fp64, "fp64")
            ex["serving_fp64"]["note"] = ("FP64 plain form on the first %d requests of the same "
                                          "stream (its queue grows without bound on the whole "
                                          "stream)" % args.serve_requests_fp64)
        except Exception as e:
            ex["serving"] = {"error": repr(e)}
        try:
            ex["errors_vs_oracle"] = errors_vs_oracle()
        except Exception as e:
            ex["errors_vs_oracle"] = {"error": repr(e)}
        line.update(_compact(ex))
        line["cpu_baseline"] = cpu_baseline_sw2d(args.n)
        line["cpu_single_thread"] = _compact(cpu_single_thread())
        line["summary"] = summary(line)
    elif rank == 0:
        line["e2e"] = e2e_sw2d("fp64", max(5, args.steps // 4), 3, args.n)
        line["cpu_baseline"] = cpu_baseline_sw2d(args.n, budget_s=5.0)
    if rank == 0:
        print(json.dumps(line, separators=(",", ":")))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
