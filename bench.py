#!/usr/bin/env python
"""Benchmark of the explicit shallow-water finite-volume step on one GB300.

Workload: the synthetic 13,004,160-triangle river mesh (meandering channel in
a 40 km x 15 km floodplain, ~50 % dry, inflow 8000 m^3/s, fixed downstream
level, Manning friction, Morton order), MUSCL-HLLC, FP32 state and fluxes with
FP64 mass and time.  One "step" is one explicit time step of the whole mesh,
so the metric is cell-updates/s = cells x steps / time.

Printed on one JSON line (rank 0): the device-timed value (inputs resident,
CUDA events on the library's stream), the end-to-end value through the C ABI
with host buffers, the roofline of the dominant kernel against the measured
HBM peak, the FP64 GPU path and the FP32-vs-FP64 error at matched time, the
FP64 oracle timed on the host cores (cpu_baseline), and the SM clocks sampled
during the timed region.

--impl reference times the FP64 CPU oracle instead (the reference arm).
With torchrun (N > 1) every rank advances its own independent river (a
replica with its own seed): no data-path collective; value = all cells x
steps / max over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s MUSCL-HLLC 13M tri, FP32 vs FP64 at stated error; % HBM peak"
UNIT = "cell-updates/s"
SCHEME_NAMES = {"muscl": "MUSCL-HLLC", "muscl_edge": "edge-upwind MUSCL-HLLC", "hllc": "first-order HLLC",
                "waf": "WAF-HLLC"}
RIVER_GRID = (4160, 1563)
SEED = 20230733

# Algorithmic bytes per cell and launch: every array element the kernel must
# touch counted once (neighbour gathers assumed to hit in cache).
#   split MUSCL prep : state 3 + z + nbr(3 int) + scaled normals 6, writes 12 face values (the
#                      centroid offsets of the gradient come from the neighbours' normals)
#   split MUSCL flux : state 3 + z + nbr + normals 6 + own face values 12 + Manning n, writes state 3
#   fused MUSCL      : state 3 + z + nbr + normals 6 + n, writes state 3 (the whole step)
#   HLLC flux        : state 3 + z + nbr + normals 6 + n, writes state 3
def algo_bytes(kind: str, scheme: str, precision: str, wet: float = 1.0) -> float:
    """Bytes a kernel itself reads and writes per cell; for the split MUSCL kernels a dry cell
    (h <= h_eps) stores and reads no face values, so their figure is the mix at wet fraction `wet`
    (prep: wet 100, dry 8 B in FP32; flux: wet 116, dry 68 B).  The tile step's figure counts the
    12 B of neighbour words that its plan replaces; the plan itself is 16-18 B per cell on river
    meshes (swe_tile_plan_info), so the kernel reads about 4-6 B per cell more than this."""
    f = 4 if precision == "fp32" else 8
    nbr = 12
    if scheme in ("muscl", "muscl_edge") and kind == "prep":
        return wet * (3 * f + f + nbr + 6 * f + 12 * f) + (1.0 - wet) * 2 * f
    if scheme in ("muscl", "muscl_edge") and kind == "flux":
        return wet * (3 * f + f + nbr + 6 * f + 12 * f + f + 3 * f) + (1.0 - wet) * (3 * f + f + nbr + 6 * f + f + 3 * f)
    if kind == "fused":
        return 3 * f + f + nbr + 6 * f + f + 3 * f
    if scheme == "hllc" and kind == "flux":
        return 3 * f + f + nbr + 6 * f + f + 3 * f
    if scheme == "waf" and kind == "prep":
        return 3 * f + nbr + 3 * f + f + 4 * f + 12 * f      # reads nbr state, writes P and U
    if scheme == "waf" and kind == "flux":
        return 3 * f + f + nbr + 6 * f + 6 * f + 4 * f + 12 * f + f + 3 * f
    return 0


def step_bytes_ideal(scheme: str, precision: str) -> int:
    """Bytes per cell-update of the whole step if every array is read or written once."""
    return algo_bytes("fused" if scheme != "hllc" else "flux", scheme, precision)


def roofline_bytes(scheme: str, precision: str) -> int:
    """Algorithmic bytes per cell-update of the roofline: every array element touched once per step,
    neighbour gathers assumed to hit in cache, LSQ centroid offsets counted as stored (24 B in FP32):
    FP32 MUSCL / WAF 92 B (state read and written 24, bed and Manning n 8, neighbour words 12, scaled
    normals 24, offsets 24), first-order HLLC 68 B (no offsets); FP64 172 B and 124 B."""
    f = 4 if precision == "fp32" else 8
    base = 6 * f + 2 * f + 12 + 6 * f             # state r+w, z + n, neighbour words, scaled normals
    return base + (6 * f if scheme != "hllc" else 0)


# Kernel names as ncu lists them, per profiled kind and path.
KERNEL_NAMES = {("fused", "fused"): "k_tile", ("split", "flux"): "k_flux", ("split", "prep"): "k_prep"}


def roofline_entry(scheme, n, step_ms, prof, kname, peak, peak_src, traffic, wet=1.0):
    """The contract's roofline object: the whole step and its dominant kernel against the measured HBM
    copy rate, each with the algorithmic bytes of roofline_bytes() per cell-update (frac is the step's;
    with the one-pass tile step the step is one launch of the dominant kernel); each kernel's own
    bytes (what it reads and writes, face-value scratch included, at the state's wet fraction) under
    own_bytes; traffic is the dominant kernel's DRAM bytes per launch from the stored ncu counters."""
    per_cell = roofline_bytes(scheme, "fp32")
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / prof[dom][1]
    step_ach = per_cell * n / (step_ms / 1e3) / 1e9
    dom_ach = per_cell * n / (dom_ms / 1e3) / 1e9
    own = {}
    for k, (tot, cnt) in prof.items():
        b = algo_bytes(k, scheme, "fp32", wet)
        if b:
            a = b * n / (tot / cnt / 1e3) / 1e9
            own[k] = {"bytes_per_cell": b, "ms": tot / cnt, "achieved": a, "frac": a / peak}
    if own:
        own["wet_fraction"] = wet
    extra = {}
    if traffic is not None:
        extra["traffic_source"] = ("dram__bytes_read.sum + dram__bytes_write.sum of the dominant kernel, ncu on the "
                                   "3,252,084-cell river of the same generator (profiles/ncu_traffic.json), "
                                   "scaled to this launch by the cell count")
    return {"bound": "hbm", "achieved": step_ach, "peak": peak, "unit": "GB/s", "frac": step_ach / peak,
            "traffic": traffic, **extra, "peak_source": peak_src, "algo_bytes_per_cell": per_cell,
            "scope": "whole step (all launches of one time step)", "step_ms": step_ms,
            "kernel": {"name": KERNEL_NAMES.get((kname, dom), dom), "ms": dom_ms, "achieved": dom_ach,
                       "frac": dom_ach / peak},
            "per_kernel_ms": {k: v[0] / v[1] for k, v in prof.items()}, "own_bytes": own}


# The files the split kernels (k_prep_*, k_flux*) and the tile step (k_tile)
# are compiled from: stored ncu counters stay valid while these hash the same.
KERNEL_SOURCES = ("paper_2307_16758_gb300/csrc/swe_kernels.cu", "paper_2307_16758_gb300/csrc/swe_split.cuh",
                  "paper_2307_16758_gb300/csrc/swe_device.cuh", "paper_2307_16758_gb300/csrc/swe_dev.h",
                  "paper_2307_16758_gb300/csrc/swe_tile.cu", "paper_2307_16758_gb300/csrc/swe_tile.cuh",
                  "paper_2307_16758_gb300/csrc/swe_async.cuh", "include/swe.h")


def kernel_source_sha() -> str:
    """Hash of the kernel sources' code: comments and blank space do not count, so that
    stored counters outlive edits of the prose around the code."""
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        text = open(os.path.join(ROOT, p), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_counters(kernel_key: str):
    """Per-cell counters of a kernel from the committed ncu summary, if taken on the current kernels."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path)).get(kernel_key)
    if not d or d.get("source_sha") != kernel_source_sha():
        return None
    return d


def ncu_traffic(kernel_key: str, cells: int):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current kernels."""
    d = ncu_counters(kernel_key)
    return float(d["dram_bytes_per_cell"]) * cells if d else None


def issue_roofline(kernel_key: str, cells: int, kernel_ms: float, sm_mhz: float, n_sm: int):
    """The kernel against the SMs' instruction-issue rate (one warp instruction per scheduler and
    clock, four schedulers per SM), with the warp instructions per cell that ncu counted."""
    d = ncu_counters(kernel_key)
    if not d or "warp_inst_per_cell" not in d or not sm_mhz:
        return None
    peak = 4.0 * n_sm * sm_mhz * 1e6 / 1e9                     # G warp instructions / s
    achieved = float(d["warp_inst_per_cell"]) * cells / (kernel_ms / 1e3) / 1e9
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "G warp-inst/s",
            "frac": achieved / peak, "warp_inst_per_cell": d["warp_inst_per_cell"],
            "peak_source": f"4 schedulers x {n_sm} SMs x {sm_mhz:.0f} MHz (median SM clock under load)"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0, t1):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [l for (t, l) in self.lines if t0 - 0.05 <= t <= t1 + 0.15] or [l for (_, l) in self.lines[-3:]]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The sum of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(cells: int, steps: int, ms_local: float, dist=None, device="cpu"):
    """Whole-job cell-updates/s: every rank's cells x steps over the slowest rank's time (replicas,
    no data-path collective).  Returns (value, max ms)."""
    ms = max_over_ranks(ms_local, dist, device)
    total = sum_over_ranks(cells, dist, device)
    return total * steps / (ms / 1e3), ms


def river_workload(rank: int, scale: float, moving: bool = False):
    from paper_2307_16758_gb300 import workloads as W
    nx, ny = RIVER_GRID
    if scale != 1.0:
        nx, ny = W.river_grid_for_cells(int(2 * nx * ny * scale))
    w = W.river(nx, ny, seed=SEED + 1000 * rank)
    if moving:
        # every cell wet and in motion, no two neighbours alike: a free surface 4 m above the
        # median bed with a 0.3 m ripple (at least 0.5 m deep), a varying downstream flow and a
        # cross flow, so that no edge takes the equal-state shortcut and no cell a zero gradient
        cx, cy = w.centroids()
        eta = float(np.median(w.z)) + 4.0 + 0.3 * np.sin(cx / 53.0) * np.cos(cy / 71.0)
        w.h = np.maximum(eta - w.z, 0.5)
        w.hu = w.h * (0.6 + 0.2 * np.sin(cy / 37.0))
        w.hv = w.h * (0.3 * np.cos(cx / 41.0))
    return w, (nx, ny)


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle as it stands
# ---------------------------------------------------------------------------

def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2307_16758_gb300 import workloads as W
    oracle.build()
    # the oracle on the bench's own workload, the full 13M-cell river: W untimed warm-up steps (at most
    # 10), then one oracle step per bench step for as many of the K steps as fit in about two minutes of
    # host time (at least 3); the line states how many were timed
    nx, ny = RIVER_GRID
    w = W.river(nx, ny, seed=SEED)
    om = oracle.Mesh(w.nodes, w.tris, w.bnd_edges, w.bnd_tag)
    cores = os.cpu_count() or 1
    o = oracle.opts("muscl", threads=cores)
    state = (w.h, w.hu, w.hv)

    def one_step(st):
        t0 = time.perf_counter()
        h, hu, hv, dts, d = oracle.run(om, o, w.z, w.nman, *st, 1, q_in=w.q_in, level=w.level)
        return (h, hu, hv), time.perf_counter() - t0

    t_warm = []
    for _ in range(max(1, min(args.warmup, 10))):
        state, t = one_step(state)
        t_warm.append(t)
    n_timed = int(min(args.steps, max(3, 120.0 // max(min(t_warm), 1e-3))))
    t_steps = []
    for _ in range(n_timed):
        state, t = one_step(state)
        t_steps.append(t)
    el = sum(t_steps)
    value = om.n * len(t_steps) / el
    sample = (f"one FP64 MUSCL-HLLC Euler step of the full {om.n}-cell river per bench step, OpenMP over "
              f"cells; {n_timed} of the {args.steps} steps timed (about two minutes of host time) after "
              f"{len(t_warm)} warm-up steps")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / len(t_steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"river {RIVER_GRID[0]}x{RIVER_GRID[1]} jittered grid, "
                               f"{2 * RIVER_GRID[0] * RIVER_GRID[1]} triangles, MUSCL-HLLC, Euler, CFL 0.9, "
                               "Morton order",
                   "cells": om.n, "timed_steps": n_timed, "scheme": "muscl", "precision": "fp64"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def rel_l1(a, b):
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


def rel_inf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def run_gpu(args):
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    from paper_2307_16758_gb300 import swe

    if rank == 0 or ws == 1:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    swe.load_library()
    stream = torch.cuda.current_stream()

    w, grid = river_workload(rank, args.scale, args.moving)
    mesh = swe.Mesh.from_workload(w, "morton")
    n = mesh.n
    p32 = swe.swe_params_default(args.scheme, "fp32", kernel=args.kernel, hr_order=args.hr_order)
    if args.block:
        p32.block = args.block
    st = swe.State.from_workload(mesh, p32, w)
    part = None
    if args.parts > 1:                       # boundary-first schedule over Morton sub-domains
        part = swe.Partition(mesh, args.parts)
        st.set_partition(part)
    dev_bytes, kernel_used, block = st.info()
    kname = {1: "split", 2: "fused"}.get(kernel_used, str(kernel_used))

    # warm-up, then the timed region (production path, inputs resident in HBM)
    st.step(args.warmup, args.cfl)
    st.sync()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tw0 = time.time()
    e0.record(stream)
    st.step(args.steps, args.cfl)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    tw1 = time.time()
    if dist:
        dist.barrier()
    clocks = sampler.stop(tw0, tw1)
    ms = e0.elapsed_time(e1)
    st.sync()
    value, ms = job_throughput(n, args.steps, ms, dist, "cuda")

    # per-kernel device time over a second timed region of the same length
    st.profile_begin()
    st.step(args.steps, args.cfl)
    prof = st.profile_end()
    launches = sum(c for _, c in prof.values())
    dom = max(prof, key=lambda k: prof[k][0])
    peak, peak_src = measured_peaks()
    skey = args.scheme + (":hr2" if args.hr_order == 2 else "")      # counters key of the kernels
    traffic = ncu_traffic(f"{kname}:{dom}:{skey}:fp32", n)
    step_ms = ms / args.steps

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory().numpy()
    hin = [pin(w.h), pin(w.hu), pin(w.hv)]
    hout = [pin(np.zeros(n)) for _ in range(3)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st.set_state(*hin)
    st.step(args.steps, args.cfl)
    st.get_state(hout)
    mass = st.mass()
    t1 = time.perf_counter()
    e2e, _ = job_throughput(n, args.steps, (t1 - t0) * 1e3, dist, "cuda")
    h2d = 3 * 8 * n / args.steps
    d2h = (3 * 8 * n + 8 * 3) / args.steps
    # the same with one call per step and the step's result (its mass budget, 24 bytes) read back
    # after every step, as a caller that monitors the run would
    k1 = min(args.steps, 500)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st.set_state(*hin)
    for _ in range(k1):
        st.step(1, args.cfl)
        st.mass()
    st.get_state(hout)
    t1 = time.perf_counter()
    e2e1, _ = job_throughput(n, k1, (t1 - t0) * 1e3, dist, "cuda")

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {
            "workload": f"river {grid[0]}x{grid[1]} jittered grid, {n} triangles, "
                        f"{SCHEME_NAMES[args.scheme]} FP32 bulk "
                        "(FP64 mass/time), Euler, CFL 0.9, Morton order"
                        + (", second-order hydrostatic reconstruction" if args.hr_order == 2 else "")
                        + (", all-wet moving start" if args.moving else ""),
            "cells": n, "scheme": args.scheme, "hr_order": args.hr_order, "precision": "fp32", "time_scheme": "euler", "kernel": kname,
            "block": block, "device_bytes": dev_bytes,
            "l2": f"inputs larger than L2: {dev_bytes / 1e9:.2f} GB resident per state, no flush needed",
            "parallelism": "replicas" if ws > 1 else "single GPU", "seed": SEED,
            "schedule": f"boundary-first, {args.parts} parts" if args.parts > 1 else "plain",
        },
        "roofline": roofline_entry(args.scheme, n, step_ms, prof, kname, peak, peak_src, traffic,
                                   float(np.mean(w.h > p32.h_eps))),
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "scope": "swe_set_state from pinned host arrays, swe_step(K), swe_get_state and swe_mass into "
                         "host memory, all inside the timed region; the state crosses once per run, so the "
                         "bytes per step are the run's copies over its K steps",
                "per_step_calls": {"value": e2e1, "unit": UNIT, "steps": k1,
                                   "h2d_bytes_per_step": 3 * 8 * n / k1, "d2h_bytes_per_step": 24 + 3 * 8 * n / k1,
                                   "scope": "the same with swe_step(1) and a swe_mass read-back (24 bytes) "
                                            "after every step"}},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    iss = {k: issue_roofline(f"{kname}:{k}:{skey}:fp32", n, v[0] / v[1], clocks.get("sm_mhz") or 0.0,
                             torch.cuda.get_device_properties(local).multi_processor_count)
           for k, v in prof.items()}
    if any(iss.values()):
        out["issue_roofline"] = {k: v for k, v in iss.items() if v}

    c32 = ncu_counters(f"{kname}:{dom}:{skey}:fp32")
    if c32 and "flops_per_cell" in c32:
        out["roofline"]["flops_per_cell"] = c32["flops_per_cell"]
    if c32 and "dram_bytes_per_cell" in c32:
        out["roofline"]["dram_bytes_per_cell_measured"] = c32["dram_bytes_per_cell"]
    if rank == 0 and not args.quick:
        out.update(fp64_comparison(args, mesh, w, swe, torch, p32))
        out["fp64"]["fp32_speedup"] = out["fp64"]["ms_per_step"] / step_ms
        out["alu_peaks"] = alu_peaks(swe, torch, local, clocks)
        out["fp64"]["roofline"] = fp64_alu_roofline(out["fp64"], out["alu_peaks"], skey, n)
        if ws == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(w, n)
        if ws == 1 and not args.no_extras:
            out["river_4m"] = river4m_study(args, swe, torch)
            out["ensemble_40m"] = ensemble_study(args, swe, torch)
    if rank == 0:
        print(json.dumps(out))
    st.close()
    if part is not None:
        part.close()
    mesh.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def alu_peaks(swe, torch, dev, clocks):
    """FMA rates of this GPU measured by the library's probe, next to the figures that the
    unit counts give (per SM and clock: 128 FP32 FMAs, 2 FP64 FMAs) at the highest SM clock."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clocks.get("sm_max_mhz") or 0.0
    stream = torch.cuda.current_stream().cuda_stream
    return {"unit": "TFLOP/s",
            "fp32": swe.swe_fma_peak("fp32", stream=stream) / 1e12,
            "fp64": swe.swe_fma_peak("fp64", stream=stream) / 1e12,
            "fp32_from_units": 2 * 128 * sms * mhz * 1e6 / 1e12,
            "fp64_from_units": 2 * 2 * sms * mhz * 1e6 / 1e12,
            "source": "swe_fma_peak (8 independent FMA chains per thread, 8 x 256 threads per SM)"}


def fp64_alu_roofline(fp64, peaks, skey, n):
    """The FP64 path's dominant kernel against the measured FP64 FMA rate: ncu's FP64 operations per
    cell (add, mul, 2 x fma) over the kernel's CUDA-event time."""
    prof = fp64.get("per_kernel_ms", {})
    if not prof:
        return None
    dom = max(prof, key=prof.get)
    ms = prof[dom]
    c = ncu_counters(f"{fp64.get('kernel', 'split')}:{dom}:{skey}:fp64")
    if not c or "fp64_flops_per_cell" not in c or not ms:
        return None
    achieved = c["fp64_flops_per_cell"] * n / (ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": KERNEL_NAMES.get((fp64.get("kernel", "split"), dom), dom),
            "achieved": achieved, "peak": peaks["fp64"], "unit": "TFLOP/s",
            "frac": achieved / peaks["fp64"], "fp64_flops_per_cell": c["fp64_flops_per_cell"],
            "peak_source": "measured FP64 FMA rate (swe_fma_peak)", "kernel_ms": ms}


def fp64_comparison(args, mesh, w, swe, torch, p32_timed):
    """FP64 GPU path: its throughput, and the error of the timed FP32 configuration against it at
    matched time.  The FP64 run takes the FP32 run's thresholds (h_eps, r_eps: same algorithm, only
    the precision differs) and config 3's step count; the FP32 run replays its time steps."""
    n = mesh.n
    m_steps = args.fp64_steps
    p64 = swe.swe_params_default(args.scheme, "fp64", kernel=args.kernel, hr_order=args.hr_order)
    p64.h_eps, p64.r_eps = p32_timed.h_eps, p32_timed.r_eps
    s64 = swe.State.from_workload(mesh, p64, w)
    s64.step(3, args.cfl)
    s64.sync()
    s64.close()
    s64 = swe.State.from_workload(mesh, p64, w)
    kernel64 = {1: "split", 2: "fused"}.get(s64.info()[1], "split")
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s64.step(m_steps, args.cfl)
    e1.record(stream)
    e1.synchronize()
    ms64 = e0.elapsed_time(e1)
    dts = s64.dt_history(m_steps)
    h64, hu64, hv64 = s64.get_state()
    mass64 = s64.mass()
    # per-kernel device time of the FP64 path (CUDA events around each launch)
    s64.profile_begin()
    s64.step(10, args.cfl)
    prof64 = s64.profile_end()
    s32 = swe.State.from_workload(mesh, p32_timed, w)
    m0 = s32.mass()[0]
    s32.step_dt(dts)
    h32, hu32, hv32 = s32.get_state()
    mass32 = s32.mass()
    err = state_error(w, h32, hu32, hv32, h64, hu64, hv64)
    err.update({"steps": m_steps, "t_end": float(np.sum(dts)), "h_eps": p32_timed.h_eps, "r_eps": p32_timed.r_eps,
                "thresholds": "the timed FP32 run's h_eps and r_eps on both sides",
                "mass_drift_fp32": abs(mass32[0] - m0 - mass32[1] - mass32[2]) / m0,
                "mass_drift_fp64": abs(mass64[0] - m0 - mass64[1] - mass64[2]) / m0})
    s32.close()
    s64.close()
    v64 = n * m_steps / (ms64 / 1e3)
    return {"fp64": {"value": v64, "unit": UNIT, "ms_per_step": ms64 / m_steps, "steps": m_steps,
                     "kernel": kernel64, "per_kernel_ms": {k: v[0] / v[1] for k, v in prof64.items()}},
            "error_fp32_vs_fp64": err}


def state_error(w, h32, hu32, hv32, h64, hu64, hv64):
    """Relative L1 / Linf of h and the discharges, first over the cells the flow has reached (a cell
    still at rest is exact in both precisions, so the whole-mesh figure dilutes the error), then over
    the mesh; and L1 of h against the FP64 change of h since t = 0."""
    qs = max(np.abs(hu64).max(), np.abs(hv64).max(), 1e-300)
    act = (h64 != w.h) | (hu64 != 0) | (hv64 != 0)
    dh = np.abs(h64 - w.h)[act].sum()
    return {
        "active_cells": int(act.sum()),
        "l1_h_active": rel_l1(h32[act], h64[act]) if act.any() else 0.0,
        "l1_q_active": float((np.abs(hu32 - hu64) + np.abs(hv32 - hv64))[act].sum()
                             / max((np.abs(hu64) + np.abs(hv64))[act].sum(), 1e-300)),
        "l1_h_vs_change": float(np.abs(h32 - h64)[act].sum() / dh) if dh > 0 else 0.0,
        "l1_h": rel_l1(h32, h64), "linf_h": rel_inf(h32, h64),
        "l1_hu": rel_l1(hu32, hu64), "linf_hu": float(np.abs(hu32 - hu64).max() / qs),
        "l1_hv": rel_l1(hv32, hv64), "linf_hv": float(np.abs(hv32 - hv64).max() / qs),
    }


def cpu_baseline(w, n):
    """The FP64 oracle as it stands, on the host cores: 20 steps of the full mesh on all cores and
    one step on one core (bounded samples)."""
    import oracle
    import platform
    oracle.build()
    om = oracle.Mesh(w.nodes, w.tris, w.bnd_edges, w.bnd_tag)
    cores = os.cpu_count() or 1
    steps = 20
    t0 = time.perf_counter()
    oracle.run(om, oracle.opts("muscl", threads=cores), w.z, w.nman, w.h, w.hu, w.hv, steps, q_in=w.q_in,
               level=w.level)
    el = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.run(om, oracle.opts("muscl", threads=1), w.z, w.nman, w.h, w.hu, w.hv, 1, q_in=w.q_in, level=w.level)
    el1 = time.perf_counter() - t0
    return {"value": n * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "one_core": {"value": n / el1, "unit": UNIT, "sample": "1 step of the full mesh, 1 thread"},
            "cpu": platform.processor() or platform.machine(),
            "sample": f"{steps} FP64 MUSCL-HLLC Euler steps of the full {n}-cell river mesh "
                      f"(mesh build excluded), OpenMP over cells"}


def ensemble_study(args, swe, torch):
    """64 river scenarios of uneven size (40M cells in total), MUSCL-HLLC FP32, one batched launch
    per step (autotuned) against one launch sequence per member; per-member FP32 error against the
    FP64 path (at the FP32 thresholds) after a bounded number of replayed steps."""
    from paper_2307_16758_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    sizes = W.ensemble_sizes(n_members=args.members, total=int(40_000_000 * args.scale))
    ws = [W.ensemble_member(k, int(c)) for k, c in enumerate(sizes)]
    meshes = [swe.Mesh.from_workload(w) for w in ws]
    n = sum(m.n for m in meshes)
    p = swe.swe_params_default("muscl", "fp32")
    states = [swe.State.from_workload(m, p, w) for m, w in zip(meshes, ws)]
    ens = swe.Ensemble(states)
    kernel, block, tune_ms = ens.autotune(meshes, trial_steps=4)
    steps = max(args.steps, 24)
    ens.step(args.warmup, args.cfl)
    ens.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ens.step(steps, args.cfl)
    e1.record(stream)
    e1.synchronize()
    ms_batched = e0.elapsed_time(e1) / steps
    # one launch sequence per member per step
    e0.record(stream)
    for _ in range(steps):
        for st in states:
            st.step(1, args.cfl)
    e1.record(stream)
    e1.synchronize()
    ms_separate = e0.elapsed_time(e1) / steps
    ens.sync()
    wet = sum(int((st.get_state()[0] > p.h_eps).sum()) for st in states) / n     # prep's bytes depend on it
    ens.close()
    for st in states:
        st.close()
    # per-member FP32 error against the FP64 GPU path at matched time, same thresholds
    m_steps = min(args.fp64_steps, 200)
    errs = []
    p64 = swe.swe_params_default("muscl", "fp64")
    p64.h_eps, p64.r_eps = p.h_eps, p.r_eps
    for m, w in zip(meshes, ws):
        s64 = swe.State.from_workload(m, p64, w)
        s64.step(m_steps, args.cfl)
        dts = s64.dt_history(m_steps)
        h64 = s64.get_state()[0]
        s32 = swe.State.from_workload(m, p, w)
        s32.step_dt(dts)
        h32 = s32.get_state()[0]
        act = (h64 != w.h)
        errs.append((rel_l1(h32, h64), rel_l1(h32[act], h64[act]) if act.any() else 0.0))
        s64.close()
        s32.close()
    for m in meshes:
        m.close()
    peak, src = measured_peaks()
    per_cell = roofline_bytes("muscl", "fp32")
    ach = per_cell * n / (ms_batched / 1e3) / 1e9
    e = np.array(errs)
    return {
        "workload": f"ensemble of {len(ws)} river scenarios, {n} cells, sizes {int(sizes.min())}-{int(sizes.max())}, "
                    "own inflow, Manning n and initial level each",
        "cells": n, "steps": steps, "kernel": kernel, "block": block, "autotune_ms_per_step": tune_ms,
        "batched": {"value": n / (ms_batched / 1e3), "unit": UNIT, "ms_per_step": ms_batched},
        "separate_launches": {"value": n / (ms_separate / 1e3), "unit": UNIT, "ms_per_step": ms_separate,
                              "launches_per_step": len(ws) * (2 if kernel == "split" else 1)},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                     "algo_bytes_per_cell": per_cell, "peak_source": src, "wet_fraction": wet},
        "error_fp32_vs_fp64": {"steps": m_steps, "h_eps": p.h_eps, "l1_h_active_max": float(e[:, 1].max()),
                               "l1_h_active_median": float(np.median(e[:, 1])), "l1_h_max": float(e[:, 0].max())},
    }


def run_ensemble(args):
    """The batched ensemble on its own (one JSON line)."""
    import torch

    from paper_2307_16758_gb300 import swe
    import __graft_entry__

    __graft_entry__.build()
    swe.load_library()
    r = ensemble_study(args, swe, torch)
    print(json.dumps({"metric": "cell-updates/s, batched ensemble (MUSCL-HLLC FP32)", "value": r["batched"]["value"],
                      "unit": UNIT, "n_gpus": 1, "steps": r["steps"], "warmup": args.warmup,
                      "ms_per_step": r["batched"]["ms_per_step"], "higher_is_better": True, "dtype": "f32",
                      "data": "synthetic", "config": {"workload": r["workload"], "kernel": r["kernel"],
                                                      "block": r["block"]},
                      "ensemble": r}))


def river4m_study(args, swe, torch):
    """WAF-HLLC against MUSCL-HLLC on the 4,000,920-cell river (the 13M generator at 4M cells), FP32
    with compensated FP64 mass: GPU time per step and its HBM rate, FP32 error and mass drift against
    the FP64 path at the FP32 thresholds after 2000 replayed steps, wetting front in both precisions."""
    from paper_2307_16758_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    w = W.river(2310, 866)
    mesh = swe.Mesh.from_workload(w, "morton")
    n = mesh.n
    steps = 2000
    peak, src = measured_peaks()
    cx = w.centroids()[0]
    dry0 = w.h <= 0.0

    def front(hh):
        m = (hh > 1e-3) & dry0
        return float(cx[m].max()) if m.any() else None

    res = {"workload": "river 2310x866 jittered grid, 4,000,920 triangles", "cells": n, "steps": steps, "schemes": {}}
    for scheme in ("muscl", "waf"):
        p32 = swe.swe_params_default(scheme, "fp32")
        st = swe.State.from_workload(mesh, p32, w)
        st.step(24, args.cfl)
        st.sync()
        st.close()
        st = swe.State.from_workload(mesh, p32, w)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st.step(steps, args.cfl)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        st.close()
        p64 = swe.swe_params_default(scheme, "fp64")
        p64.h_eps, p64.r_eps = p32.h_eps, p32.r_eps
        s64 = swe.State.from_workload(mesh, p64, w)
        s64.step(steps, args.cfl)
        dts = s64.dt_history(steps)
        h64, hu64, hv64 = s64.get_state()
        s64.close()
        s32 = swe.State.from_workload(mesh, p32, w)
        m0 = s32.mass()[0]
        s32.step_dt(dts)
        h32, hu32, hv32 = s32.get_state()
        mass32 = s32.mass()
        s32.close()
        per_cell = roofline_bytes(scheme, "fp32")
        ach = per_cell * n / (ms / 1e3) / 1e9
        speed = lambda hh, qx, qy: float(np.where(hh > 1e-3, np.hypot(qx, qy) / np.maximum(hh, 1e-300), 0.0).max())
        err = state_error(w, h32, hu32, hv32, h64, hu64, hv64)
        err["mass_drift_fp32"] = abs(mass32[0] - m0 - mass32[1] - mass32[2]) / m0
        res["schemes"][scheme] = {
            "value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "hbm": {"achieved": ach, "unit": "GB/s", "frac": ach / peak, "algo_bytes_per_cell": per_cell,
                    "peak_source": src},
            "error_fp32_vs_fp64": err, "t_end": float(np.sum(dts)),
            "front_x": {"fp32": front(h32), "fp64": front(h64), "unit": "m"},
            "max_speed": {"fp32": speed(h32, hu32, hv32), "fp64": speed(h64, hu64, hv64), "unit": "m/s"},
        }
    mesh.close()
    return res


def run_time_error(args):
    """Time against L2 error on the paper's wet-bed dam break (Sec. 6.3: [0,10] x [0,1], h = 1 | 0.5,
    t = 1 s) for 20k-600k cells, every scheme, FP32 and FP64: GPU time of the CFL steps that reach
    t = 1 (CUDA events, after an untimed run that counts them) and the area-weighted relative L2
    error of h against the closed form (Stoker) at the time reached.  The MUSCL schemes also run
    with Heun steps and with Euler at CFL 0.45 (Euler at 0.9 does not converge for them)."""
    import torch

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from exact import stoker
    from paper_2307_16758_gb300 import swe
    from paper_2307_16758_gb300 import workloads as W
    import __graft_entry__

    __graft_entry__.build()
    swe.load_library()
    stream = torch.cuda.current_stream()
    rows = []
    for cells in (20_000, 50_000, 100_000, 200_000, 400_000, 600_000):
        ny = max(2, int(round(math.sqrt(cells / 20.0))))
        nx = int(round(cells / (2.0 * ny)))
        w = W.dam_break_1d(nx, ny, 10.0, 1.0, 1.0, 0.5, x_dam=5.0)
        mesh = swe.Mesh.from_workload(w, "morton")
        area = mesh.export()["area"][np.argsort(mesh.export()["perm"])]
        cx, _ = w.centroids()
        runs = [("hllc", "euler", 0.9), ("waf", "euler", 0.9)]
        for s in ("muscl", "muscl_edge"):
            runs += [(s, "euler", 0.9), (s, "heun", 0.9), (s, "euler", 0.45)]
        for precision in ("fp32", "fp64"):
            for scheme, ts, cfl in runs:
                p = swe.swe_params_default(scheme, precision, time_scheme=ts)
                st = swe.State.from_workload(mesh, p, w)
                steps = 0
                while st.time()[0] < 1.0:                      # count the CFL steps to t = 1
                    st.step(1, cfl)
                    steps += 1
                st.close()
                # warm-up on the state that is timed (it captures the 24-step CUDA graph the timed
                # run replays), then back to the initial condition; the time is taken from there
                st = swe.State.from_workload(mesh, p, w)
                st.step(24, cfl)
                st.set_state(w.h, w.hu, w.hv)
                t0 = st.time()[0]
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st.step(steps, cfl)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                t = st.time()[0] - t0
                h = st.get_state()[0]
                st.close()
                hex_, _ = stoker(cx, t, 5.0, 1.0, 0.5)
                l2 = float(np.sqrt(np.sum(area * (h - hex_) ** 2) / np.sum(area * hex_ ** 2)))
                rows.append({"cells": w.n_cells, "precision": precision, "scheme": scheme, "time_scheme": ts,
                             "cfl": cfl, "steps": steps, "t": t, "ms": ms, "l2_h": l2})
                print(f"{w.n_cells:8d} {precision} {scheme:10s} {ts:5s} cfl {cfl:.2f} steps {steps:5d} "
                      f"t {t:.4f} {ms:8.2f} ms  L2(h) {l2:.3e}", file=sys.stderr)
        mesh.close()
    print(json.dumps({"study": "GPU time against L2 error, wet-bed dam break (Sec. 6.3)",
                      "unit": {"ms": "GPU ms to t = 1 s", "l2_h": "relative L2 of h against Stoker"},
                      "rows": rows}))


def run_configs(args):
    """The CPU-baseline leg for every configuration of the workload list at its full size: GPU
    throughput (CFL steps in CUDA graphs, device events) in the precisions each one names, and the
    FP64 oracle timed on the host cores,
    all cores and one core, over the full step count (the 13M river: 20 steps; one core: at most 20
    steps), with the GPU result after the oracle's steps (its time steps replayed) against the
    oracle's, at checkpoints along the run.  One JSON line per configuration and scheme."""
    import torch

    import oracle
    from paper_2307_16758_gb300 import swe
    from paper_2307_16758_gb300 import workloads as W
    import __graft_entry__

    __graft_entry__.build()
    swe.load_library()
    oracle.build()
    stream = torch.cuda.current_stream()
    cores = os.cpu_count() or 1
    cfgs = [
        (1, "dam break, 100x10 squares (Sec. 6.3 setup)", lambda: W.dam_break_1d(100, 10, 100.0, 10.0, 1.0, 0.5),
         ["hllc"], ["fp64"], 200, 200),
        (2, "partial dam break over Gaussian bathymetry, 1000x500 jittered grid", lambda: W.partial_dam_break(),
         ["muscl", "waf"], ["fp64"], 1000, 1000),
        (3, "river 4160x1563 jittered grid", lambda: W.river(), ["muscl"], ["fp32", "fp64"], 2000, 20),
        (4, "river 2310x866 jittered grid", lambda: W.river(2310, 866), ["waf", "waf:depth", "waf:minbee", "muscl"],
         ["fp32"], 2000, 2000),
    ]
    for cid, name, make, schemes, precisions, steps, o_steps in cfgs:
        if args.config and cid not in args.config:
            continue
        w = make()
        mesh = swe.Mesh.from_workload(w, "morton")
        om = oracle.Mesh(w.nodes, w.tris, w.bnd_edges, w.bnd_tag, w.cut_edges)
        n = mesh.n
        for label in schemes:
            # "waf:depth": WAF with its ratios on the cell depth; "waf:minbee" / "waf:vanleer": another
            # limiter than SUPERBEE (the default WAF takes the free-surface ratio and SUPERBEE)
            scheme, opt = (label.split(":") + [""])[:2]
            kw = {"waf_ratio": "depth"} if opt == "depth" else ({"waf_limiter": opt} if opt else {})
            row = {"config": cid, "workload": name, "cells": n, "scheme": label, "steps": steps, "gpu": {}}
            for precision in precisions:
                p = swe.swe_params_default(scheme, precision, **kw)
                st = swe.State.from_workload(mesh, p, w)
                st.step(24, args.cfl)              # captures the 24-step graph that the timed run replays
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st.step(steps, args.cfl)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                row["gpu"][precision] = {"ms_per_step": ms / steps, "value": n * steps / (ms / 1e3), "unit": UNIT}
                st.close()
            # the oracle with the GPU's thresholds of the first precision named (same algorithm)
            p0 = swe.swe_params_default(scheme, precisions[0], **kw)
            o = oracle.opts(scheme, h_eps=p0.h_eps, r_eps=p0.r_eps, cfl=args.cfl, threads=cores, **kw)
            # the oracle in chunks; after each the GPU replays the chunk's time steps and the two
            # are compared (how far they drift apart with the number of steps)
            st = swe.State.from_workload(mesh, p0, w)
            oh, ohu, ohv = w.h, w.hu, w.hv
            el, done, growth = 0.0, 0, []
            for mark in [c for c in (25, 50, 100, 200, 500, 1000, 2000) if c < o_steps] + [o_steps]:
                t0 = time.perf_counter()
                oh, ohu, ohv, dts, _ = oracle.run(om, o, w.z, w.nman, oh, ohu, ohv, mark - done, q_in=w.q_in,
                                                  level=w.level)
                el += time.perf_counter() - t0
                done = mark
                st.step_dt(dts)
                gh, ghu, ghv = st.get_state()
                growth.append({"steps": done, "l1_h": rel_l1(gh, oh), "l1_hu": rel_l1(ghu, ohu),
                               "l1_hv": rel_l1(ghv, ohv)})
            st.close()
            s1 = min(o_steps, 20)
            o1 = oracle.opts(scheme, h_eps=p0.h_eps, r_eps=p0.r_eps, cfl=args.cfl, threads=1, **kw)
            t0 = time.perf_counter()
            oracle.run(om, o1, w.z, w.nman, w.h, w.hu, w.hv, s1, q_in=w.q_in, level=w.level)
            el1 = time.perf_counter() - t0
            row["oracle"] = {"steps": o_steps, "cores": cores, "value": n * o_steps / el, "unit": UNIT,
                             "one_core": {"steps": s1, "value": n * s1 / el1}}
            qs = max(np.abs(ohu).max(), np.abs(ohv).max(), 1e-300)
            cx = w.centroids()[0]
            # wetting front: the largest along-valley x of the cells that were dry at t = 0 and now
            # hold more than 1 mm (NaN while the flow has wetted none)
            front = lambda hh: float(cx[(hh > 1e-3) & (w.h <= 0.0)].max()) if ((hh > 1e-3) & (w.h <= 0.0)).any() \
                else float("nan")
            row["front_x"] = {"gpu": front(gh), "oracle": front(oh), "steps": o_steps}
            speed = lambda hh, qx, qy: float(np.where(hh > 1e-3, np.hypot(qx, qy) / np.maximum(hh, 1e-300), 0.0).max())
            row["max_speed"] = {"gpu": speed(gh, ghu, ghv), "oracle": speed(oh, ohu, ohv), "steps": o_steps,
                                "unit": "m/s", "over": "cells deeper than 1 mm"}
            row["error_vs_oracle"] = {"precision": precisions[0], "steps": o_steps, "l1_h": rel_l1(gh, oh),
                                      "linf_h": rel_inf(gh, oh), "l1_hu": rel_l1(ghu, ohu), "l1_hv": rel_l1(ghv, ohv),
                                      "linf_q": float(max(np.abs(ghu - ohu).max(), np.abs(ghv - ohv).max()) / qs),
                                      "growth": growth}
            print(json.dumps(row), flush=True)
        mesh.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cfl", type=float, default=0.9)
    ap.add_argument("--kernel", default="auto", choices=["auto", "split", "fused"])
    ap.add_argument("--moving", action="store_true",
                    help="start from an all-wet moving state of the same river (no exact shortcuts apply)")
    ap.add_argument("--block", type=int, default=0,
                    help="threads per block of the flux kernel (cells per tile for the tile step); 0: the default")
    ap.add_argument("--scheme", default="muscl", choices=list(SCHEME_NAMES),
                    help="MUSCL-HLLC with least-squares gradients (default), the paper's edge-upwind MUSCL, "
                         "first-order HLLC or WAF-HLLC")
    ap.add_argument("--hr-order", type=int, default=1, choices=[1, 2],
                    help="hydrostatic reconstruction: 1 (cell bed) or 2 (linear bed; LSQ MUSCL only)")
    ap.add_argument("--fp64-steps", type=int, default=2000)
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the 13M-cell mesh (testing only)")
    ap.add_argument("--quick", action="store_true", help="skip the FP64 comparison and the CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 4M-cell WAF/MUSCL study and the 40M-cell ensemble in the default line")
    ap.add_argument("--ensemble", action="store_true", help="the 64-scenario batched ensemble instead")
    ap.add_argument("--parts", type=int, default=1,
                    help="step with the boundary-first schedule over this many Morton sub-domains")
    ap.add_argument("--time-error", action="store_true",
                    help="GPU time against L2 error on the paper's dam break, 20k-600k cells, all schemes")
    ap.add_argument("--members", type=int, default=64)
    ap.add_argument("--configs", action="store_true",
                    help="every workload configuration at full size: GPU and FP64 oracle throughput, GPU vs oracle")
    ap.add_argument("--config", type=int, action="append", help="with --configs: only this configuration")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.ensemble:
        run_ensemble(args)
    elif args.time_error:
        run_time_error(args)
    elif args.configs:
        run_configs(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
