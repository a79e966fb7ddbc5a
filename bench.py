#!/usr/bin/env python
"""Throughput of the sLdG projection sweep on GB300: DoF updates/s and HBM GB/s.

Workload (default): the 4D (x1, x2, v1, v2) split advection with 64^4 cells,
degree k = 2 (81 tensor-product Legendre coefficients per cell), FP64 cell
means + FP32 higher coefficients, Strang splitting with dt = 0.1 (6 sweeps per
step), initial data a Maxwellian with random x-modes (seeded).  The state is
5.5 GB (mixed) / 10.9 GB (FP64), far above the 129 MB L2, so no L2 flush is
needed between steps.  The same steps are also timed on the all-FP64 store for
the mixed-vs-FP64 comparison.

One step = one Strang step (all sweeps, each with its on-device shift/matrix
construction).  value = DoF updates per second over K timed steps, timed with
CUDA events on the library's stream; the per-sweep-kernel times come from the
library's own event pairs around every sweep launch.

--impl reference times the CPU FP64 oracle (the deliberately plain reference)
on a bounded sub-grid of the same workload on the host cores.

Multi-GPU (torchrun): every rank runs its own replica of the workload (weak
scaling, no collective on the data path); the barrier-bracketed time is the
maximum over ranks and value counts every rank's DoF updates.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DoF updates/s and HBM GB/s per sweep: mixed vs FP64 on GB300, mass drift <=1e-13"
UNIT = "DoF/s"
L2_BYTES = 129 * 1024 * 1024


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="4d", choices=["4d", "2d", "batch", "6d", "1d", "vp", "paper1d"],
                    help="4d: 64^4 k=2 (default); 2d: 512^2 k=2; batch: 256 uneven 2D problems; "
                         "6d: 20^6 k=1; 1d: N=1024 k=2; paper1d: the 1D stores of Tables III-VI "
                         "(order 2 and 4, every # double) on N = 2^27 cells")
    ap.add_argument("--n", type=int, default=None, help="cells per dimension (4d/2d/6d)")
    ap.add_argument("--storage", default=None, help="store of the timed arm (default per workload)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison arm")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--shapes", default=None,
                    help="JSON list of per-dimension launch shapes (sl_set_tune fields) used "
                         "instead of the autotuner, or 'default' for the library's defaults "
                         "(e.g. to profile one fixed kernel)")
    ap.add_argument("--nprob", type=int, default=256, help="problems of the batched workload")
    ap.add_argument("--order", type=int, default=None, help="paper1d: only the rows of this order (2 or 4)")
    ap.add_argument("--arith", choices=["store", "fp64"], default="store",
                    help="arithmetic of the timed arm's FP32 rows (sl_set_arithmetic): the store's own "
                         "(FP32) or FP64 with FP32 storage")
    ap.add_argument("--nodal-v", action="store_true",
                    help="4d/2d: x-sweeps with the velocity at the Gauss nodes of every v-cell")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# distributed bookkeeping (host logic; covered by CPU gloo tests)
# ---------------------------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(elapsed_ms: float, units: float, world: int, device=None):
    """Max of the elapsed time and sum of the work units over all ranks."""
    if world <= 1:
        return elapsed_ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return summarise_clocks(lines)


def summarise_clocks(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen in
    nvidia-smi samples of ClockSampler.FIELDS (csv, no header, no units)."""
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
        except ValueError:
            continue
    if not rows:
        return None
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
    sm = [r[0] for r in rows]
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows),
            "reasons": reasons, "samples": len(rows)}


# DRAM traffic of the sweep launches (dram__bytes_read.sum + dram__bytes_write.sum),
# taken from ncu captures of smaller cases of the same kernels and stored as a
# ratio to the launch's algorithmic bytes (2 x state bytes), so that it scales
# with the units a launch processes.  Each ratio is the launch-weighted mean over
# one Strang step's sweeps, the captured unit-stride kernel standing for the
# dimension-0 sweeps and the captured strided kernel for the others.  A ratio
# holds only for the kernel sources it was taken on: if their hash differs, the
# traffic is reported as null.
TRAFFIC = {
    ("4d", "mix_fp32"): {
        "ratio": (0.98529 + 1.00005 + 1.00636 + 0.99558 + 0.98462 + 1.00005) / 6,
        "sources": ["sl_internal.cuh", "sl_sweep.cuh", "sl_sweep_fp.inc", "sl_sweep_f32.cu"],
        "sha256": "455d482ff0cd9efd",
        "capture": "48^4 cells, k=2, one Strang step (6 launches: vector form along dimension 0, walks with 1 fibre, "
                   "4 cells per step along the others): 3.431-3.504 GB per launch against 3.482 GB algorithmic"},
    ("6d", "mix_bf16"): {
        "ratio": (1.00631 + 1.03328 + 1.03146 + 1.03033 + 1.03041 + 1.03252 + 1.00555 + 1.03325 + 1.03157) / 9,
        "sources": ["sl_internal.cuh", "sl_sweep.cuh", "sl_sweep_rec.cu"],
        "sha256": "ef12c01954e28a04",
        "capture": "16^6 cells, k=1, BF16 records, lane groups, one Strang step (9 launches): 4.656-4.785 GB per "
                   "launch against 4.631 GB algorithmic"},
    ("6d", "mix_fp16"): {
        "ratio": (1.00630 + 1.03332 + 1.03149 + 1.03040 + 1.03058 + 1.03263 + 1.00563 + 1.03329 + 1.03147) / 9,
        "sources": ["sl_internal.cuh", "sl_sweep.cuh", "sl_sweep_rec.cu"],
        "sha256": "ef12c01954e28a04",
        "capture": "16^6 cells, k=1, FP16 records, lane groups, one Strang step (9 launches): 4.656-4.785 GB per "
                   "launch against 4.631 GB algorithmic"},
    ("2d", "mix_fp32"): {
        "ratio": (0.96416 + 0.97316 + 0.96173) / 3,
        "sources": ["sl_internal.cuh", "sl_sweep.cuh", "sl_sweep_fp.inc", "sl_sweep_f32.cu"],
        "sha256": "455d482ff0cd9efd",
        "capture": "4096^2 cells, k=2 (the size of the workload), library default shapes, one Strang step: "
                   "1.291-1.306 GB per launch against 1.342 GB algorithmic"},
    ("vp", "mix_fp32"): {
        "ratio": (0.96424 + 0.97247 + 0.96162) / 3,
        "sources": ["sl_internal.cuh", "sl_sweep.cuh", "sl_sweep_fp.inc", "sl_sweep_f32.cu"],
        "sha256": "455d482ff0cd9efd",
        "capture": "4096^2 cells, k=2 (the size of the workload), self-consistent field, library default shapes, one "
                   "Strang step (sweeps only): 1.291-1.305 GB per launch against 1.342 GB algorithmic"},
    ("4d_nodal_v", "mix_fp32"): {
        "ratio": (0.94464 + 0.93238 + 0.95927 + 0.94212 + 0.94070 + 0.93180) / 6,
        "sources": ["sl_internal.cuh", "sl_sweep.cuh", "sl_sweep_fp.inc", "sl_sweep_f32.cu", "sl_nodal.h", "sl_nodal.cu"],
        "sha256": "2515eb9747e6448e",
        "capture": "32^4 cells, k=2, nodal x-sweeps (runs of 2 along dimension 0, of 4 along dimension 1), one "
                   "Strang step: 0.641-0.660 GB per launch against 0.688 GB algorithmic"},
    ("2d_nodal_v", "mix_fp32"): {
        "ratio": (0.96784 + 0.97304 + 0.96557) / 3,
        "sources": ["sl_internal.cuh", "sl_sweep.cuh", "sl_sweep_fp.inc", "sl_sweep_f32.cu", "sl_nodal.h", "sl_nodal.cu"],
        "sha256": "2515eb9747e6448e",
        "capture": "4096^2 cells, k=2 (the size of the workload), nodal x-sweep, one Strang step: 1.296-1.306 GB per "
                   "launch against 1.342 GB algorithmic"},
    ("paper1d", "mix_fp32"): {
        "ratio": 0.96349,
        "sources": ["sl_internal.cuh", "sl_sweep.cuh", "sl_sweep_fp.inc", "sl_sweep_f32.cu"],
        "sha256": "455d482ff0cd9efd",
        "capture": "2^25 cells, order 4, c_0 in FP64: 1.293 GB per launch against 1.342 GB algorithmic"},
    ("batch", "mix_fp32"): {
        "ratio": (0.96774 + 1.04429 + 0.96494) / 3,
        "sources": ["sl_internal.cuh", "sl_sweep.cuh", "sl_batch.cu", "sl_batch_api.cu"],
        "sha256": "5771a059f0504081",
        "capture": "64 problems, shapes (3 fibres, runs of 2) / (1 fibre, 4 rows per step, 32-line by 32-row items), "
                   "one Strang step: 1.054-1.140 GB per launch against 1.092 GB algorithmic"},
}


def launches_per_step(args, info):
    """Kernels one bench step launches.  A split step builds each dimension's
    shift table once (Strang's two x half-steps share theirs) besides its
    sweeps; a nodal x-sweep builds its node table before it (and, in the mixed
    store, the per-v-cell record); the self-consistent field builds its v-table
    right before the v-sweep, after two launches (density sums, field); the 1D
    advection graph is one thread-block cluster launch in
    the FP64 store (every step's table built in the kernel), (table build,
    sweep) pairs otherwise."""
    sweeps = info["sweeps"]
    if args.workload == "1d":
        return 1 if args.storage == "fp64" else 2 * sweeps
    if args.workload == "vp":
        return sweeps + info["ndim"] + 2
    nodal = info.get("nodal_x_sweeps", 0)
    if nodal:
        x_dims = info["ndim"] // 2
        per_nodal = 2 if args.storage == "fp64" else 3
        return nodal * per_nodal + (sweeps - nodal) + (info["ndim"] - x_dims)
    return sweeps + info["ndim"]


def sweep_traffic(workload, storage, bytes_per_launch):
    """DRAM bytes per sweep launch at this size, or (None, why)."""
    import hashlib
    t = TRAFFIC.get((workload, storage))
    if t is None:
        return None, "no ncu capture of this workload's kernels"
    m = hashlib.sha256()
    for f in t["sources"]:
        with open(os.path.join(ROOT, "paper_1603_07008_gb300", "csrc", f), "rb") as fh:
            m.update(fh.read())
    if m.hexdigest()[:16] != t["sha256"]:
        return None, "kernel sources changed since the ncu capture"
    return t["ratio"] * bytes_per_launch, ("scaled by units from an ncu capture of " +
                                           t["capture"])


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline / reference arm)
# ---------------------------------------------------------------------------

def oracle_sample_problem(n_x: int, n_v: int):
    """The 4D workload on an n_x^2 x n_v^2 sub-grid (same box, k, dt, data)."""
    from paper_1603_07008_gb300 import workloads as W
    p = W.config3(n=n_x, steps=1)
    p.grid = W.Grid(n=(n_x, n_x, n_v, n_v), lo=p.grid.lo, hi=p.grid.hi, pair=p.grid.pair)
    return p


def time_oracle(n_x: int, n_v: int, steps: int):
    import oracle as O
    p = oracle_sample_problem(n_x, n_v)
    u = O.project(p.grid, p.k, p.nq, p.weights, p.params)
    sched = O.schedule(p.grid, "strang", p.dt, p.field_list())
    t0 = time.perf_counter()
    for _ in range(steps):
        for dim, sd, s in sched:
            u = O.sweep(u, p.grid.n, p.k, dim, sd, s)
    dt = time.perf_counter() - t0
    dof_updates = steps * len(sched) * u.size
    return dof_updates / dt, dt, dof_updates, p


# Bounds of each store against the FP64 oracle: FP64 max relative, the
# mixed and split FP32 stores relative L2, the scaled 16-bit stores relative L2.
ERROR_BOUND = {"fp64": ("rel_max", 1e-12), "mix_fp32": ("rel_l2", 1e-5), "fp32": ("rel_l2", 1e-5),
               "mix_fp32_d2": ("rel_l2", 1e-5), "mix_fp32_d3": ("rel_l2", 1e-5),
               "mix_bf16": ("rel_l2", 1e-2), "mix_fp16": ("rel_l2", 1e-2)}


def oracle_error(samples, storage):
    """Error of sampled cells of the timed path (Arm.samples) against the
    FP64 oracle evaluated on their dependency cones (oracle.sample_after)
    from the same initial projection.  Runs after the timed region, on the
    host; the GPU values were downloaded before."""
    if not samples:
        return {"note": "no sampled oracle check for this line"}
    import oracle as O
    if "whole" in samples:   # the self-consistent field: the whole state after one step
        q, got = samples["whole"]
        t0 = time.perf_counter()
        ref = O.vp_step(O.project(q.grid, q.k, q.nq, q.weights, q.params), q.grid, q.k, "strang", q.dt, 1)
        kind, bound = ERROR_BOUND[storage]
        rel_l2, rel_max = O.rel_l2(got, ref, q.k, q.grid.ndim), O.rel_max(got, ref)
        val = rel_l2 if kind == "rel_l2" else rel_max
        return {"rel_l2": rel_l2, "rel_max": rel_max, "cells": int(got.shape[0]), "problems": 1, "steps": 1,
                "bound": {kind: bound}, "within_bound": bool(val <= bound),
                "oracle_s": time.perf_counter() - t0,
                "how": "the whole state after one self-consistent Strang step from the initial projection on "
                       "the timed context, against the FP64 oracle's step (the field depends on every cell)"}
    t0 = time.perf_counter()
    l2_num = l2_den = 0.0
    max_num = max_den = 0.0
    ncells = 0
    for item in samples["items"]:
        q, cells, got, nsweeps = item[:4]
        if len(item) > 4:            # an explicit sweep list (the 1D stores of Tables III-VI)
            sched = item[4]
        elif samples.get("nodal"):   # x-sweeps with the velocity at the Gauss nodes of each v-cell
            sched = O.schedule_nodal(q.grid, "strang", q.dt, q.field_list())
        elif q.splitting == "advect":   # the 1D workload: one constant shift per sweep
            h = (q.grid.hi[0] - q.grid.lo[0]) / q.grid.n[0]
            sched = [(0, -1, np.array([q.velocity * q.dt / h]))]
        else:
            sched = O.schedule(q.grid, "strang", q.dt, q.field_list())
        reps = nsweeps // len(sched)
        ref = O.sample_after(q.grid, q.k, q.nq, q.weights, q.params, sched * reps, cells)
        w = O.l2_weights(q.k, q.grid.ndim)
        d = np.asarray(got, dtype=np.float64) - ref
        l2_num += float(np.sum(d * d * w))
        l2_den += float(np.sum(ref * ref * w))
        max_num = max(max_num, float(np.max(np.abs(d))))
        max_den = max(max_den, float(np.max(np.abs(ref))))
        ncells += len(cells)
    rel_l2 = math.sqrt(l2_num / l2_den) if l2_den > 0 else math.sqrt(l2_num)
    rel_max = max_num / max_den if max_den > 0 else max_num
    kind, bound = ERROR_BOUND[storage]
    val = rel_l2 if kind == "rel_l2" else rel_max
    return {"rel_l2": rel_l2, "rel_max": rel_max, "cells": ncells, "problems": len(samples["items"]),
            "steps": samples["steps"], "bound": {kind: bound}, "within_bound": bool(val <= bound),
            "oracle_s": time.perf_counter() - t0,
            "how": "sampled cells (first, last, random) after these steps from the initial projection on the "
                   "timed context and launch path, against the FP64 oracle on their dependency cones"}


def _oracle_worker(sample):
    rate, secs, ndof, _ = time_oracle(*sample)
    return rate, secs, ndof


def time_oracle_all_cores(n_x: int, n_v: int, steps: int):
    """The same oracle sample in one process per host core at once (spawned,
    since the parent has used the GPU): (summed DoF updates/s, processes)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(n_x, n_v, steps)] * cores)
    return sum(r[0] for r in res), cores


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    # one step = one oracle Strang step on a 32 x 32 x 16 x 16 sub-grid
    for _ in range(args.warmup):
        time_oracle(32, 16, 1)
    rate, secs, dof, p = time_oracle(32, 16, args.steps)
    out = {
        "metric": METRIC, "value": rate, "unit": UNIT, "impl": "reference",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * secs / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "4d_xxvv_64^4_k2_mix_fp32_strang",
                   "sample": "each step one Strang step of the oracle (FP64) on a 32x32x16x16 sub-grid of "
                             "that workload, reported per DoF update",
                   "l2": "host run", "parallelism": "rank 0 only"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} Strang steps (6 sweeps) of the 4D k=2 workload "
                                   f"on a 32x32x16x16 sub-grid, FP64 oracle, single thread"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def apply_shapes(ctx, shapes):
    if shapes is None:
        ctx.autotune(3)
        return
    if shapes == "default":   # the library's default shapes, no autotuning
        return
    for d, sh in enumerate(json.loads(shapes)):
        ctx.set_tune(d, **sh)


DEFAULT_STORE = {"4d": "mix_fp32", "2d": "mix_fp32", "batch": "mix_fp32", "6d": "mix_bf16",
                 "1d": "fp64", "vp": "mix_fp32"}
DEFAULT_N = {"4d": 64, "2d": 512, "6d": 20, "1d": 1024, "vp": 4096}


# sweeps per CUDA graph of the 1D workload: its 100 time steps
ADVECT_GRAPH_SWEEPS = 100


def make_problem(W, workload, n, storage, nprob=256):
    if workload == "4d":
        return W.config3(n=n, steps=1, storage=storage)
    if workload in ("2d", "vp"):
        return W.config2(n=n, steps=1, storage=storage)
    if workload == "6d":
        return W.config5(n=n, steps=1, storage=storage)
    if workload == "1d":
        return W.config1()
    return W.config4(nprob=nprob, storage=storage)


class Arm:
    """One store of one workload behind the library's public API: a context,
    or a batch for the batched workload."""

    def __init__(self, S, W, args, storage, stream, shapes=None):
        self.workload = args.workload
        self.p = make_problem(W, args.workload, args.n, storage, args.nprob)
        if self.workload == "batch":
            probs = self.p
            self.obj = S.Batch([q.grid for q in probs], [q.k for q in probs], storage, stream=stream)
            for i, q in enumerate(probs):
                self.obj.project(i, q.nq, q.weights, q.params)
            self.obj.set_fields([q.field_list()[0] for q in probs])
            if shapes is None:
                self.obj.autotune(3)
            elif shapes != "default":   # sl_batch_set_tune fields per dimension
                for d, sh in enumerate(json.loads(shapes)):
                    self.obj.set_tune(d, **sh)
            self.dof = self.obj.info["dof"]
            self.state_bytes = self.obj.info["state_bytes"]
            self.sweeps = 3
            self.dt = probs[0].dt
            self.order = None
            # the time loop replayed from a CUDA graph (one Strang step: 3 sweeps
            # with their table launches; the batch keeps one graph per parity)
            self.graph = True
            self.obj.graph_capture("strang", self.dt, 1)
        else:
            p = self.p
            self.obj = S.Context(p.grid, p.k, storage, stream=stream)
            self.obj.project(p.nq, p.weights, p.params)
            if storage != "fp64":
                self.obj.set_arithmetic(getattr(args, "arith", "store"))
            if self.workload == "vp":      # field from the state before every v-sweep
                self.obj.set_poisson(True)
            elif p.splitting != "advect":
                self.obj.set_fields(p.field_list())
            self.nodal = getattr(args, "nodal_v", False)
            if self.nodal:
                self.obj.set_nodal_velocity(True)
            apply_shapes(self.obj, shapes)
            self.dof = p.dof
            self.order = p.k + 1
            self.state_bytes = self.obj.info["state_bytes"]
            # the 1D workload: one bench step is the whole 100-step run (one graph:
            # in the FP64 store a single cluster launch that builds every step's
            # table and runs its sweep)
            self.sweeps = ADVECT_GRAPH_SWEEPS if p.splitting == "advect" else \
                2 * len(p.grid.x_dims()) + len(p.grid.v_dims())
            self.dt = p.dt
            # a state that fits in L2 makes every sweep a few microseconds: replay
            # the split step from a CUDA graph instead of launching its kernels
            self.graph = p.splitting != "advect" and 2 * self.state_bytes < L2_BYTES
            if self.graph:
                self.obj.graph_capture("strang", self.dt, 1)
            if p.splitting == "advect":
                h = (p.grid.hi[0] - p.grid.lo[0]) / p.grid.n[0]
                self.shift = p.velocity * p.dt / h
                self.obj.graph_capture_advect(0, -1, [self.shift], ADVECT_GRAPH_SWEEPS)

    def step(self, n, eager=False):
        if not eager and (self.workload == "1d" or getattr(self, "graph", False)):
            for _ in range(n):
                self.obj.graph_launch()
        else:
            self.obj.step("strang", self.dt, n)

    def restart(self):
        """Back to the initial projection (the state the timed steps started from)."""
        if self.workload == "batch":
            for i, q in enumerate(self.p):
                self.obj.project(i, q.nq, q.weights, q.params)
        else:
            self.obj.project(self.p.nq, self.p.weights, self.p.params)

    def samples(self, seed=7):
        """Coefficients of sampled cells after a few timed-path steps from the
        initial projection, for the error against the FP64 oracle (computed
        by the oracle leg after the timed region).  The steps run on the same
        context and launch path as the timed ones: 2 split steps in up to four
        dimensions, 1 in six (each target cell depends on two source cells per
        sweep, so the oracle evaluates a cone of at most 2^sweeps cells per
        sample), the 1D workload's 100-sweep graph once."""
        rng = np.random.default_rng(seed)
        self.restart()
        if self.workload == "vp":   # the field reads every cell: the whole state after one step
            self.step(1)
            return {"steps": 1, "whole": (self.p, self.obj.get_coeffs())}
        if self.workload == "batch":
            steps = 2
            self.step(steps)
            picks = sorted({0, len(self.p) // 3, 2 * len(self.p) // 3, len(self.p) - 1})
            out = []
            for i in picks:
                q = self.p[i]
                cells = np.concatenate([[0, q.grid.cells - 1], rng.integers(0, q.grid.cells, 6)])
                out.append((q, cells, self.obj.get_coeffs(i)[cells], steps * 3))
            return {"steps": steps, "items": out}
        q = self.p
        steps = 1 if q.grid.ndim > 4 or self.workload == "1d" else 2
        self.step(steps)
        cells = np.concatenate([[0, q.grid.cells - 1], rng.integers(0, q.grid.cells, 14)])
        nsw = steps * self.sweeps
        return {"steps": steps, "items": [(q, cells, self.obj.get_cells(cells), nsw)],
                "nodal": bool(getattr(self, "nodal", False))}

    def mass_total(self):
        m = self.obj.mass()
        return float(np.sum(m)) if self.workload == "batch" else m

    def tunes(self):
        nd = self.p[0].grid.ndim if self.workload == "batch" else self.p.grid.ndim
        return [self.obj.get_tune(d) for d in range(nd)]


def run_ours(args):
    import torch
    import paper_1603_07008_gb300 as S
    from paper_1603_07008_gb300 import workloads as W

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    args.storage = args.storage or DEFAULT_STORE[args.workload]
    args.n = args.n or DEFAULT_N.get(args.workload)
    peaks, peak_src = measured_peaks()

    def timed(storage, shapes):
        arm = Arm(S, W, args, storage, stream, shapes)
        m0 = arm.mass_total()
        for _ in range(args.warmup):
            arm.step(1)
        arm.obj.synchronize()
        arm.obj.profile_query()
        arm.obj.profile_enable(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier(world)
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        torch.cuda.synchronize()
        e0.record(stream)
        arm.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        prof = arm.obj.profile_query()
        dims = arm.obj.profile_dims() if hasattr(arm.obj, "profile_dims") else None
        arm.obj.profile_enable(False)
        m1 = arm.mass_total()
        info = {"state_bytes": arm.state_bytes, "dof": arm.dof, "sweeps": arm.sweeps,
                "nodal_x_sweeps": 2 * len(arm.p.grid.x_dims()) if getattr(arm, "nodal", False) else 0,
                "ndim": 2 if arm.workload == "batch" else len(arm.p.grid.n),
                "tune": arm.tunes(), "order": arm.order,
                "graph": arm.workload == "1d" or getattr(arm, "graph", False)}
        if arm.workload == "batch":
            # the graph has no per-sweep events: one eager, profiled step after
            # the timed region gives the per-dimension kernel times
            arm.obj.profile_enable(True)
            arm.step(1, eager=True)
            arm.obj.synchronize()
            arm.obj.profile_query()
            dims = arm.obj.profile_dims()
            arm.obj.profile_enable(False)
            info["per_dim_from"] = "one eager step after the timed region"
        if dims:
            nd, msd = dims
            info["per_dim"] = [{"dim": d, "launches": nd[d], "ms_per_launch": msd[d] / max(nd[d], 1),
                                "gbs": 2.0 * arm.state_bytes / (msd[d] / max(nd[d], 1) / 1e3) / 1e9
                                if nd[d] else None} for d in range(len(nd)) if nd[d]]
        info["samples"] = arm.samples() if rank == 0 else None
        arm.obj.close()
        return ms, prof, abs(m1 - m0) / abs(m0), clk, info

    ms, prof, drift, clk, info = timed(args.storage, args.shapes)
    units_local = float(args.steps * info["sweeps"] * info["dof"])
    ms_max, units = aggregate(ms, units_local, world, dev)
    value = units / (ms_max / 1000.0)
    nl, sweep_ms, sweep_bytes = prof
    if nl == 0:   # graph replay: no per-sweep events, the step time (graph launch included) per sweep
        nl = args.steps * info["sweeps"]
        sweep_ms = ms
        sweep_bytes = 2.0 * info["state_bytes"] * nl
    avg_sweep_ms = sweep_ms / max(nl, 1)
    bytes_per_sweep = sweep_bytes / max(nl, 1)
    achieved_gbs = bytes_per_sweep / (avg_sweep_ms / 1000.0) / 1e9
    peak_gbs = float(peaks["hbm_gbs"])
    # the captured ratios are of the plain sweeps; the nodal x-sweeps have none
    traffic, traffic_note = sweep_traffic(args.workload + ("_nodal_v" if args.nodal_v else "") +
                                          ("_arith_fp64" if args.arith == "fp64" else ""), args.storage,
                                          bytes_per_sweep)

    fp64 = None
    if not args.no_fp64 and args.storage != "fp64":
        ms64, prof64, drift64, clk64, info64 = timed("fp64", None)
        ms64_max, units64 = aggregate(ms64, units_local, world, dev)
        v64 = units64 / (ms64_max / 1000.0)
        nl64, sms64, sb64 = prof64
        if nl64 == 0:   # graph replay: the step time per sweep, as for the timed arm
            nl64 = args.steps * info64["sweeps"]
            sms64 = ms64
            sb64 = 2.0 * info64["state_bytes"] * nl64
        # The FP64 store's sweep is bound by the FP64 pipe, not by HBM: 2o FMAs
        # (4o flops) per DoF update against 2 FP64 FMAs per clock per SM
        # (1.25 TFLOP/s nominal at 152 SMs and 2.07 GHz).
        alu = None
        if info64["order"]:          # one degree for the whole state (not the mixed batch)
            flops64 = 4.0 * info64["order"] * info64["dof"]
            mhz = (clk64 or {}).get("sm_mhz") or 2070.0
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            alu_ach = flops64 / (sms64 / max(nl64, 1) / 1000.0) / 1e12
            alu_peak = S.sl_selftest_fp64_rate(1 << 14, stream) / 1e12
            alu = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s",
                   "frac": alu_ach / alu_peak,
                   "peak_source": "measured in this run: sl_selftest_fp64_rate (8 independent chains of FP64 "
                                  "FMAs with register operands per thread, 1024 or 2048 threads per SM, CUDA events)",
                   "derived_peak": 2.0 * 2.0 * sms * mhz * 1e6 / 1e12,
                   "derived_peak_note": f"2 FP64 FMA/clk/SM x {sms} SMs x {mhz:.0f} MHz (sampled clock)",
                   "flops_per_launch": flops64}
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": ms64_max / args.steps,
                "sweep_ms": sms64 / max(nl64, 1),
                "sweep_gbs": (sb64 / max(nl64, 1)) / (sms64 / max(nl64, 1) / 1000.0) / 1e9,
                "mass_drift": drift64, "state_bytes": info64["state_bytes"], "clocks": clk64,
                "per_dim": info64.get("per_dim"),
                "roofline": alu,
                "error": oracle_error(info64.get("samples"), "fp64") if rank == 0 else None}

    e2e = None
    if not args.no_e2e and args.workload == "4d":
        p = make_problem(W, "4d", args.n, args.storage)
        e2e = run_e2e(S, W, p, args, stream, world, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and args.workload == "4d":
        rate, secs, ndof, _ = time_oracle(64, 16, 5)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"5 Strang steps (6 sweeps each, {ndof:.3g} DoF updates, {secs:.1f} s) of "
                         "the 4D k=2 workload on a 64x64x16x16 sub-grid, FP64 oracle, one thread"}
        rate_all, ncores = time_oracle_all_cores(64, 16, 5)
        cpu["all_cores"] = {"value": rate_all, "unit": UNIT, "cores": ncores,
                            "sample": "the same sample in one oracle process per host core at once, "
                                      "DoF updates/s summed over the processes"}

    if rank == 0:
        nod = "_nodal_v" if args.nodal_v else ""
        wl = {"4d": f"4d_xxvv_{args.n}^4_k2_{args.storage}_strang{nod}",
              "2d": f"2d_xv_{args.n}^2_k2_{args.storage}_strang{nod}",
              "vp": f"2d_xv_{args.n}^2_k2_{args.storage}_strang_self_consistent_field",
              "6d": f"6d_xxxvvv_{args.n}^6_k1_{args.storage}_strang",
              "1d": f"1d_n{args.n}_k2_{args.storage}_advect_100_steps_per_graph",
              "batch": f"batch256_2d_xv_k1k2_{args.storage}_strang"}[args.workload]
        l2note = (f"state {info['state_bytes'] / 1e9:.2f} GB > L2; no flush needed"
                  if info["state_bytes"] > 4 * L2_BYTES else
                  f"state {info['state_bytes'] / 1e6:.1f} MB fits in L2: GB/s is not an HBM figure")
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"mix_fp32": "f32+f64", "fp64": "f64", "mix_bf16": "bf16+f64",
                      "mix_fp16": "f16+f64"}[args.storage],
            "data": "synthetic",
            "config": {"workload": wl, "dof": info["dof"], "sweeps_per_step": info["sweeps"],
                       "state_bytes": info["state_bytes"], "l2": l2note,
                       "parallelism": f"replicas x{world}", "tune": info["tune"],
                       "cuda_graph": info["graph"], "per_dim_from": info.get("per_dim_from"),
                       "arithmetic": args.arith},
            "mass_drift": drift,
            "error": oracle_error(info.get("samples"), args.storage),
            "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": peak_gbs, "unit": "GB/s",
                         "frac": achieved_gbs / peak_gbs, "traffic": traffic,
                         "traffic_note": traffic_note,
                         "kernel": "sweep (all dims)", "peak_source": peak_src,
                         "bytes_per_launch": bytes_per_sweep, "avg_launch_ms": avg_sweep_ms,
                         "launches": nl, "per_dim": info.get("per_dim")},
            "fp64": fp64,
            "speedup_mixed_vs_fp64": (value / fp64["value"]) if fp64 else None,
            "e2e": e2e,
            "gpu_launches": args.steps * launches_per_step(args, info),
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# The stores of Tables III-VI (Sec. III): (degree, store), "# double" per store.
PAPER1D_ROWS = [(1, "fp64"), (1, "mix_fp32"), (1, "fp32"),
                (3, "fp64"), (3, "mix_fp32_d3"), (3, "mix_fp32_d2"), (3, "mix_fp32"), (3, "fp32")]
PAPER1D_NDOUBLE = {"fp32": 0, "mix_fp32": 1, "mix_fp32_d2": 2, "mix_fp32_d3": 3}


def run_paper1d(args):
    """The GB300 counterpart of Tables III-VI: the 1D advection (constant
    velocity, CFL 0.37: sigma = 0, alpha = 0.37) of orders 2 and 4 with every
    store, on N = 2^27 cells (2.1 to 4.3 GB per state copy, far above L2).
    Per store: sweep GB/s (algorithmic bytes: read + write of the state),
    DoF updates/s, speedup over the FP64 store and memory reduction, as the
    paper's columns; the headline value is order 4 with c_0 in FP64."""
    import torch
    import paper_1603_07008_gb300 as S
    from paper_1603_07008_gb300 import workloads as W

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    n = args.n or (1 << 27)
    peaks, peak_src = measured_peaks()
    peak_gbs = float(peaks["hbm_gbs"])
    g = W.Grid(n=(n,), lo=(0.0,), hi=(1.0,), pair=(-1,))
    shift = 0.37
    rows, fp64_rate = [], {}
    clk_all = None
    # --storage: that store's rows only (e.g. to profile one kernel)
    todo = [r for r in PAPER1D_ROWS if args.storage in (None, r[1]) and args.order in (None, r[0] + 1)]
    if not todo:
        raise SystemExit(f"no paper1d row with store {args.storage!r}")
    head = head_launch = None
    for k, store in todo:
        ctx = S.Context(g, k, store, stream=stream)
        if store != "fp64":
            ctx.set_arithmetic(args.arith)
        # 1 + cos(2 pi 8 x + 0.3): the oscillatory profile of Table II
        prof_w, prof_p = [1.0, 1.0], [[[0.0, 0.0, 0.0, 0.0]], [[0.0, 0.0, 2 * math.pi * 8, 0.3]]]
        ctx.project(k + 2, prof_w, prof_p)
        apply_shapes(ctx, args.shapes)
        m0 = ctx.mass()
        for _ in range(args.warmup):
            ctx.advect(0, -1, [shift])
        ctx.synchronize()
        ctx.profile_query()
        ctx.profile_enable(True)
        barrier(world)
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            ctx.advect(0, -1, [shift])
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        nl, sms, sbytes = ctx.profile_query()
        ctx.profile_enable(False)
        drift = abs(ctx.mass() - m0) / abs(m0)
        info = ctx.info
        tune = ctx.get_tune(0)
        # sampled cells after 4 sweeps from the initial projection, for the
        # oracle leg below
        ctx.project(k + 2, prof_w, prof_p)
        for _ in range(4):
            ctx.advect(0, -1, [shift])
        rng = np.random.default_rng(7)
        cells = np.concatenate([[0, n - 1], rng.integers(0, n, 14)])
        q = W.Problem(name=f"1d_{store}", grid=g, k=k, storage=store, dt=0.0, steps=4, splitting="advect",
                      weights=np.asarray(prof_w), params=np.asarray(prof_p), nq=k + 2)
        sample = {"steps": 4, "items": [(q, cells, ctx.get_cells(cells), 4, [(0, -1, np.array([shift]))])]}
        ctx.close()
        ms_max, units = aggregate(ms, float(args.steps * info["dof"]), world, dev)
        sweep_ms = sms / max(nl, 1)
        gbs = (sbytes / max(nl, 1)) / (sweep_ms / 1000.0) / 1e9
        rate = units / (ms_max / 1000.0)
        if store == "fp64":
            fp64_rate[k] = (rate, info["state_bytes"])
        r64, b64 = fp64_rate.get(k, (None, None))
        rows.append({"order": k + 1, "store": store,
                     "n_double": k + 1 if store == "fp64" else PAPER1D_NDOUBLE[store],
                     "sweep_gbs": gbs, "frac_of_hbm": gbs / peak_gbs, "sweep_ms": sweep_ms,
                     "dof_per_s": rate, "speedup_vs_fp64": rate / r64 if r64 else None,
                     "memorydown": b64 / info["state_bytes"] if b64 else None, "mass_drift": drift,
                     "state_bytes": info["state_bytes"], "tune": tune, "clocks": clk,
                     "error": oracle_error(sample, store) if rank == 0 else None})
        if head is None or (k == 3 and store == "mix_fp32"):
            head = rows[-1]
            head_launch = (nl, sms, sbytes)
            clk_all = clk
    if rank == 0:
        nl, sms, sbytes = head_launch
        avg = sms / max(nl, 1)
        head_traffic = sweep_traffic("paper1d" + ("_arith_fp64" if args.arith == "fp64" else ""), head["store"],
                                     sbytes / max(nl, 1)) if head["order"] == 4 else \
            (None, "no ncu capture of this row's kernel")
        out = {
            "metric": METRIC, "value": head["dof_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["sweep_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32"}.get(head["store"], "f32+f64"),
            "data": "synthetic",
            "config": {"workload": f"1d_n{n}_k{head['order'] - 1}_{head['store']}_advect_cfl0.37"
                                   + (" (with every store of orders 2, 4)" if len(todo) > 1 else ""),
                       "dof": n * head["order"], "sweeps_per_step": 1, "state_bytes": head["state_bytes"],
                       "arithmetic": args.arith,
                       "l2": f"state {head['state_bytes'] / 1e9:.2f} GB > L2; no flush needed",
                       "parallelism": f"replicas x{world}"},
            "mass_drift": head["mass_drift"],
            "error": head["error"],
            "roofline": {"bound": "hbm", "achieved": head["sweep_gbs"], "peak": peak_gbs, "unit": "GB/s",
                         "frac": head["sweep_gbs"] / peak_gbs, "traffic": head_traffic[0],
                         "traffic_note": head_traffic[1],
                         "kernel": "sweep along dimension 0", "peak_source": peak_src,
                         "bytes_per_launch": sbytes / max(nl, 1), "avg_launch_ms": avg, "launches": nl},
            "table": rows,
            "speedup_mixed_vs_fp64": head["speedup_vs_fp64"],
            "e2e": None,
            "gpu_launches": args.steps * 2 * len(todo),
            "clocks": clk_all,
            "cpu_baseline": None,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_e2e(S, W, p, args, stream, world, dev):
    """Through the public API with host buffers, as for a stream of states that
    live on the host: every step uploads one state from pinned host memory
    (sl_set_planes), advances it one Strang step (sl_step) and reads its mass
    back (sl_mass, 8 bytes).  Two contexts on two CUDA streams take the steps in
    turn, so that one step's upload overlaps the previous step's sweeps; each
    step's result is read before the step after next is issued."""
    import numpy as np
    import torch
    streams = [stream, torch.cuda.Stream(device=dev)]
    ctxs = []
    for i, st in enumerate(streams):
        ctx = S.Context(p.grid, p.k, args.storage, stream=st)
        ctx.project(p.nq, p.weights, p.params)
        ctx.set_fields(p.field_list())
        if args.storage != "fp64":
            ctx.set_arithmetic(args.arith)
        if args.nodal_v:
            ctx.set_nodal_velocity(True)
        if i == 0:
            apply_shapes(ctx, args.shapes)
        else:   # the first context's shapes
            for d in range(p.grid.ndim):
                t = ctxs[0].get_tune(d)
                ctx.set_tune(d, **t)
        ctxs.append(ctx)
    mean, hi, scale = S.plane_arrays(ctxs[0].handle)
    # pinned host copies of the planes
    t_mean = torch.empty(mean.size, dtype=torch.float64, pin_memory=True)
    t_hi = torch.empty(hi.size * hi.itemsize // 4, dtype=torch.int32, pin_memory=True)
    S.sl_get_planes(ctxs[0].handle, t_mean.numpy(), t_hi.numpy().view(hi.dtype).reshape(hi.shape), None)
    h2d = t_mean.numel() * 8 + t_hi.numel() * 4

    def issue(i):   # upload + one Strang step of step i, enqueued only
        c = ctxs[i % 2]
        S.sl_set_planes(c.handle, t_mean.data_ptr(), t_hi.data_ptr(), None)
        c.step("strang", p.dt, 1)

    def run(n):
        masses = []
        issue(0)
        for i in range(n):
            if i + 1 < n:
                issue(i + 1)
            masses.append(ctxs[i % 2].mass())   # waits for step i only
        return masses

    run(max(args.warmup, 2))
    barrier(world)
    t0 = time.perf_counter()
    masses = run(args.steps)
    secs = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    sweeps = 2 * len(p.grid.x_dims()) + len(p.grid.v_dims())
    ms_max, units = aggregate(secs * 1000.0, float(args.steps * sweeps * p.dof), world, dev)
    return {"value": units / (ms_max / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": 8, "ms_per_step": ms_max / args.steps,
            "note": "per step: upload of a whole state from pinned host memory, one Strang step, its mass "
                    "read back; two contexts on two streams take the steps in turn, so each upload "
                    "overlaps the previous step's sweeps (the host link's H2D bandwidth bounds it)",
            "masses_equal": bool(np.all(np.asarray(masses) == masses[0]))}


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "paper1d":
        run_paper1d(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
