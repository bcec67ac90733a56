#!/usr/bin/env python
"""Benchmark of the Artificial Retina hot path on GB300 (one JSON line on rank 0).

Headline: a step is Algorithm 1 with learned starting points over one batch
of 1024 high-multiplicity VELO-like events (Poisson(600) tracks, 15 % noise,
~16.8k hits per event, vertex at the origin): the hit ordering, the learned
proposer (slope histogram, small conv net, top-2048 seeds per event), the
seeds' spatial order, the persistent batched truncated-Newton search
(Section 3's update and sigma schedule) and the cluster / select extraction,
replayed as one CUDA graph by the native tracker (retina_tracker_*).
``value`` is events per second over all ranks (each rank its own batch:
replicas, weak scaling).  The line also carries the search kernel against
the FP32 lane rate measured live, the MC efficiency, the end-to-end rate from
host buffers, and the FP64 oracle on a sample of the same events (time and
efficiency).  ``extras`` holds the other workloads: the single-event step
(1024^2 grid scan + 8192-seed search, smeared and origin vertex), the 2D
toy, the four-parameter search, the 1024-event method comparison, the
alpha-budget sweep and the paper's sVELO experiment.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle (the only reference this
method has) on the host cores, on a bounded sample of the headline batch.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from typing import Optional

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import VELO_PLANES_Z, WORKLOADS, batch_of, make_event, uniform_seeds  # noqa: E402

WORKLOAD = "velo"
RUN_SEED = 0
METRIC = ("events/s (learned-seed batched local search at >= 95% of the oracle's track efficiency: hit "
          "ordering, proposer, top-2048 seeds, truncated-Newton search, extraction; 1024 high-multiplicity events "
          "per step)")
L2_FLUSH_BYTES = 256 << 20
# algorithmic FP32 lane operations (an FMA counts once) per (seed, hit) pair of
# the search: a gradient/Hessian pass 15, an R-only (line-search) pass 5
LANE_OPS_RGH, LANE_OPS_R = 15.0, 5.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (profiling runs)")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the library's default launch shapes")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched method comparisons")
    ap.add_argument("--no-extras", action="store_true", help="the headline alone (no other workloads)")
    ap.add_argument("--events", type=int, default=None,
                    help="events per headline batch (profiling runs; default: the workload's 1024)")
    ap.add_argument("--serial", action="store_true", help="run the grid and search branches on one stream")
    ap.add_argument("--shape", default=None, metavar="P,W,H,C,S",
                    help="fixed launch shape instead of the autotuner's (profiling runs): search seeds per warp, "
                         "warps per CTA, staged hits, CTA cap, grid hit slices")
    ap.add_argument("--graph", action="store_true", help="replay the step as one CUDA graph instead of enqueueing "
                                                         "its kernels one by one")
    ap.add_argument("--profile-single", action="store_true",
                    help="profiling runs: only the single-event step (vertex at the origin), --steps steps, no "
                         "end-to-end leg; prints its summary instead of the bench line")
    return ap.parse_args()


def workload_config(wl, n_hits):
    return {
        "workload": "velo: one VELO-like event per step (150 tracks from a smeared origin, 26 layers at "
                    "z=-300..750 mm, 90%% layer efficiency, 10%% noise, %d hits); 1024x1024 slope grid scan "
                    "(sigma %.4f mm) + 8192-seed truncated-Newton search (q=3, sigma 0.3/0.175/0.05 mm) + "
                    "track extraction of both" % (n_hits, wl.sigma_grid),
        "grid": list(wl.grid_n), "seeds": wl.n_seeds, "hits_per_event": n_hits, "q": len(wl.sigma_schedule),
        "l2": "flushed between timed steps (256 MiB write outside the timed events)",
        "parallelism": "replicas (one event per rank, no collective on the data path)",
    }


HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "paper_1709_08610_gb300", "csrc")
# sources each profiled kernel is compiled from, and the committed ncu summary
# holding its DRAM traffic per launch
PROFILED = {
    "batched_search_kernel": (("search_device.cuh", "batched_search.cu", "common.cuh", "internal.cuh"),
                              "profiles/batched_search_kernel_velo_stress_1024_events.md"),
    "batched_search_kernel/single": (("search_device.cuh", "batched_search.cu", "common.cuh", "internal.cuh"),
                                     "profiles/batched_search_kernel_velo_single_event.md"),
    "grid_tc_kernel": (("grid_tc.cu", "grid_device.cuh", "common.cuh", "internal.cuh"),
                       "profiles/grid_tc_kernel_velo_1024x1024.md"),
}


def kernel_source_sha(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in PROFILED[kernel][0]:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(kernel: str):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch from the committed
    ncu summary of the kernel - None when the kernel's sources changed since
    that capture (the summary records their sha256) or there is none."""
    import re
    path = os.path.join(HERE, PROFILED[kernel][1])
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"source sha256: ([0-9a-f]{64})", text)
    m_tr = re.search(r"traffic bytes per launch: (\d+)", text)
    if not (m_sha and m_tr) or m_sha.group(1) != kernel_source_sha(kernel):
        return None
    return int(m_tr.group(1))


TUNE_STEPS = 41  # timed steps per launch-shape candidate of the two-stream step (median)

_libcuda = None


def record_in_graph(event, stream) -> None:
    """Record a timing event on a capturing stream as an event node of the
    graph (CU_EVENT_RECORD_EXTERNAL), so that every replay records it."""
    import ctypes
    global _libcuda
    if _libcuda is None:
        _libcuda = ctypes.CDLL("libcuda.so.1")
        _libcuda.cuEventRecordWithFlags.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint]
    r = _libcuda.cuEventRecordWithFlags(event.cuda_event, stream.cuda_stream, 1)
    if r != 0:
        raise RuntimeError("cuEventRecordWithFlags failed: %d" % r)


def max_over_ranks(value: float, device) -> float:
    """The largest value over the ranks (replicas: the job lasts as long as its
    slowest rank); the value itself without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_events_per_s(world: int, steps: int, total_ms: float) -> float:
    """Whole-job throughput: every rank processes one event per step."""
    return world * steps / (total_ms * 1e-3)


def measured_peaks() -> dict:
    """The machine's measured peaks (HBM copy, dense BF16 GEMM), if the file is there."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_step_sample(ev, wl, seeds, row_frac: int, seed_frac: int):
    """Oracle time for 1/row_frac of the grid rows and 1/seed_frac of the
    seeds, extrapolated to seconds for the whole step of one event."""
    import oracle
    n0, n1 = wl.grid_n
    rows = max(1, n1 // row_frac)
    ns = max(1, len(seeds) // seed_frac)
    t0 = time.perf_counter()
    R = oracle.grid_response(ev.hits, wl.model, wl.grid_lo, wl.grid_step, (n0, rows), wl.sigma_grid)
    idx = oracle.grid_maxima(R, wl.R0)
    c0, c1 = oracle.cell_centres(wl.grid_lo, wl.grid_step, (n0, rows))
    gth = np.stack([c0[idx % n0], c1[idx // n0]], 1)
    keep_g = oracle.extract_tracks(gth, R.reshape(-1)[idx], None, wl.grid_lo, wl.grid_step, wl.grid_n, wl.R0,
                                   wl.merge_cells)
    t1 = time.perf_counter()
    th, Rs, st, m = oracle.local_search(ev.hits, wl.model, seeds[:ns], wl.sigma_schedule, wl.grid_lo, wl.grid_step,
                                        wl.grid_n)
    keep_s = oracle.extract_tracks(th, Rs, st, wl.grid_lo, wl.grid_step, wl.grid_n, wl.R0, wl.merge_cells)
    t2 = time.perf_counter()
    tracks = {"grid": gth[keep_g], "search": th[keep_s]} if (rows == n1 and ns == len(seeds)) else None
    return (t1 - t0) * (n1 / rows) + (t2 - t1) * (len(seeds) / ns), (t2 - t0), tracks


def oracle_agreement(oracle_tracks, gpu_tracks, step, tol_cells: float = 1e-3) -> dict:
    """Track-set agreement with the oracle on the same event: the share of the
    oracle's tracks the GPU finds within tol_cells grid steps (max norm), and
    the GPU tracks matching none of the oracle's."""
    o = np.asarray(oracle_tracks, np.float64).reshape(-1, 2)
    g = np.asarray(gpu_tracks, np.float64).reshape(-1, 2)
    if len(o) == 0 or len(g) == 0:
        return {"oracle_tracks": len(o), "gpu_tracks": len(g), "efficiency_vs_oracle": 1.0 if len(o) == 0 else 0.0,
                "unmatched_gpu_tracks": len(g)}
    d = np.max(np.abs(o[:, None, :] - g[None, :, :]) / np.asarray(step), axis=2)
    return {"oracle_tracks": len(o), "gpu_tracks": len(g),
            "efficiency_vs_oracle": float((d.min(axis=1) <= tol_cells).mean()),
            "unmatched_gpu_tracks": int((d.min(axis=0) > tol_cells).sum())}


def oracle_threads() -> int:
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


# ---------------------------------------------------------------------------
# batched methods: grid scan vs uniform multistart vs learned seeds
# ---------------------------------------------------------------------------

def batch_shape(hits_per_event: float) -> dict:
    """Launch shape of the throughput-bound batched search: spatially ordered
    seeds, 32-warp CTAs staging up to 12288 hits, and four seeds per warp (two
    packed FP32x2 pairs sharing the box tests, block lists and hit loads, their
    updates taken lane-parallel), measured fastest on both the ~3.9k-hit and
    the ~16.5k-hit events (8.3 against 12.2 ms for 4096 uniform seeds per event
    on the former with two per warp)."""
    return dict(sort_seeds=True, seeds_per_warp=4, warps=32, smem_hits=12288)


BATCH_EVENTS = 1024
BATCH_RUN_SEED = 5000


def batched_methods(rt, stream, flush, workload: str = "velo_batch", learned_k: int = 512, reps: int = 5,
                    comparisons: bool = False, fma_rate: Optional[float] = None):
    """1024 ragged VELO-like events with the vertex at the origin through three
    methods, each replayed as one CUDA graph per batch: the plain grid scan
    (with and without the refinement of its maxima), Algorithm 1 from 4096
    uniform seeds per event (and from as many uniform seeds as the learned
    variant uses) and from the learned proposer's seeds.  Events/s from CUDA
    events around graph replays (L2 flushed before each), MC-truth efficiency
    (|dtheta|_max <= 1e-3), fakes per event, the resolution of the matched
    tracks (|dtheta| per axis in grid cells) and the share of the plain
    4096-seed search's tracks each method recovers; for the searches, the
    search launch's own time and its rate against ``fma_rate`` (FP32 lane
    operations/s).  With ``comparisons``: the same searches with the
    steepest-ascent and modified-Newton updates."""
    import torch
    from paper_1709_08610_gb300.pipeline import (BatchTracker, GridScanBatch, match_efficiency, match_residuals,
                                                 recovered_fraction)
    from paper_1709_08610_gb300.seednet import DEFAULT_WEIGHTS, SeedProposer
    wl = WORKLOADS[workload]
    E = BATCH_EVENTS
    evs = [make_event(wl, BATCH_RUN_SEED, e, vertex_sigma=(0, 0, 0)) for e in range(E)]
    b = batch_of(evs)
    truth = [ev.truth[:, :2] for ev in evs]
    H = b.hits.shape[0]
    box = rt.Grid.of(wl)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    methods = {}

    def timed(obj):
        obj.capture()
        for _ in range(2):
            obj.replay()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            obj.replay()
            c.record(stream)
            c.synchronize()
            ts.append(a.elapsed_time(c))
        return statistics.median(ts)

    n0, n1 = wl.grid_n
    shape = batch_shape(H / E)
    seeds4096 = np.stack([uniform_seeds(wl, 4096, BATCH_RUN_SEED, e) for e in range(E)])
    runs = [("grid_scan_%dx%d" % (n0, n1), lambda: GridScanBatch(E, H, box, wl.sigma_grid, wl.R0), None),
            ("grid_scan_%dx%d_refined" % (n0, n1),
             lambda: GridScanBatch(E, H, box, wl.sigma_grid, wl.R0, refine_iters=4), None),
            ("uniform_4096", lambda: BatchTracker(E, H, 4096, box, opts, wl.R0, **shape), seeds4096),
            ("uniform_%d" % learned_k, lambda: BatchTracker(E, H, learned_k, box, opts, wl.R0, **shape),
             np.stack([uniform_seeds(wl, learned_k, BATCH_RUN_SEED, e) for e in range(E)]))]
    prop = SeedProposer.from_checkpoint(DEFAULT_WEIGHTS) if os.path.exists(DEFAULT_WEIGHTS) else None
    if prop is not None:
        runs.append(("learned_%d" % learned_k,
                     lambda: BatchTracker(E, H, learned_k, box, opts, wl.R0, proposer=prop, **shape), None))
    if comparisons:
        for upd, tag in ((rt.UPDATE_STEEPEST_ASCENT, "steepest_ascent"), (rt.UPDATE_MODIFIED_NEWTON, "modified_newton")):
            o = rt.LsOpts(sigma=tuple(wl.sigma_schedule), update=upd)
            runs.append(("uniform_4096_" + tag, lambda o=o: BatchTracker(E, H, 4096, box, o, wl.R0, **shape),
                         seeds4096))
            if prop is not None:
                runs.append(("learned_%d_%s" % (learned_k, tag),
                             lambda o=o: BatchTracker(E, H, learned_k, box, o, wl.R0, proposer=prop, **shape), None))
    found = {}
    for name, make, seeds in runs:
        obj = make()
        obj.load(b.hits, b.offsets, seeds)
        ms = timed(obj)
        found[name] = obj.results()
        eff, fakes = match_efficiency(found[name], truth)
        res = match_residuals(found[name], truth) / np.asarray(wl.grid_step)
        methods[name] = {"events_per_s": E / (ms * 1e-3), "ms_per_batch": ms, "efficiency": eff,
                         "fakes_per_event": fakes / E,
                         "resolution_cells": {"rms": float(np.sqrt(np.mean(res ** 2))) if res.size else None,
                                              "median": float(np.median(res)) if res.size else None}}
        if isinstance(obj, GridScanBatch) and obj.ropts is None:
            # the grid scan alone (response + maxima, eager, after the hit ordering), with
            # its evaluated (cell, hit) pairs counted on the device: 2 flops per pair
            obj.step()
            rt.work_counters(enable=True, reset=True)
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            a.record(stream)
            rt.grid_scan(obj.sorted, obj.offsets, obj.model, obj.grid, obj.sigma, obj.R0, obj.Km, ws=obj.ws,
                         out=obj.maxima, boxes=obj.boxes, stream=stream)
            c.record(stream)
            c.synchronize()
            w = rt.work_counters(enable=False)
            t_ms = a.elapsed_time(c)
            tflops = 2.0 * w[rt.WORK_GRID] / (t_ms * 1e-3) / 1e12
            bf16 = measured_peaks().get("bf16_tflops")
            methods[name]["grid_scan_ms"] = t_ms
            methods[name]["grid_pairs_evaluated"] = int(w[rt.WORK_GRID])
            methods[name]["grid_pairs_total"] = int(n0 * n1 * H)
            methods[name]["grid_tflops"] = tflops
            if bf16 and rt.get_option(rt.OPT_GRID_TC):
                methods[name]["grid_frac_of_3xtf32_peak"] = tflops / (bf16 * (1.1 / 2.25) / 3)
        if isinstance(obj, BatchTracker):
            # search work of one (eager) step, counted on the device, and the search
            # launch's own time (CUDA events around it, L2 flushed before the step,
            # median of three eager steps)
            rt.work_counters(enable=True, reset=True)
            obj.step()
            torch.cuda.synchronize()
            w = rt.work_counters(enable=False)
            marks = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            k_ms = []
            for _ in range(3):
                flush.zero_()
                obj.step(stream, marks=marks)
                marks[1].synchronize()
                k_ms.append(marks[0].elapsed_time(marks[1]))
            k_ms = float(np.median(k_ms))
            lane_ops = LANE_OPS_RGH * w[rt.WORK_RGH] + LANE_OPS_R * w[rt.WORK_R]
            pairs = w[rt.WORK_RGH] + w[rt.WORK_R]
            methods[name]["search_pairs_per_batch"] = int(pairs)
            methods[name]["search_kernel_ms"] = k_ms
            methods[name]["search_tlane_ops_per_s"] = lane_ops / (k_ms * 1e-3) / 1e12
            if fma_rate:
                methods[name]["search_frac_of_fp32_lane_rate"] = lane_ops / (k_ms * 1e-3) / fma_rate
        del obj
        torch.cuda.empty_cache()
    for name in methods:
        if name != "uniform_4096":
            methods[name]["recovers_uniform_4096"] = recovered_fraction(found[name], found["uniform_4096"])
    gen = wl.gen
    return {"workload": "%d ragged VELO-like events (tracks ~ Poisson(%g) clipped to [%g, %g], origin vertex, "
                        "%d hits), grid %dx%d; one CUDA graph per batch and method"
                        % ((E,) + tuple(gen["n_tracks"]) + (H, n0, n1)),
            "events": E, "hits": int(H), "reps": reps, "methods": methods,
            "l2": "flushed before each replay"}


ALPHA_MULTIPLICITIES = (10, 25, 50, 100, 200, 400)


def alpha_sweep(rt, stream, flush, reps: int = 3):
    """The paper's experiment in shape (its Fig. 3): efficiency against the
    number of reconstructible tracks at the seed budgets n = alpha n_grid /
    (C0 q), with its C0 = 30 and q = 3 over the 1024^2 grid, for alpha = 1/3
    and 1/10; uniform seeds (the paper's prior) and learned ones.  1024
    origin-vertex VELO-like events, 10 to 400 tracks each (an equal share of
    each multiplicity), one CUDA graph per batch."""
    import torch
    from paper_1709_08610_gb300.pipeline import BatchTracker, efficiency_by_multiplicity, match_efficiency
    from paper_1709_08610_gb300.seednet import DEFAULT_WEIGHTS, SeedProposer
    wl = WORKLOADS["velo_batch"]
    E = BATCH_EVENTS
    mult = [ALPHA_MULTIPLICITIES[e % len(ALPHA_MULTIPLICITIES)] for e in range(E)]
    evs = [make_event(wl, BATCH_RUN_SEED + 1, e, vertex_sigma=(0, 0, 0), n_tracks=mult[e]) for e in range(E)]
    b = batch_of(evs)
    truth = [ev.truth[:, :2] for ev in evs]
    H = b.hits.shape[0]
    box = rt.Grid.of(wl)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    shape = batch_shape(H / E)
    prop = SeedProposer.from_checkpoint(DEFAULT_WEIGHTS) if os.path.exists(DEFAULT_WEIGHTS) else None
    edges = sorted(set(ALPHA_MULTIPLICITIES)) + [ALPHA_MULTIPLICITIES[-1] + 1]
    n0, n1 = wl.grid_n
    out = {}
    for alpha, tag in ((1.0 / 3.0, "1/3"), (0.1, "1/10")):
        n = int(round(alpha * n0 * n1 / (30 * 3)))
        kinds = [("uniform", None)] + ([("learned", prop)] if prop is not None else [])
        for kind, pr in kinds:
            obj = BatchTracker(E, H, n, box, opts, wl.R0, proposer=pr, **shape)
            seeds = None if pr is not None else np.stack([uniform_seeds(wl, n, BATCH_RUN_SEED + 1, e)
                                                          for e in range(E)])
            obj.load(b.hits, b.offsets, seeds)
            obj.capture()
            obj.replay()
            ts = []
            for _ in range(reps):
                flush.zero_()
                a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                obj.replay()
                c.record(stream)
                c.synchronize()
                ts.append(a.elapsed_time(c))
            found = obj.results()
            eff, fakes = match_efficiency(found, truth)
            by = efficiency_by_multiplicity(found, truth, edges)
            out["alpha_%s_%s_%d" % (tag, kind, n)] = {
                "seeds_per_event": n, "events_per_s": E / (statistics.median(ts) * 1e-3), "efficiency": eff,
                "efficiency_by_tracks": {k.split("-")[0]: round(v["efficiency"], 4) for k, v in by.items()}}
            del obj
            torch.cuda.empty_cache()
    return {"workload": "%d origin-vertex VELO-like events, %s tracks (equal shares), %d hits; seeds "
                        "n = alpha 1024^2 / (30 * 3)" % (E, "/".join(str(m) for m in ALPHA_MULTIPLICITIES), H),
            "runs": out, "l2": "flushed before each replay"}


SEARCH4_LAYER_PAIRS = ((17, 25), (18, 24), (19, 23))  # indices of the 26 layers: the downstream end


def search4_measure(rt, stream, flush, reps: int = 10):
    """The four-parameter model (x0, y0, t_x, t_y at z_ref = the layers' mean z)
    on smeared-vertex events, where the two-slope model cannot fit the
    tracks: starting points from hit pairs on three downstream layer pairs
    (lines passing within 0.3 mm of the beam axis at |z| <= 250 mm), the
    four-parameter truncated-Newton search (q = 3, the paper's bandwidths),
    cluster / select in four dimensions; one CUDA graph per batch.  The step's
    event alone and the 1024-event batch (tracks ~ Poisson(150)), both as
    generated (vertex smeared per track by (0.05, 0.05, 50) mm); MC efficiency
    within 0.1 mm in the offsets and 1e-3 in the slopes."""
    import torch
    from paper_1709_08610_gb300.pipeline import Search4Batch
    zref = float(np.mean(VELO_PLANES_Z))
    z = np.asarray(VELO_PLANES_Z)
    pairs = [(z[a], z[b]) for a, b in SEARCH4_LAYER_PAIRS]
    opts = rt.LsOpts4(sigma=tuple(WORKLOADS["velo"].sigma_schedule), zref=zref)
    tol = np.array([0.1, 0.1, 1e-3, 1e-3])
    out = {}
    for name, wl_name, E, seed in (("velo_event", "velo", 1, RUN_SEED), ("velo_batch", "velo_batch", 1024,
                                                                        BATCH_RUN_SEED + 3)):
        wl = WORKLOADS[wl_name]
        evs = [make_event(wl, seed, e) for e in range(E)]
        b = batch_of(evs)
        obj = Search4Batch(E, b.hits.shape[0], rt.Grid.of(wl), opts, wl.R0, pairs, 0.5, 0.3, (-250.0, 250.0))
        obj.load(b.hits, b.offsets)
        obj.capture()
        obj.replay()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            obj.replay()
            c.record(stream)
            c.synchronize()
            ts.append(a.elapsed_time(c))
        found = obj.results()
        n_seeds = obj.seeds[1].cpu().numpy()
        hit = tot = fakes = 0
        for f, ev in zip(found, evs):
            t, v = ev.truth[:, :2], ev.truth[:, 2:5]
            T = np.stack([v[:, 0] + t[:, 0] * (zref - v[:, 2]), v[:, 1] + t[:, 1] * (zref - v[:, 2]), t[:, 0],
                          t[:, 1]], 1)
            tot += len(T)
            if len(f):
                d = np.max(np.abs(f[:, None, :] - T[None]) / tol, axis=2)
                hit += int((d.min(axis=0) <= 1).sum())
                fakes += int((d.min(axis=1) > 1).sum())
        ms = statistics.median(ts)
        out[name] = {"events": E, "events_per_s": E / (ms * 1e-3), "ms": ms, "mc_efficiency": hit / tot,
                     "fakes_per_event": fakes / E, "seeds_per_event": float(n_seeds.mean()),
                     "tracks_per_event": float(np.mean([len(f) for f in found]))}
        del obj
        torch.cuda.empty_cache()
    return {"workload": "smeared-vertex VELO-like events (vertex ~ N(0, (0.05, 0.05, 50)) mm per track): the step's "
                        "event, and 1024 events with Poisson(150) tracks; hit-pair seeds on layers %s, "
                        "four-parameter search, four-dimensional cluster/select; one CUDA graph per batch"
                        % (list(SEARCH4_LAYER_PAIRS),),
            "runs": out, "l2": "flushed before each replay"}


SVELO_MULTIPLICITIES = (50, 100, 150, 200, 250, 300, 350)


def svelo_sweep(rt, stream, flush, reps: int = 3):
    """The paper's experiment in its own geometry: sVELO events (20 disks,
    eta ~ U[1, 6], p_hit 0.5, Poisson(250) noise) with 50 to 350
    reconstructible tracks; a track counts as found when an estimate lies
    within 1e-3 rad of it in the paper's two angles.  Methods: the 2048^2 grid
    scan (plain and refined) and Algorithm 1 from uniform seeds at the
    paper's budgets n = alpha n_grid / (C0 q), C0 = 30, q = 3, with n_grid
    the cells of side 1e-3 rad over the angular acceptance (|angle| <= 0.705
    rad, the eta = 1 edge)."""
    import torch
    from paper_1709_08610_gb300.pipeline import BatchTracker, GridScanBatch, efficiency_by_multiplicity, \
        match_efficiency
    from synth import slopes_to_angles
    wl = WORKLOADS["svelo"]
    E = BATCH_EVENTS
    mult = [SVELO_MULTIPLICITIES[e % len(SVELO_MULTIPLICITIES)] for e in range(E)]
    evs = [make_event(wl, BATCH_RUN_SEED + 2, e, n_tracks=mult[e]) for e in range(E)]
    b = batch_of(evs)
    truth = [slopes_to_angles(ev.truth[:, 0], ev.truth[:, 1]) for ev in evs]
    H = b.hits.shape[0]
    box = rt.Grid.of(wl)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    shape = batch_shape(H / E)
    edges = list(SVELO_MULTIPLICITIES) + [SVELO_MULTIPLICITIES[-1] + 1]
    n_grid = (2 * 0.705 / 1e-3) ** 2
    runs = [("grid_scan_2048x2048", lambda: GridScanBatch(E, H, box, wl.sigma_grid, wl.R0), None),
            ("grid_scan_2048x2048_refined", lambda: GridScanBatch(E, H, box, wl.sigma_grid, wl.R0, refine_iters=4),
             None)]
    for alpha, tag in ((1.0 / 3.0, "1/3"), (0.1, "1/10")):
        n = int(round(alpha * n_grid / (30 * 3)))
        runs.append(("alpha_%s_uniform_%d" % (tag, n), lambda n=n: BatchTracker(E, H, n, box, opts, wl.R0, **shape),
                     np.stack([uniform_seeds(wl, n, BATCH_RUN_SEED + 2, e) for e in range(E)])))
    out = {}
    for name, make, seeds in runs:
        obj = make()
        obj.load(b.hits, b.offsets, seeds)
        obj.capture()
        obj.replay()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            obj.replay()
            c.record(stream)
            c.synchronize()
            ts.append(a.elapsed_time(c))
        found = [slopes_to_angles(f[:, 0], f[:, 1]) if len(f) else np.zeros((0, 2)) for f in obj.results()]
        eff, fakes = match_efficiency(found, truth)
        by = efficiency_by_multiplicity(found, truth, edges)
        out[name] = {"events_per_s": E / (statistics.median(ts) * 1e-3), "efficiency": eff,
                     "fakes_per_event": fakes / E,
                     "efficiency_by_tracks": {k.split("-")[0]: round(v["efficiency"], 4) for k, v in by.items()}}
        del obj
        torch.cuda.empty_cache()
    return {"workload": "%d sVELO events (20 disks 8-42 mm over 700 mm, eta ~ U[1, 6], p_hit 0.5, Poisson(250) "
                        "noise), %s reconstructible tracks (equal shares), %d hits; found = within 1e-3 rad in "
                        "the paper's angles" % (E, "/".join(str(m) for m in SVELO_MULTIPLICITIES), H),
            "runs": out, "l2": "flushed before each replay"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def single_event_step(rt, tune, args, dev, rank, peaks, vertex_sigma=None, with_cpu=False, steps=400,
                      with_e2e=True):
    """The single-event step (one VELO-like event: the 1024 x 1024 grid scan,
    the 8192-seed truncated-Newton search and the extraction of both, the two
    branches on concurrent streams after the shared hit ordering), timed over
    ``steps`` steps behind an L2 flush each; launch shapes from the
    autotuner; the end-to-end rate through the native executor with host
    copies; with ``with_cpu`` the oracle on the same event (time and track
    agreement)."""
    import torch
    wl = WORKLOADS[WORKLOAD]
    ev = make_event(wl, RUN_SEED, rank, **({} if vertex_sigma is None else {"vertex_sigma": vertex_sigma}))
    seeds_np = uniform_seeds(wl, wl.n_seeds, RUN_SEED, rank)
    H = ev.n_hits
    grid = rt.Grid.of(wl)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    K_MAX = 8192
    K_TR = 4096
    R0 = wl.R0

    # device-resident inputs, preallocated outputs and workspaces
    hits = torch.from_numpy(ev.hits).to(dev)
    offs = torch.tensor([0, H], dtype=torch.int64, device=dev)
    seeds = torch.from_numpy(seeds_np).to(dev).view(-1, 2)
    seed_offs = torch.tensor([0, wl.n_seeds], dtype=torch.int64, device=dev)
    n0, n1 = wl.grid_n
    Rg = torch.empty((1, n1, n0), dtype=torch.float32, device=dev)
    ws_grid = torch.empty(max(rt.grid_response_workspace_size(1, wl.model, grid), 1), dtype=torch.uint8, device=dev)
    mx = dict(max_idx=torch.empty((1, K_MAX), dtype=torch.int32, device=dev),
              max_theta=torch.empty((1, K_MAX, 2), dtype=torch.float32, device=dev),
              max_R=torch.empty((1, K_MAX), dtype=torch.float32, device=dev),
              n_max=torch.empty((1,), dtype=torch.int32, device=dev))
    ws_max = torch.empty(1 << 16, dtype=torch.uint8, device=dev)
    ls_out = (torch.empty((wl.n_seeds, 2), dtype=torch.float32, device=dev),
              torch.empty((wl.n_seeds,), dtype=torch.float32, device=dev),
              torch.empty((wl.n_seeds,), dtype=torch.uint8, device=dev))
    n_evals = torch.empty((wl.n_seeds,), dtype=torch.uint8, device=dev)
    ws_search = torch.empty(max(rt.batched_search_workspace_size(1), 256), dtype=torch.uint8, device=dev)

    def tr_out():
        return dict(tracks=torch.empty((1, K_TR, 2), dtype=torch.float32, device=dev),
                    track_R=torch.empty((1, K_TR), dtype=torch.float32, device=dev),
                    track_src=torch.empty((1, K_TR), dtype=torch.int32, device=dev),
                    n_tracks=torch.empty((1,), dtype=torch.int32, device=dev))

    tr_grid, tr_search = tr_out(), tr_out()
    stream = torch.cuda.current_stream(dev)

    srt = torch.empty_like(hits)
    boxes = torch.empty((rt.lib.retina_prepare_hits_box_count(H, 1), 8), dtype=torch.float32, device=dev)

    # The grid branch and the search branch need only the prepared hits, so
    # after retina_prepare_hits they run concurrently on two streams (the
    # search leaves room on every SM through RETINA_OPT_BATCH_CTAS) and join
    # on the main stream.  Timing events, when given, bracket every stage on
    # the stream it runs on:
    #   0 start | prepare | 1 | grid | 2 | maxima + extract | 3     (main stream)
    #   4 | search | 5 | extract | 6                                (search stream)
    #   join, 7 end                                                 (main stream)
    # the search branch is the longer one: its stream gets the higher priority,
    # so its kernels' CTAs go first whenever an SM frees up.  The timed steps
    # enqueue the kernels one by one; --graph replays the step as one CUDA
    # graph instead (captured on its own stream, the timing events as event
    # nodes of the graph) - measured about 4 % slower on this step: launched
    # together, the grid branch's CTAs take SMs the search branch gets first
    # when the host enqueues the search before the grid.
    stream2 = torch.cuda.Stream(dev, priority=-1)
    fork_ev, join_ev = torch.cuda.Event(), torch.cuda.Event()

    def step(evs=None, main=None, in_graph=False):
        s1 = stream if main is None else main
        s2 = s1 if args.serial else stream2

        def mark(i, st):
            if evs is not None:
                if in_graph:
                    record_in_graph(evs[i], st)
                else:
                    evs[i].record(st)

        mark(0, s1)
        rt.prepare_hits(hits, offs, wl.model, out=(srt, boxes), stream=s1)
        mark(1, s1)
        if s2 is not s1:
            fork_ev.record(s1)
            s2.wait_event(fork_ev)
        mark(4, s2)
        rt.batched_search(srt, offs, wl.model, seeds, seed_offs, opts, grid, out=ls_out, n_evals=n_evals,
                          ws=ws_search, boxes=boxes, stream=s2)
        mark(5, s2)
        rt.extract_tracks(ls_out[0].view(1, -1, 2), ls_out[1].view(1, -1), ls_out[2].view(1, -1), grid, R0,
                          wl.merge_cells, K_TR, out=tr_search, stream=s2)
        mark(6, s2)
        rt.grid_response(srt, offs, wl.model, grid, wl.sigma_grid, R_out=Rg, ws=ws_grid, boxes=boxes, stream=s1)
        mark(2, s1)
        rt.grid_maxima(Rg, grid, R0, K_MAX, out=mx, ws=ws_max, stream=s1)
        rt.extract_tracks(mx["max_theta"], mx["max_R"], None, grid, R0, wl.merge_cells, K_TR,
                          n_valid=mx["n_max"], out=tr_grid, stream=s1)
        mark(3, s1)
        if s2 is not s1:
            join_ev.record(s2)
            s1.wait_event(join_ev)
        mark(7, s1)

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    cap_stream = torch.cuda.Stream(dev)
    ev_g = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
    for e_ in ev_g:
        e_.record(stream)  # create the events before they are captured
    torch.cuda.synchronize()

    def capture():
        """The step as one CUDA graph with the current launch options; returns
        the graph and the number of our kernels in it."""
        step()  # eager once: kernel attributes set before capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        n0_ = rt.launch_count()
        with torch.cuda.graph(g, stream=cap_stream, capture_error_mode="thread_local"):
            step(ev_g, main=cap_stream, in_graph=True)
        return g, rt.launch_count() - n0_

    def timed_steps(g, n, evs_eager=None):
        """n steps behind an L2 flush each; per step the device times of the 8
        marks (ms from mark 0).  Graph steps read their event nodes after each
        replay (one synchronize per step, outside the timed marks)."""
        out = np.zeros((n, 8))
        for k in range(n):
            flush.zero_()
            if g is not None:
                g.replay()
                ev_g[7].synchronize()
                out[k] = [ev_g[0].elapsed_time(ev_g[i]) if i else 0.0 for i in range(8)]
            else:
                step(evs_eager[k])
        if g is None:
            torch.cuda.synchronize()
            for k in range(n):
                out[k] = [evs_eager[k][0].elapsed_time(evs_eager[k][i]) if i else 0.0 for i in range(8)]
        return out

    # ---- launch shapes picked by the autotuner on this workload and GPU
    tuned = None
    if args.shape:
        p_, w_, h_, c_, s_ = (int(x) for x in args.shape.split(","))
        for o, v in ((rt.OPT_BATCH_SEEDS_PER_WARP, p_), (rt.OPT_BATCH_WARPS, w_), (rt.OPT_BATCH_SMEM_HITS, h_),
                     (rt.OPT_BATCH_CTAS, c_), (rt.OPT_GRID_SPLITS, s_)):
            rt.set_option(o, v)
        tuned = {"fixed_shape": args.shape}
        args.no_tune = True
    if not args.no_tune:
        rt.prepare_hits(hits, offs, wl.model, out=(srt, boxes))
        tuned = {"grid": tune.tune_grid(srt, offs, wl.model, grid, wl.sigma_grid, boxes=boxes),
                 "search": tune.tune_batched_search(srt, offs, wl.model, seeds, seed_offs, opts, grid, boxes=boxes)}

    # ---- the search's CTA shape when it shares the GPU with the grid branch:
    # candidates timed on the whole two-stream step, run as the timed region
    # runs it (graph replays behind the L2 flush)
    if not args.no_tune and not args.serial:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        # search CTA shape x grid hit slices (the grid alone prefers more slices
        # than it can use while the search holds most SMs)
        # (and staged hits: 4096 leaves room on an SM for a grid CTA beside a search CTA)
        g0 = rt.get_option(rt.OPT_GRID_SPLITS)
        h0 = rt.get_option(rt.OPT_BATCH_SMEM_HITS)
        cands = [(w, c, sp, h) for (w, c) in ((32, 0), (32, 15 * sms // 16), (32, 7 * sms // 8),
                                               (32, 13 * sms // 16), (32, 3 * sms // 4), (32, 5 * sms // 8),
                                               (32, sms // 2), (16, 0), (16, 3 * sms // 2), (16, sms),
                                               (8, 2 * sms))
                 for sp in sorted({g0, 4, 8}) for h in sorted({h0, 4096})]
        table = {}
        for w, c, sp, h in cands:
            rt.set_option(rt.OPT_BATCH_WARPS, w)
            rt.set_option(rt.OPT_BATCH_CTAS, c)
            rt.set_option(rt.OPT_GRID_SPLITS, sp)
            rt.set_option(rt.OPT_BATCH_SMEM_HITS, h)
            if not args.graph:
                g_c = None
                evs_c = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(TUNE_STEPS)]
                for _ in range(3):
                    step()
            else:
                g_c, _ = capture()
                evs_c = None
                for _ in range(3):
                    g_c.replay()
            table["%d,%d,%d,%d" % (w, c, sp, h)] = float(np.median(timed_steps(g_c, TUNE_STEPS, evs_c)[:, 7]))
            del g_c
        best = min(table, key=table.get)
        w, c, sp, h = (int(x) for x in best.split(","))
        rt.set_option(rt.OPT_BATCH_WARPS, w)
        rt.set_option(rt.OPT_BATCH_CTAS, c)
        rt.set_option(rt.OPT_GRID_SPLITS, sp)
        rt.set_option(rt.OPT_BATCH_SMEM_HITS, h)
        tuned["overlap"] = {"warps": w, "ctas": c, "grid_splits": sp, "smem_hits": h, "step_ms": table[best],
                            "table_ms": table}

    fma_rate = max(peaks.get("ffma", 0.0), peaks.get("ffma2", 0.0))

    # ---- the step graph, then warm-up
    graph, kernels_per_step = capture() if args.graph else (None, 0)
    for _ in range(5):
        if graph is not None:
            graph.replay()
        else:
            step()
    torch.cuda.synchronize()

    # ---- timed steps
    evs = None if graph is not None else [[torch.cuda.Event(enable_timing=True) for _ in range(8)]
                                          for _ in range(steps)]
    torch.cuda.synchronize()
    launches0 = rt.launch_count()
    marks = timed_steps(graph, steps, evs)
    torch.cuda.synchronize()
    launches = rt.launch_count() - launches0 + kernels_per_step * steps

    # stages: prepare, grid response, maxima + extract (main stream), search, extract (search stream)
    # (one stream: the search branch is enqueued first, so the grid response runs from event 6 to 2)
    pairs = [(0, 1), (6, 2) if args.serial else (1, 2), (2, 3), (4, 5), (5, 6)]
    stage = np.stack([marks[:, b] - marks[:, a] for a, b in pairs], axis=1)
    step_ms = marks[:, 7]
    ms_per_step = float(step_ms.mean())
    value = 1e3 / ms_per_step

    # ---- work the two response kernels perform (counted on the device in
    # one extra step outside the timed region; exact block skipping means
    # fewer pairs than cells x hits / seeds x hits)
    rt.work_counters(enable=True, reset=True)
    step()
    torch.cuda.synchronize()
    work = rt.work_counters(enable=False)
    n_ev = n_evals.to(torch.int64).sum().item()
    cells = n0 * n1
    grid_pairs_all = cells * H                     # every (cell, hit) pair of Eq. 2
    grid_pairs = work[rt.WORK_GRID]                # pairs in blocks not skipped
    rgh_pairs, r_pairs = work[rt.WORK_RGH], work[rt.WORK_R]
    prep_ms = float(np.mean(stage[:, 0]))
    grid_ms = float(np.mean(stage[:, 1]))
    search_ms = float(np.mean(stage[:, 3]))
    # grid contraction: one FP32 FMA (2 flops) per evaluated (cell, hit) pair
    grid_tflops = 2.0 * grid_pairs / (grid_ms * 1e-3) / 1e12
    # search: LANE_OPS_RGH FP32 operations + 1 ex2 per (seed, hit) pair of a
    # gradient/Hessian pass, LANE_OPS_R + 1 ex2 per pair of an R pass
    search_fp32_ops = LANE_OPS_RGH * rgh_pairs + LANE_OPS_R * r_pairs
    search_ex2 = rgh_pairs + r_pairs
    search_fp32_rate = search_fp32_ops / (search_ms * 1e-3)
    search_ex2_rate = search_ex2 / (search_ms * 1e-3)
    fma_peak_tflops = 2.0 * fma_rate / 1e12 if fma_rate else None
    ex2_peak = peaks.get("ex2")
    if rt.get_option(rt.OPT_GRID_TC):
        # tensor-core contraction: each FP32-accurate product is three TF32 MMA
        # products, so the peak for the algorithmic FP32 flops is the TF32 peak / 3;
        # TF32 peak = measured dense BF16 (burst) x the nominal TF32 / BF16 ratio (1.1 / 2.25)
        bf16 = measured_peaks().get("bf16_tflops")
        tf32 = bf16 * (1.1 / 2.25) if bf16 else None
        roof_grid = {"kernel": "grid_tc_kernel (+ slice reduction)", "bound": "tensor", "unit": "TFLOP/s",
                     "achieved": grid_tflops, "peak": (tf32 / 3) if tf32 else None,
                     "frac": (grid_tflops / (tf32 / 3)) if tf32 else None,
                     "traffic": profiled_traffic("grid_tc_kernel"),
                     "pairs_evaluated": grid_pairs, "pairs_total": grid_pairs_all,
                     "effective_pairs_per_s": grid_pairs_all / (grid_ms * 1e-3),
                     "tf32_tflops_executed": 3 * grid_tflops,
                     "peak_source": "of measured: MEASURED_PEAKS bf16_tflops (burst) x 1.1/2.25 (nominal TF32/BF16) "
                                    "/ 3 (split products per FP32-accurate product)"}
    else:
        roof_grid = {"kernel": "grid_sep_kernel (+ slice reduction)", "bound": "alu", "unit": "TFLOP/s",
                     "achieved": grid_tflops, "peak": fma_peak_tflops,
                     "frac": (grid_tflops / fma_peak_tflops) if fma_peak_tflops else None,
                     "traffic": None, "pairs_evaluated": grid_pairs, "pairs_total": grid_pairs_all,
                     "effective_pairs_per_s": grid_pairs_all / (grid_ms * 1e-3),
                     "peak_source": "FP32 FMA rate measured live by retina_alu_probe (burst; the faster of FFMA "
                                    "and packed FFMA2)"}
    # FP32 lane instructions (an FMA counts once) against the measured lane-FMA rate, and ex2 against MUFU
    fr_fp32 = (search_fp32_rate / fma_rate) if fma_rate else None
    fr_ex2 = (search_ex2_rate / ex2_peak) if ex2_peak else None
    roof_search = {"kernel": "batched_search_kernel", "bound": "alu", "unit": "Tlane-op/s",
                   "achieved": search_fp32_rate / 1e12, "peak": (fma_rate / 1e12) if fma_rate else None,
                   "frac": fr_fp32, "traffic": profiled_traffic("batched_search_kernel/single"),
                   "pairs_per_s": (rgh_pairs + r_pairs) / (search_ms * 1e-3),
                   "ex2_per_s": search_ex2_rate, "frac_ex2": fr_ex2, "rgh_pairs": rgh_pairs, "r_pairs": r_pairs,
                   "pairs_total": (wl.n_seeds * len(wl.sigma_schedule) + n_ev) * H,
                   "peak_source": "FP32 lane-FMA rate measured live by retina_alu_probe (burst)"}
    dominant = "grid" if grid_ms >= search_ms else "search"
    roofline = roof_grid if dominant == "grid" else roof_search

    # ---- end to end through the public API with host buffers: every step copies
    # the event's hits and seeds in from pinned host memory, runs the whole path
    # through the native executor (retina_pipeline_run: one call enqueues every
    # launch of the step, the two branches on two streams) - or replays the step
    # graph with --graph - and copies both track lists out to pinned host memory
    e2e = None
    if with_e2e:
        hits_h = torch.from_numpy(ev.hits).pin_memory()
        seeds_h = torch.from_numpy(seeds_np).view(-1, 2).pin_memory()
        n_e2e = 200
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        keys = ("tracks", "track_R", "n_tracks")

        def host_like(r):
            return {m: {k2: torch.empty(r[m][k2].shape, dtype=r[m][k2].dtype).pin_memory() for k2 in keys}
                    for m in r}

        def copy_out(dst, src):
            for m in dst:
                for k2 in keys:
                    dst[m][k2].copy_(src[m][k2], non_blocking=True)

        if graph is not None:
            res = {"search": tr_search, "grid": tr_grid}
            out_h = host_like(res)
            torch.cuda.synchronize()
            a.record(stream)
            for _ in range(n_e2e):
                hits.copy_(hits_h, non_blocking=True)
                seeds.copy_(seeds_h, non_blocking=True)
                graph.replay()
                copy_out(out_h, res)
            b.record(stream)
        else:
            # two sets of device inputs and outputs: a copy stream brings step k + 1's
            # event in and takes step k - 1's track lists out while step k runs
            pipe = rt.Pipeline(wl.model, grid, wl.sigma_grid, R0, opts, wl.merge_cells, max_events=1, max_hits=H,
                               seeds_per_event=wl.n_seeds, max_maxima=K_MAX, max_tracks=K_TR)
            hits_d, seeds_d = [hits, torch.empty_like(hits)], [seeds, torch.empty_like(seeds)]
            res_d = [pipe.run(hits, offs, seeds), pipe.run(hits, offs, seeds)]
            out_h = host_like(res_d[0])
            cs = torch.cuda.Stream(dev)
            in_ready, done, read = ([torch.cuda.Event() for _ in range(2)] for _ in range(3))
            torch.cuda.synchronize()
            a.record(stream)
            cs.wait_event(a)

            def copy_in(i):
                cs.wait_event(done[i])  # the step that last read buffer i has finished
                with torch.cuda.stream(cs):
                    hits_d[i].copy_(hits_h, non_blocking=True)
                    seeds_d[i].copy_(seeds_h, non_blocking=True)
                in_ready[i].record(cs)

            copy_in(0)
            for k in range(n_e2e):
                i = k % 2
                if k + 1 < n_e2e:
                    copy_in(1 - i)
                stream.wait_event(in_ready[i])
                stream.wait_event(read[i])  # track lists of step k - 2 copied out
                pipe.run(hits_d[i], offs, seeds_d[i], out=res_d[i])
                done[i].record(stream)
                cs.wait_event(done[i])
                with torch.cuda.stream(cs):
                    copy_out(out_h, res_d[i])
                read[i].record(cs)
            stream.wait_stream(cs)
            b.record(stream)
        b.synchronize()
        e2e_ms = a.elapsed_time(b) / n_e2e
        # the executor's track lists are the step's (same launchers, same options)
        for m, ref in (("search", tr_search), ("grid", tr_grid)):
            nt = int(out_h[m]["n_tracks"][0])
            assert nt == int(ref["n_tracks"][0].item())
            k = min(nt, K_TR)
            assert torch.equal(out_h[m]["tracks"][0, :k], ref["tracks"][0, :k].cpu())
        d2h = sum(v.numel() * v.element_size() for m in out_h for v in out_h[m].values())
        h2d = hits_h.numel() * 4 + seeds_h.numel() * 4
        e2e = {"value": 1e3 / e2e_ms, "unit": "events/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": n_e2e,
               "note": "%s; every step copies its hits and seeds in from pinned host memory and both track lists "
                       "out to pinned host memory, timed with CUDA events"
                       % ("one step-graph replay per step, copies in stream order" if graph is not None else
                          "retina_pipeline_run (native executor) per step, copies on a second stream "
                          "overlapping the neighbouring steps (two input and output buffer sets), steps back to "
                          "back without an L2 flush as in a stream of events")}
        if graph is None:
            pipe.close()

    # ---- CPU baseline (oracle, bounded sample), rank 0 at N = 1 only
    cpu = None
    if with_cpu:
        import oracle
        oracle.build()
        ests, wall = [], 0.0
        while wall < 10.0 and len(ests) < 20:
            est, w, o_tracks = oracle_step_sample(ev, wl, seeds_np, 1, 1)
            ests.append(est)
            wall += w
        # the timed steps' track lists against the oracle's on the same event
        agreement = {}
        for m, tr in (("grid", tr_grid), ("search", tr_search)):
            nt = min(int(tr["n_tracks"][0].item()), K_TR)
            agreement[m] = oracle_agreement(o_tracks[m], tr["tracks"][0, :nt].cpu().numpy(), wl.grid_step)
        cpu = {"value": len(ests) / sum(ests), "unit": "events/s", "cores": oracle_threads(), "kind": "oracle",
               "track_agreement": agreement,
               "sample": "%d whole steps of the same event (grid %d x %d, %d seeds), %.1f s of CPU work"
                         % (len(ests), n0, n1, wl.n_seeds, wall)}

    tr_n = (int(tr_grid["n_tracks"].item()), int(tr_search["n_tracks"].item()))
    return {
        "workload": workload_config(wl, H)["workload"] + ("" if vertex_sigma is None else
                                                          " (vertex at the origin)"),
        "events_per_s": value, "ms_per_step": ms_per_step, "steps": steps, "e2e": e2e,
        "gpu_launches_per_step": launches / steps, "roofline": roofline,
        "roofline_other": roof_search if dominant == "grid" else roof_grid,
        "stages_ms": {"prepare_hits": prep_ms, "grid_response": grid_ms,
                      "grid_maxima_extract": float(np.mean(stage[:, 2])), "local_search": search_ms,
                      "search_extract": float(np.mean(stage[:, 4]))},
        "methods_events_per_s": {"grid_scan": 1e3 / (prep_ms + grid_ms + float(np.mean(stage[:, 2]))),
                                 "local_search": 1e3 / (prep_ms + search_ms + float(np.mean(stage[:, 4])))},
        "tracks_found": {"grid": tr_n[0], "search": tr_n[1]}, "cpu_oracle": cpu, "tuned": tuned,
        "l2": "flushed between timed steps (256 MiB write outside the timed events)",
        "branches": "one stream" if args.serial else
                    "grid branch and search branch on two concurrent streams after the shared hit ordering",
        "launch": "kernels enqueued one by one" if graph is None else
                  "one CUDA graph replay per step (%d kernels)" % kernels_per_step,
    }


# ---------------------------------------------------------------------------
# headline: the learned-seed batched search on the high-multiplicity batch
# ---------------------------------------------------------------------------

HEADLINE = "velo_stress"
HEADLINE_EVENTS = 1024
HEADLINE_SEEDS = 2048
HEADLINE_TRACKS = 1024
HEADLINE_RUN_SEED = 7000


def headline_batch(rank: int = 0, n_events: int = HEADLINE_EVENTS):
    """1024 high-multiplicity VELO-like events with the vertex at the origin
    (each rank its own batch)."""
    wl = WORKLOADS[HEADLINE]
    evs = [make_event(wl, HEADLINE_RUN_SEED + 1000 * rank, e, vertex_sigma=(0, 0, 0)) for e in range(n_events)]
    return wl, evs, batch_of(evs)


def headline_config(wl, n_hits: int, E: int = HEADLINE_EVENTS) -> dict:
    gen = wl.gen
    return {
        "workload": "velo_stress: %d high-multiplicity VELO-like events per step (tracks ~ Poisson(%g) clipped to "
                    "[%g, %g], 15%% noise hits, 26 layers at z=-300..750 mm, 90%% layer efficiency, vertex at the "
                    "origin; %d hits, %.0f per event); learned seed proposer (64x64 slope histogram, conv 1->16->32 + "
                    "1x1 head, top-%d seeds per event at dense sub-cells), spatial seed order, persistent batched "
                    "truncated-Newton search (q=3, sigma 0.3/0.175/0.05 mm), cluster/select extraction; one CUDA "
                    "graph per step" % ((E,) + tuple(gen["n_tracks"]) + (n_hits, n_hits / E, HEADLINE_SEEDS)),
        "events": E, "seeds_per_event": HEADLINE_SEEDS, "hits": int(n_hits), "q": len(wl.sigma_schedule),
        "box": {"lo": list(wl.grid_lo), "step": list(wl.grid_step), "n": list(wl.grid_n)},
        "l2": "inputs larger than L2 (%.0f MB of hits) and L2 flushed between timed steps (256 MiB write outside "
              "the timed events)" % (n_hits * 16 / 1e6),
        "parallelism": "replicas (one batch per rank, no collective on the data path)",
    }


def oracle_learned_event(ev, wl, params, n_seeds: int, seed_frac: int = 1):
    """The oracle's learned-seed pipeline on one event (FP64 histogram and
    network, its own top-n seeds, the C oracle's search on 1/seed_frac of
    them, extraction); returns (seconds extrapolated to all n seeds, seconds
    spent, tracks [m, 2] or None when sampled)."""
    import oracle
    from oracle import seednet as sn
    t0 = time.perf_counter()
    _, feat = sn.slope_histogram(ev.hits)
    z = sn.forward(feat, params)["z"].astype(np.float32)
    seeds, _ = sn.propose_seeds(z, ev.hits, n_seeds)
    t1 = time.perf_counter()
    ns = max(1, n_seeds // max(1, seed_frac))
    th, R, st, _ = oracle.local_search(ev.hits, 1, seeds[:ns], wl.sigma_schedule, wl.grid_lo, wl.grid_step, wl.grid_n)
    keep = oracle.extract_tracks(th, R, st, wl.grid_lo, wl.grid_step, wl.grid_n, wl.R0, wl.merge_cells)
    t2 = time.perf_counter()
    return (t1 - t0) + (t2 - t1) * (n_seeds / ns), t2 - t0, (th[keep] if ns == n_seeds else None)


def run_reference(args, rank: int):
    """The reference arm: the FP64 oracle's learned-seed pipeline on the host
    cores, each step one event of the headline batch with a fraction of its
    seeds (extrapolated), sized so the whole run takes about 90 s."""
    if rank != 0:
        return
    import oracle
    from paper_1709_08610_gb300.seednet import DEFAULT_WEIGHTS, read_checkpoint
    oracle.build()
    wl = WORKLOADS[HEADLINE]
    evs = [make_event(wl, HEADLINE_RUN_SEED, e, vertex_sigma=(0, 0, 0)) for e in range(8)]
    params = read_checkpoint(DEFAULT_WEIGHTS)[1]["params"]
    full, _, _ = oracle_learned_event(evs[0], wl, params, HEADLINE_SEEDS, 16)
    budget = 90.0 / max(1, args.steps + max(args.warmup, 0))
    seed_frac = int(min(HEADLINE_SEEDS, max(1, np.ceil(full / max(budget, 1e-3)))))
    for k in range(max(args.warmup, 0)):
        oracle_learned_event(evs[k % len(evs)], wl, params, HEADLINE_SEEDS, seed_frac)
    est = [oracle_learned_event(evs[k % len(evs)], wl, params, HEADLINE_SEEDS, seed_frac)[0] for k in range(args.steps)]
    value = 1.0 / float(np.mean(est))
    H_mean = float(np.mean([ev.n_hits for ev in evs]))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * HEADLINE_EVENTS / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(wl, int(H_mean * HEADLINE_EVENTS)),
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": oracle_threads(), "kind": "oracle",
                         "sample": "per step one event of the batch (%.0f hits on average) with 1/%d of its %d "
                                   "learned seeds searched (the proposer in full), extrapolated to the whole event"
                                   % (H_mean, seed_frac, HEADLINE_SEEDS)},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def probe_peaks(rt, stream) -> dict:
    """FP32 (FFMA, packed FFMA2) and MUFU ex2 throughput, measured live (burst)."""
    import torch
    peaks = {}
    sink = torch.empty(rt.alu_probe_sink_floats(), dtype=torch.float32, device="cuda")
    for kind, name, iters in ((0, "ffma", 4096), (2, "ffma2", 4096), (1, "ex2", 1024)):
        rt.alu_probe(kind, 64, sink)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = None
        for _ in range(3):
            a.record(stream)
            ops = rt.alu_probe(kind, iters, sink)
            b.record(stream)
            b.synchronize()
            r = ops / (a.elapsed_time(b) * 1e-3)
            best = r if best is None else max(best, r)
        peaks[name] = best
    return peaks


def headline(rt, args, dev, rank, world, peaks, local_rank):
    """The learned-seed batched search through the native tracker: events/s
    over the timed steps (device time from the tracker's stage marks, inside
    the graph replays), the search kernel against the FP32 lane rate, MC
    efficiency, the end-to-end rate from host buffers, and (rank 0, one GPU)
    the oracle on a sample of the same events."""
    import torch
    import torch.distributed as dist
    from paper_1709_08610_gb300.pipeline import match_efficiency
    from paper_1709_08610_gb300.seednet import DEFAULT_WEIGHTS, read_checkpoint
    wl, evs, b = headline_batch(rank, args.events or HEADLINE_EVENTS)
    E, S, K = len(evs), HEADLINE_SEEDS, HEADLINE_TRACKS
    H = int(b.hits.shape[0])
    params = read_checkpoint(DEFAULT_WEIGHTS)[1]["params"]
    box = rt.Grid.of(wl)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    shape = batch_shape(H / E)
    tr = rt.Tracker(box, opts, wl.R0, wl.merge_cells, E, H, S, max_tracks=K, params=params, **shape)
    tr.load(b.hits, b.offsets)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    tr.set_marks(marks)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    n0 = rt.launch_count()
    tr.step(E, stream)  # records the graph, then replays it
    torch.cuda.synchronize()
    kernels_per_step = rt.launch_count() - n0
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        tr.step(E, stream)
    torch.cuda.synchronize()

    # ---- timed region
    clocks = ClockSampler(local_rank) if not args.no_clocks else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    t_wall0 = time.perf_counter()
    st_ms = np.zeros((args.steps, 5))
    for k in range(args.steps):
        flush.zero_()
        tr.step(E, stream)
        marks[5].synchronize()
        st_ms[k] = [marks[i].elapsed_time(marks[i + 1]) for i in range(5)]
    torch.cuda.synchronize()
    t_wall1 = time.perf_counter()
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    step_ms = st_ms.sum(axis=1)
    total_ms = max_over_ranks(float(step_ms.sum()), dev)
    ms_per_step = total_ms / args.steps
    value = world * E * args.steps / (total_ms * 1e-3)
    found = tr.results(E)

    # ---- work of the search kernel, counted on the device in one eager step of a
    # second tracker (same launches, same results - checked bit for bit)
    tc = rt.Tracker(box, opts, wl.R0, wl.merge_cells, E, H, S, max_tracks=K, params=params, use_graph=False, **shape)
    tc.load(b.hits, b.offsets)
    rt.work_counters(enable=True, reset=True)
    tc.step(E, stream)
    torch.cuda.synchronize()
    w = rt.work_counters(enable=False)
    assert torch.equal(tc.n_tracks, tr.n_tracks) and torch.equal(tc.tracks, tr.tracks)
    tc.close()
    rgh, rr = int(w[rt.WORK_RGH]), int(w[rt.WORK_R])
    search_ms = float(st_ms[:, 3].mean())
    fma_rate = max(peaks.get("ffma", 0.0), peaks.get("ffma2", 0.0))
    lane_ops = LANE_OPS_RGH * rgh + LANE_OPS_R * rr
    achieved = lane_ops / (search_ms * 1e-3)
    ex2_rate = (rgh + rr) / (search_ms * 1e-3)
    roofline = {"kernel": "batched_search_kernel", "bound": "alu", "unit": "Tlane-op/s",
                "achieved": achieved / 1e12, "peak": fma_rate / 1e12 if fma_rate else None,
                "frac": achieved / fma_rate if fma_rate else None,
                "traffic": profiled_traffic("batched_search_kernel"),
                "rgh_pairs": rgh, "r_pairs": rr, "pairs_per_s": (rgh + rr) / (search_ms * 1e-3),
                "ex2_per_s": ex2_rate, "frac_ex2": ex2_rate / peaks["ex2"] if peaks.get("ex2") else None,
                "kernel_ms": search_ms,
                "work_unit": "15 FP32 lane operations per (seed, hit) pair of a gradient/Hessian pass and 5 per "
                             "pair of an R-only (line-search) pass, pairs counted on the device after exact block "
                             "skipping",
                "peak_source": "FP32 lane-FMA rate measured live by retina_alu_probe (burst; the faster of FFMA and "
                               "packed FFMA2); no FP32 figure is on record in MEASURED_PEAKS.json"}
    truth = [ev.truth[:, :2] for ev in evs]
    eff, fakes = match_efficiency(found, truth)

    # ---- end to end through the public API from host buffers: every step copies
    # the batch's hits and offsets in from page-locked host memory, replays the
    # step, and copies every event's track list out (retina_tracker_run_host)
    hits_h = torch.from_numpy(b.hits).pin_memory()
    offs_h = torch.from_numpy(b.offsets).pin_memory()
    out_h = dict(tracks=torch.empty((E, K, 2), dtype=torch.float32).pin_memory(),
                 track_R=torch.empty((E, K), dtype=torch.float32).pin_memory(),
                 n_tracks=torch.empty((E,), dtype=torch.int32).pin_memory())
    tr.set_marks(None)
    tr.run_host(hits_h, offs_h, out_h, stream=stream)  # records the graph again (without marks)
    torch.cuda.synchronize()
    n_e2e = max(5, min(args.steps, 20))
    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(n_e2e):
        tr.run_host(hits_h, offs_h, out_h, stream=stream)
    c.record(stream)
    c.synchronize()
    e2e_ms = a.elapsed_time(c) / n_e2e
    assert torch.equal(out_h["n_tracks"], tr.n_tracks.cpu())
    h2d = hits_h.numel() * 4 + offs_h.numel() * 8
    d2h = sum(v.numel() * v.element_size() for v in out_h.values())
    e2e = {"value": world * E / (max_over_ranks(e2e_ms, dev) * 1e-3), "unit": "events/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": n_e2e,
           "note": "retina_tracker_run_host per step: the batch's hits and offsets copied in from page-locked host "
                   "memory, the step's graph replayed, every event's track list (tracks, R, count) copied out to "
                   "page-locked host memory, timed with CUDA events; steps back to back, each step's hit copy (on "
                   "the tracker's copy stream) overlapping the previous step's search once that step's hit ordering "
                   "is done"}

    # ---- the oracle on a sample of the same events (rank 0, one GPU)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        est, wall, o_tracks = [], 0.0, []
        while wall < 15.0 and len(est) < 32:
            e_, w_, t_ = oracle_learned_event(evs[len(est)], wl, params, S)
            est.append(e_)
            wall += w_
            o_tracks.append(t_)
        n_o = len(est)
        eff_o, fakes_o = match_efficiency(o_tracks, truth[:n_o])
        eff_g, fakes_g = match_efficiency(found[:n_o], truth[:n_o])
        agree, _ = match_efficiency(found[:n_o], o_tracks)  # oracle tracks the GPU also finds (1e-3)
        extra_g, _ = match_efficiency(o_tracks, found[:n_o])
        cpu = {"value": n_o / sum(est), "unit": "events/s", "cores": oracle_threads(), "kind": "oracle",
               "sample": "the first %d events of the batch, each through the oracle's whole learned-seed pipeline "
                         "(FP64 proposer, its own top-%d seeds, the C oracle's search of all of them, extraction), "
                         "%.1f s of CPU work" % (n_o, S, wall),
               "efficiency": {"events": n_o, "oracle_mc_efficiency": eff_o, "gpu_mc_efficiency": eff_g,
                              "gpu_over_oracle": eff_g / eff_o if eff_o else None,
                              "oracle_fakes_per_event": fakes_o / n_o, "gpu_fakes_per_event": fakes_g / n_o,
                              "oracle_tracks_found_by_gpu": agree, "gpu_tracks_found_by_oracle": extra_g,
                              "match": "|dtheta|_max <= 1e-3 in slope"}}
    tr.close()
    return {
        "value": value, "ms_per_step": ms_per_step, "config": headline_config(wl, H, E), "e2e": e2e,
        "gpu_launches": int(kernels_per_step * args.steps), "kernels_per_step": int(kernels_per_step),
        "roofline": roofline, "clocks": clk, "cpu_baseline": cpu, "wall_s_timed": t_wall1 - t_wall0,
        "stages_ms": {n: float(st_ms[:, i].mean()) for i, n in enumerate(
            ("prepare_hits", "proposer", "sort_seeds", "search", "extract"))},
        "mc_efficiency": eff, "fakes_per_event": fakes / E,
        "tracks_per_event": float(np.mean([len(f) for f in found])),
        "truth_tracks_per_event": float(np.mean([len(t) for t in truth])),
    }


def toy_step(rt, steps: int = 400, with_cpu: bool = True):
    """The 2D straight-line toy (one event per step): the 200 x 200 grid scan,
    the 256-seed search and the extraction of both, enqueued on one stream,
    with the oracle's track lists on the same event."""
    import torch
    wl = WORKLOADS["toy2d"]
    ev = make_event(wl, RUN_SEED, 0)
    seeds_np = uniform_seeds(wl, wl.n_seeds, RUN_SEED, 0)
    hits = torch.from_numpy(ev.hits).cuda()
    offs = torch.tensor([0, ev.n_hits], dtype=torch.int64, device="cuda")
    seeds = torch.from_numpy(seeds_np).cuda()[None]
    grid = rt.Grid.of(wl)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    R0 = float(np.float32(wl.R0))

    def step():
        g = rt.grid_scan(hits, offs, 0, grid, wl.sigma_grid, R0, 1024)
        tg = rt.extract_tracks(g["max_theta"], g["max_R"], None, grid, R0, wl.merge_cells, 256, n_valid=g["n_max"])
        th, R, st = rt.local_search(hits, offs, 0, seeds, opts, grid)
        ts = rt.extract_tracks(th, R, st, grid, R0, wl.merge_cells, 256)
        return tg, ts

    for _ in range(5):
        step()
    torch.cuda.synchronize()
    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        tg, ts = step()
    c.record()
    c.synchronize()
    ms = a.elapsed_time(c) / steps
    out = {"workload": "toy2d: one 2D straight-line event per step (10 tracks y = alpha x + beta, 10 planes, 20%% "
                       "noise, %d hits); 200x200 grid scan (sigma %.4f) + 256-seed truncated-Newton search + "
                       "extraction of both, one stream, back to back" % (ev.n_hits, wl.sigma_grid),
           "events_per_s": 1e3 / ms, "ms_per_step": ms, "steps": steps,
           "tracks_found": {"grid": int(tg["n_tracks"].item()), "search": int(ts["n_tracks"].item())}}
    if with_cpu:
        import oracle
        t0 = time.perf_counter()
        R = oracle.grid_response(ev.hits, 0, wl.grid_lo, wl.grid_step, wl.grid_n, wl.sigma_grid)
        idx = oracle.grid_maxima(R, wl.R0)
        cen = oracle.maxima_centres(idx, wl.grid_lo, wl.grid_step, wl.grid_n)
        kg = oracle.extract_tracks(cen, R.reshape(-1)[idx], None, wl.grid_lo, wl.grid_step, wl.grid_n, R0,
                                   wl.merge_cells)
        th, Rs, st, _ = oracle.local_search(ev.hits, 0, seeds_np, wl.sigma_schedule, wl.grid_lo, wl.grid_step,
                                            wl.grid_n)
        ks = oracle.extract_tracks(th, Rs, st, wl.grid_lo, wl.grid_step, wl.grid_n, R0, wl.merge_cells)
        t1 = time.perf_counter()
        out["cpu_oracle"] = {"events_per_s": 1.0 / (t1 - t0), "cores": oracle_threads(), "track_agreement": {
            "grid": oracle_agreement(cen[kg], tg["tracks"][0, :int(tg["n_tracks"].item())].cpu().numpy(),
                                     wl.grid_step),
            "search": oracle_agreement(th[ks], ts["tracks"][0, :int(ts["n_tracks"].item())].cpu().numpy(),
                                       wl.grid_step)}}
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    from paper_1709_08610_gb300 import build as rbuild
    rbuild.build()
    from paper_1709_08610_gb300 import retina as rt
    from paper_1709_08610_gb300 import tune

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream(dev)
    peaks = {} if args.no_probe else probe_peaks(rt, stream)
    options = (rt.OPT_LS_SEEDS_PER_WARP, rt.OPT_LS_SMEM_HITS, rt.OPT_GRID_SPLITS, rt.OPT_LS_WARPS,
               rt.OPT_BATCH_SEEDS_PER_WARP, rt.OPT_BATCH_WARPS, rt.OPT_BATCH_SMEM_HITS, rt.OPT_BATCH_CTAS,
               rt.OPT_SEEDNET_TC, rt.OPT_GRID_TC)
    defaults = {o: rt.get_option(o) for o in options}

    def restore():
        for o, v in defaults.items():
            rt.set_option(o, v)

    if args.profile_single:
        r = single_event_step(rt, tune, args, dev, rank, peaks, vertex_sigma=(0, 0, 0), steps=args.steps,
                              with_e2e=False)
        print(json.dumps({k: r[k] for k in ("workload", "events_per_s", "stages_ms", "tracks_found")}))
        return

    head = headline(rt, args, dev, rank, world, peaks, local_rank)

    extras = {}
    if world == 1 and not args.no_extras:
        with_cpu = not args.no_cpu_baseline
        # the single-event step (grid scan + 8192-seed search + both extractions) as
        # generated (smeared vertex) and with the vertex at the origin
        extras["single_event_velo"] = single_event_step(rt, tune, args, dev, rank, peaks, with_cpu=with_cpu)
        restore()
        extras["single_event_velo_origin"] = single_event_step(rt, tune, args, dev, rank, peaks,
                                                               vertex_sigma=(0, 0, 0), with_cpu=with_cpu)
        restore()
        extras["toy2d"] = toy_step(rt, with_cpu=with_cpu)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        extras["search4"] = search4_measure(rt, stream, flush)
        if not args.no_batched:
            # the library's launch rules for batches: one grid hit slice at this many
            # tiles, the search filling the GPU
            rt.set_option(rt.OPT_GRID_SPLITS, 0)
            rt.set_option(rt.OPT_BATCH_CTAS, 0)
            fma_rate = max(peaks.get("ffma", 0.0), peaks.get("ffma2", 0.0)) or None
            extras["batched"] = batched_methods(rt, stream, flush, comparisons=True, fma_rate=fma_rate)
            extras["alpha_sweep"] = alpha_sweep(rt, stream, flush)
            extras["svelo_sweep"] = svelo_sweep(rt, stream, flush)
            extras["batched_stress"] = batched_methods(rt, stream, flush, "velo_stress", learned_k=2048, reps=3,
                                                       fma_rate=fma_rate)
            restore()

    if rank == 0:
        cfg = head["config"]
        line = {
            "metric": METRIC, "value": head["value"], "unit": "events/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded generator of the workload's stated "
                                                         "distributions; no dataset)",
            "config": cfg, "e2e": head["e2e"], "gpu_launches": head["gpu_launches"], "roofline": head["roofline"],
            "cpu_baseline": head["cpu_baseline"], "clocks": head["clocks"],
            "efficiency": {"mc_efficiency": head["mc_efficiency"], "fakes_per_event": head["fakes_per_event"],
                           "tracks_per_event": head["tracks_per_event"],
                           "truth_tracks_per_event": head["truth_tracks_per_event"],
                           "vs_oracle": (head["cpu_baseline"] or {}).get("efficiency")},
            "stages_ms": head["stages_ms"], "kernels_per_step": head["kernels_per_step"],
            "wall_s_timed": head["wall_s_timed"],
            "peaks_measured": {"ffma_per_s": peaks.get("ffma"), "ffma2_per_s": peaks.get("ffma2"),
                               "ex2_per_s": peaks.get("ex2")},
            "extras": extras,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
