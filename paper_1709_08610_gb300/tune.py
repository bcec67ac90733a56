"""Autotuner for the launch shapes of the retina kernels.

Sweeps, on the caller's workload and GPU, the options the C library exposes
(retina_set_option): seeds per warp and warps per CTA of the local search,
hit slices of the grid response.  Each candidate is timed with CUDA events on
the current stream (median of a few repetitions after a warm-up); the best
values are applied and returned, and cached as JSON keyed by the device name,
SM count and workload shape so a later process can reuse them
(``load_cached``).  Results never depend on these options beyond FP32
summation order (the grid slices) - the search's per-seed arithmetic is the
same in every shape.
"""
from __future__ import annotations

import json
import os
import statistics
from typing import Callable, Dict, Iterable, Optional

import torch

from . import build as _build
from . import retina as rt

CACHE = os.path.join(_build.OUT, "tuning.json")


def _time(fn: Callable[[], None], reps: int = 5, warm: int = 2) -> float:
    s = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def _key(kind: str, shape: Dict) -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s|%s|sm%d|%s" % (kind, p.name, p.multi_processor_count,
                              ",".join("%s=%s" % kv for kv in sorted(shape.items())))


def _store(key: str, value: Dict):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    data = {}
    if os.path.exists(CACHE):
        try:
            data = json.load(open(CACHE))
        except Exception:
            data = {}
    data[key] = value
    tmp = CACHE + ".tmp%d" % os.getpid()
    json.dump(data, open(tmp, "w"), indent=1)
    os.replace(tmp, CACHE)


def load_cached(kind: str, shape: Dict) -> Optional[Dict]:
    if not os.path.exists(CACHE):
        return None
    try:
        return json.load(open(CACHE)).get(_key(kind, shape))
    except Exception:
        return None


def tune_local_search(hits, offs, model: int, seeds, opts: "rt.LsOpts", box: "rt.Grid",
                      spw: Iterable[int] = (1, 2, 4), warps: Iterable[int] = (4, 8, 16),
                      reps: int = 5) -> Dict:
    """Pick seeds-per-warp and warps-per-CTA for this search; applies and returns them."""
    E = offs.numel() - 1
    n = seeds.shape[-2]
    out = (torch.empty((E, n, 2), dtype=torch.float32, device=hits.device),
           torch.empty((E, n), dtype=torch.float32, device=hits.device),
           torch.empty((E, n), dtype=torch.uint8, device=hits.device))
    old = (rt.get_option(rt.OPT_LS_SEEDS_PER_WARP), rt.get_option(rt.OPT_LS_WARPS))
    table = {}
    for p in spw:
        for w in warps:
            rt.set_option(rt.OPT_LS_SEEDS_PER_WARP, p)
            rt.set_option(rt.OPT_LS_WARPS, w)
            table["%d,%d" % (p, w)] = _time(lambda: rt.local_search(hits, offs, model, seeds, opts, box, out=out),
                                            reps=reps)
    best = min(table, key=table.get)
    p, w = (int(x) for x in best.split(","))
    rt.set_option(rt.OPT_LS_SEEDS_PER_WARP, p)
    rt.set_option(rt.OPT_LS_WARPS, w)
    res = {"seeds_per_warp": p, "warps": w, "ms": table[best], "table_ms": table, "default": list(old)}
    _store(_key("local_search", {"E": E, "n": n, "H": int(hits.shape[0]), "model": model}), res)
    return res


def tune_grid(hits, offs, model: int, grid: "rt.Grid", sigma: float, splits: Iterable[int] = (0, 4, 8, 12, 16, 19, 24, 32),
              reps: int = 5, boxes=None) -> Dict:
    """Pick the hit-slice count of the grid response (0 = the library's rule)."""
    E = offs.numel() - 1
    n0, n1 = grid.n
    R = torch.empty((E, n1, n0), dtype=torch.float32, device=hits.device)
    table = {}
    for s in splits:
        rt.set_option(rt.OPT_GRID_SPLITS, s)
        ws = torch.empty(max(rt.grid_response_workspace_size(E, model, grid), 1), dtype=torch.uint8,
                         device=hits.device)
        table[str(s)] = _time(lambda: rt.grid_response(hits, offs, model, grid, sigma, R_out=R, ws=ws, boxes=boxes),
                              reps=reps)
    best = min(table, key=table.get)
    rt.set_option(rt.OPT_GRID_SPLITS, int(best))
    res = {"splits": int(best), "ms": table[best], "table_ms": table}
    _store(_key("grid", {"E": E, "n0": n0, "n1": n1, "H": int(hits.shape[0]), "model": model}), res)
    return res


def tune_batched_search(hits, offs, model: int, seeds, seed_offs, opts: "rt.LsOpts", box: "rt.Grid",
                        spw: Iterable[int] = (1, 2, 4), warps: Iterable[int] = (8, 16, 32),
                        smem_hits: Iterable[int] = (4096, 8192), reps: int = 5, boxes=None) -> Dict:
    """Pick seeds-per-warp, warps-per-CTA and staged hits of the persistent search."""
    E = offs.numel() - 1
    S = seeds.numel() // 2
    dev = hits.device
    out = (torch.empty((S, 2), dtype=torch.float32, device=dev), torch.empty((S,), dtype=torch.float32, device=dev),
           torch.empty((S,), dtype=torch.uint8, device=dev))
    ws = torch.empty(max(rt.batched_search_workspace_size(E), 256), dtype=torch.uint8, device=dev)
    table = {}
    for p in spw:
        for w in warps:
            for h in smem_hits:
                rt.set_option(rt.OPT_BATCH_SEEDS_PER_WARP, p)
                rt.set_option(rt.OPT_BATCH_WARPS, w)
                rt.set_option(rt.OPT_BATCH_SMEM_HITS, h)
                table["%d,%d,%d" % (p, w, h)] = _time(
                    lambda: rt.batched_search(hits, offs, model, seeds, seed_offs, opts, box, out=out, ws=ws,
                                              boxes=boxes),
                    reps=reps)
    best = min(table, key=table.get)
    p, w, h = (int(x) for x in best.split(","))
    rt.set_option(rt.OPT_BATCH_SEEDS_PER_WARP, p)
    rt.set_option(rt.OPT_BATCH_WARPS, w)
    rt.set_option(rt.OPT_BATCH_SMEM_HITS, h)
    res = {"seeds_per_warp": p, "warps": w, "smem_hits": h, "ms": table[best], "table_ms": table}
    _store(_key("batched_search", {"E": E, "S": S, "H": int(hits.shape[0]), "model": model}), res)
    return res
