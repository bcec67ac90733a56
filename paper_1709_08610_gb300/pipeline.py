"""Batched track finding over a ragged batch of events, replayable as one CUDA graph.

One step is Algorithm 1 end to end on every event of the batch:
spatial ordering of the hits (retina_prepare_hits), the starting points -
either given (a uniform draw from the prior P_theta) or proposed by the
learned seed network (slope histogram -> network -> ranked cells -> seeds
at the hit means of their dense sub-cells) -
the q truncated-Newton updates of all seeds in one persistent launch
(retina_batched_search), then cluster + select (retina_extract_tracks).

Every buffer is allocated once for a fixed capacity (events, hits, seeds per
event), so ``capture`` can record the whole step in a CUDA graph and
``replay`` re-runs it on new inputs copied into ``hits`` / ``offsets``
(events may change size as long as the total fits the hit capacity).
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from . import retina as rt
from .seednet import SeedProposer


class BatchTracker:
    def __init__(self, n_events: int, hit_capacity: int, seeds_per_event: int, box: "rt.Grid", opts: "rt.LsOpts",
                 R0: float, merge_cells: float = 2.0, max_tracks: int = 1024,
                 proposer: Optional[SeedProposer] = None, model: int = rt.VELO_SLOPES,
                 sort_seeds: bool = False, seeds_per_warp: Optional[int] = None, warps: Optional[int] = None,
                 smem_hits: Optional[int] = None, device="cuda"):
        """sort_seeds orders each event's starting points spatially before the
        search (retina_sort_seeds); seeds_per_warp, warps and smem_hits set the
        search's RETINA_OPT_BATCH_SEEDS_PER_WARP / _WARPS / _SMEM_HITS for this
        tracker's launches (the options are process-wide; the tracker restores
        them after each launch)."""
        E, H, n = int(n_events), int(hit_capacity), int(seeds_per_event)
        if proposer is not None and model != rt.VELO_SLOPES:
            raise ValueError("the learned proposer works on slope-model hits")
        self.E, self.H, self.n = E, H, n
        self.box, self.opts, self.R0, self.merge = box, opts, float(R0), float(merge_cells)
        self.model, self.proposer, self.K = model, proposer, int(max_tracks)
        dev = torch.device(device)
        f32 = dict(dtype=torch.float32, device=dev)
        self.hits = torch.zeros((H, 4), **f32)
        self.offsets = torch.zeros(E + 1, dtype=torch.int64, device=dev)
        self.sorted = torch.empty((H, 4), **f32)
        self.boxes = torch.empty((int(rt.lib.retina_prepare_hits_box_count(H, E)), 8), **f32)
        self.seeds = torch.zeros((E, n, 2), **f32)
        self.sort, self.spw, self.warps, self.smem_hits = bool(sort_seeds), seeds_per_warp, warps, smem_hits
        self.seeds_sorted = torch.zeros((E * n, 2), **f32) if self.sort else None
        self.seed_offsets = torch.arange(E + 1, dtype=torch.int64, device=dev) * n
        self.search_out = (torch.empty((E * n, 2), **f32), torch.empty((E * n,), **f32),
                           torch.empty((E * n,), dtype=torch.uint8, device=dev))
        self.ws = torch.empty(max(rt.batched_search_workspace_size(E), 256), dtype=torch.uint8, device=dev)
        self.tracks = dict(tracks=torch.empty((E, self.K, 2), **f32), track_R=torch.empty((E, self.K), **f32),
                           track_src=torch.empty((E, self.K), dtype=torch.int32, device=dev),
                           n_tracks=torch.empty((E,), dtype=torch.int32, device=dev))
        self.graph: Optional[torch.cuda.CUDAGraph] = None

    def load(self, hits: np.ndarray, offsets: np.ndarray, seeds: Optional[np.ndarray] = None):
        """Copy a batch (host arrays) into the device buffers."""
        if hits.shape[0] > self.H or offsets.shape[0] != self.E + 1:
            raise ValueError("batch does not fit the tracker's capacity")
        self.hits[:hits.shape[0]].copy_(torch.from_numpy(np.ascontiguousarray(hits, dtype=np.float32)))
        self.offsets.copy_(torch.from_numpy(np.ascontiguousarray(offsets, dtype=np.int64)))
        if seeds is not None:
            self.seeds.copy_(torch.from_numpy(np.ascontiguousarray(seeds, dtype=np.float32)).reshape(self.seeds.shape))

    def step(self, stream=None, marks=None):
        """Launch the whole step on the current (or given) stream.  ``marks``: two
        CUDA events, recorded on that stream just before and just after the
        search launch (eager steps only)."""
        rt.prepare_hits(self.hits, self.offsets, self.model, out=(self.sorted, self.boxes), stream=stream)
        if self.proposer is not None:
            self.proposer.propose(self.hits, self.offsets, self.n, seeds=self.seeds, stream=stream)
        seeds = self.seeds.reshape(-1, 2)
        if self.sort:
            rt.sort_seeds(seeds, self.seed_offsets, self.box, out=self.seeds_sorted, stream=stream)
            seeds = self.seeds_sorted
        shape = [(o, v) for o, v in ((rt.OPT_BATCH_SEEDS_PER_WARP, self.spw), (rt.OPT_BATCH_WARPS, self.warps),
                                     (rt.OPT_BATCH_SMEM_HITS, self.smem_hits)) if v]
        old = [(o, rt.get_option(o)) for o, _ in shape]
        for o, v in shape:
            rt.set_option(o, v)
        st = stream if stream is not None else torch.cuda.current_stream()
        try:
            if marks:
                marks[0].record(st)
            rt.batched_search(self.sorted, self.offsets, self.model, seeds, self.seed_offsets, self.opts, self.box,
                              out=self.search_out, ws=self.ws, boxes=self.boxes, stream=stream)
            if marks:
                marks[1].record(st)
        finally:
            for o, v in old:
                rt.set_option(o, v)
        th, R, st = self.search_out
        rt.extract_tracks(th.reshape(self.E, self.n, 2), R.reshape(self.E, self.n), st.reshape(self.E, self.n),
                          self.box, self.R0, self.merge, self.K, out=self.tracks, stream=stream)

    def capture(self):
        """Record one step in a CUDA graph (after one eager warm-up step)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step()
        return self.graph

    def replay(self):
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()

    def results(self):
        """Per event: float64 [n_tracks, 2] track parameters (host)."""
        n = self.tracks["n_tracks"].cpu().numpy()
        tr = self.tracks["tracks"].cpu().numpy()
        return [tr[e, :min(int(n[e]), self.K)].astype(np.float64) for e in range(self.E)]


class GridScanBatch:
    """The plain grid method over a batch: spatial ordering, Eq. 2 on the grid,
    strict local maxima above R0, optionally the refinement of each maximum
    (step 4: ``refine_iters`` truncated-Newton updates at the grid's
    bandwidth, each capped to ``refine_cap_cells``), cluster + select;
    graph-capturable like BatchTracker (the response grids live in the
    workspace)."""

    def __init__(self, n_events: int, hit_capacity: int, grid: "rt.Grid", sigma: float, R0: float,
                 merge_cells: float = 2.0, max_maxima: int = 4096, max_tracks: int = 1024,
                 model: int = rt.VELO_SLOPES, refine_iters: int = 0, refine_cap_cells: float = 1.0,
                 device="cuda"):
        E, H = int(n_events), int(hit_capacity)
        self.E, self.H, self.grid, self.sigma, self.R0, self.merge = E, H, grid, float(sigma), float(R0), float(merge_cells)
        self.model, self.Km, self.K = model, int(max_maxima), int(max_tracks)
        self.ropts = rt.refine_opts(self.sigma, refine_iters, refine_cap_cells) if refine_iters > 0 else None
        dev = torch.device(device)
        f32 = dict(dtype=torch.float32, device=dev)
        self.hits = torch.zeros((H, 4), **f32)
        self.offsets = torch.zeros(E + 1, dtype=torch.int64, device=dev)
        self.sorted = torch.empty((H, 4), **f32)
        self.boxes = torch.empty((int(rt.lib.retina_prepare_hits_box_count(H, E)), 8), **f32)
        self.maxima = dict(max_idx=torch.empty((E, self.Km), dtype=torch.int32, device=dev),
                           max_theta=torch.empty((E, self.Km, 2), **f32), max_R=torch.empty((E, self.Km), **f32),
                           n_max=torch.empty((E,), dtype=torch.int32, device=dev), R=None)
        self.ws = torch.empty(max(rt.grid_scan_workspace_size(E, model, grid), 1), dtype=torch.uint8, device=dev)
        self.refined = None if self.ropts is None else (
            torch.empty((E, self.Km, 2), **f32), torch.empty((E, self.Km), **f32),
            torch.empty((E, self.Km), dtype=torch.uint8, device=dev))
        self.refine_ws = None if self.ropts is None else \
            torch.empty(max(rt.refine_maxima_workspace_size(E), 256), dtype=torch.uint8, device=dev)
        self.tracks = dict(tracks=torch.empty((E, self.K, 2), **f32), track_R=torch.empty((E, self.K), **f32),
                           track_src=torch.empty((E, self.K), dtype=torch.int32, device=dev),
                           n_tracks=torch.empty((E,), dtype=torch.int32, device=dev))
        self.graph: Optional[torch.cuda.CUDAGraph] = None

    load = BatchTracker.load

    def step(self, stream=None):
        rt.prepare_hits(self.hits, self.offsets, self.model, out=(self.sorted, self.boxes), stream=stream)
        rt.grid_scan(self.sorted, self.offsets, self.model, self.grid, self.sigma, self.R0, self.Km, ws=self.ws,
                     out=self.maxima, boxes=self.boxes, stream=stream)
        m = self.maxima
        if self.ropts is None:
            th, R, st = m["max_theta"], m["max_R"], None
        else:
            # 32-warp CTAs: ~22 % faster than the default 16 on 1024-event batches
            # (~160 maxima per event), the same on one event
            old = rt.get_option(rt.OPT_BATCH_WARPS)
            rt.set_option(rt.OPT_BATCH_WARPS, 32)
            try:
                th, R, st = rt.refine_maxima(self.sorted, self.offsets, self.model, m["max_theta"], m["n_max"],
                                             self.ropts, self.grid, out=self.refined, ws=self.refine_ws,
                                             boxes=self.boxes, stream=stream)
            finally:
                rt.set_option(rt.OPT_BATCH_WARPS, old)
        rt.extract_tracks(th, R, st, self.grid, self.R0, self.merge, self.K, n_valid=m["n_max"], out=self.tracks,
                          stream=stream)

    capture = BatchTracker.capture
    replay = BatchTracker.replay
    results = BatchTracker.results


class Search4Batch:
    """Tracks with the four-parameter model (x0, y0, t_x, t_y) at z_ref over a
    batch: starting points from hit pairs on given layer pairs
    (retina_pair_seeds4), the four-parameter search from each
    (retina_local_search4 with the per-event seed counts), cluster / select in
    four dimensions (retina_extract_tracks4).  No host synchronisation
    between the launches, so ``capture`` records the step as one CUDA graph."""

    def __init__(self, n_events: int, hit_capacity: int, slope_box: "rt.Grid", opts: "rt.LsOpts4", R0: float,
                 layer_pairs, dz_tol: float, d_max: float, zc_range, max_seeds: int = 2048,
                 merge_units: float = 2.0, max_tracks: int = 1024, device="cuda"):
        E, H = int(n_events), int(hit_capacity)
        self.E, self.H, self.K, self.S = E, H, int(max_tracks), int(max_seeds)
        self.box, self.opts, self.R0, self.merge = slope_box, opts, float(R0), float(merge_units)
        self.pairs, self.cuts = list(layer_pairs), dict(dz_tol=dz_tol, d_max=d_max, zc_range=tuple(zc_range),
                                                         zref=opts.zref)
        dev = torch.device(device)
        f32 = dict(dtype=torch.float32, device=dev)
        self.hits = torch.zeros((H, 4), **f32)
        self.offsets = torch.zeros(E + 1, dtype=torch.int64, device=dev)
        self.seeds = (torch.empty((E, self.S, 4), **f32), torch.empty((E,), dtype=torch.int32, device=dev))
        self.search_out = (torch.empty((E, self.S, 4), **f32), torch.empty((E, self.S), **f32),
                           torch.empty((E, self.S), dtype=torch.uint8, device=dev))
        self.tracks = dict(tracks=torch.empty((E, self.K, 4), **f32), track_R=torch.empty((E, self.K), **f32),
                           track_src=torch.empty((E, self.K), dtype=torch.int32, device=dev),
                           n_tracks=torch.empty((E,), dtype=torch.int32, device=dev))
        self.graph: Optional[torch.cuda.CUDAGraph] = None

    load = BatchTracker.load

    def step(self, stream=None):
        rt.pair_seeds4(self.hits, self.offsets, self.pairs, K=self.S, out=self.seeds, stream=stream, **self.cuts)
        rt.local_search4(self.hits, self.offsets, self.seeds[0], self.opts, out=self.search_out, stream=stream,
                         seed_count=self.seeds[1])
        th, R, st = self.search_out
        rt.extract_tracks4(th, R, st, self.box, self.opts.scale, self.R0, self.merge, self.K, n_valid=self.seeds[1],
                           out=self.tracks, stream=stream)

    capture = BatchTracker.capture
    replay = BatchTracker.replay

    def results(self):
        """Per event: float64 [n_tracks, 4] track parameters (host)."""
        n = self.tracks["n_tracks"].cpu().numpy()
        tr = self.tracks["tracks"].cpu().numpy()
        return [tr[e, :min(int(n[e]), self.K)].astype(np.float64) for e in range(self.E)]


def match_efficiency(found, truth, eps: float = 1e-3):
    """Fraction of truth tracks with a found track within eps (max norm) and
    the number of found tracks matching none (fakes)."""
    n_truth = n_hit = n_fake = 0
    for f, t in zip(found, truth):
        t = np.asarray(t, dtype=np.float64).reshape(-1, 2)
        f = np.asarray(f, dtype=np.float64).reshape(-1, 2)
        n_truth += len(t)
        if len(f) == 0 or len(t) == 0:
            n_fake += len(f)
            continue
        d = np.abs(f[:, None, :] - t[None, :, :]).max(-1)
        n_hit += int((d <= eps).any(0).sum())
        n_fake += int((~(d <= eps).any(1)).sum())
    return (n_hit / max(n_truth, 1)), n_fake


def match_residuals(found, truth, eps: float = 1e-3) -> np.ndarray:
    """|found - truth| per axis [n, 2] of every truth track's nearest found
    track (max norm), for the truth tracks matched within eps."""
    out = []
    for f, t in zip(found, truth):
        t = np.asarray(t, dtype=np.float64).reshape(-1, 2)
        f = np.asarray(f, dtype=np.float64).reshape(-1, 2)
        if len(f) == 0 or len(t) == 0:
            continue
        d = np.abs(f[:, None, :] - t[None, :, :])
        j = d.max(-1).argmin(0)
        near = d[j, np.arange(len(t))]
        out.append(near[near.max(-1) <= eps])
    return np.concatenate(out) if out else np.zeros((0, 2))


def efficiency_by_multiplicity(found, truth, edges, eps: float = 1e-3) -> dict:
    """MC efficiency over the events whose number of truth tracks lies in
    [edges[i], edges[i+1]), keyed "lo-hi" (the shape of the paper's Fig. 3:
    efficiency against the number of reconstructible tracks)."""
    out = {}
    n = np.array([len(np.asarray(t).reshape(-1, 2)) for t in truth])
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = [i for i in range(len(truth)) if lo <= n[i] < hi]
        if sel:
            eff, _ = match_efficiency([found[i] for i in sel], [truth[i] for i in sel], eps)
            out["%d-%d" % (lo, hi)] = {"events": len(sel), "efficiency": eff}
    return out


def recovered_fraction(found, reference, eps: float = 1e-3):
    """Fraction of the reference method's tracks that ``found`` also has (within eps)."""
    eff, _ = match_efficiency(found, reference, eps)
    return eff
