"""The batched path (one persistent search launch over a ragged batch, the
batched grid scan) at the sizes of the batched workloads, on subsets of their
events, against the FP64 oracle event by event:

* 1024-event VELO-like batch (tracks ~ Poisson(150), smeared vertex): 4
  events, 4096 uniform seeds each through BatchTracker in the throughput
  shape (spatially sorted seeds, four per warp, 32-warp CTAs) - found-track
  sets equal up to near-ties; the whole 1024^2 grid of each event through
  GridScanBatch - maxima and tracks equal up to near-ties;
* high-multiplicity batch (Poisson(600) tracks, ~16.8k hits: more hits than
  a CTA stages): 4 events, 2048 uniform seeds each - found-track sets; the
  2048^2 grid's maxima on windows around found tracks.
"""
import numpy as np
import pytest
import torch

import oracle
from parity_rules import R_ABS, R_REL, candidates, compare_track_sets, search_tolerance
from synth import WORKLOADS, batch_of, make_event, uniform_seeds
from test_gpu_parity import _converged_2d, _grid_sets

pytestmark = pytest.mark.gpu
RUN_SEED = 41


@pytest.fixture(scope="module")
def rt():
    from paper_1709_08610_gb300 import build as rbuild
    rbuild.build()
    from paper_1709_08610_gb300 import retina
    return retina


def _batched_search_sets(rt, wl, evs, n_seeds):
    from paper_1709_08610_gb300.pipeline import BatchTracker
    E = len(evs)
    b = batch_of(evs)
    box = rt.Grid.of(wl)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    tr = BatchTracker(E, b.hits.shape[0], n_seeds, box, opts, wl.R0, max_tracks=4096, sort_seeds=True,
                      seeds_per_warp=4, warps=32, smem_hits=12288)
    seeds = np.stack([uniform_seeds(wl, n_seeds, RUN_SEED, e) for e in range(E)])
    tr.load(b.hits, b.offsets, seeds)
    tr.step()
    torch.cuda.synchronize()
    th_all, R_all, st_all = (x.cpu().numpy() for x in tr.search_out)
    sorted_seeds = tr.seeds_sorted.cpu().numpy().reshape(E, n_seeds, 2)
    n_tr = tr.tracks["n_tracks"].cpu().numpy()
    src_all = tr.tracks["track_src"].cpu().numpy()
    R0 = float(np.float32(wl.R0))
    boxa = (wl.grid_lo, wl.grid_step, wl.grid_n)
    compared = 0
    for e, ev in enumerate(evs):
        sl = slice(e * n_seeds, (e + 1) * n_seeds)
        th_g, R_g, st_g = th_all[sl].astype(float), R_all[sl].astype(float), st_all[sl]
        seeds_e = sorted_seeds[e].astype(np.float32)
        # the sort permutes each event's seeds; the oracle runs on the same order

        def run(pt):
            return oracle.local_search(ev.hits, 1, seeds_e, wl.sigma_schedule, *boxa, perturb=pt)

        th_o, R_o, st_o, m_o = base = run(None)
        keep_o = oracle.extract_tracks(th_o, R_o, st_o, *boxa, R0, wl.merge_cells)
        cand_o = candidates(th_o, R_o, st_o, *boxa, R0)
        cand_g = candidates(th_g, R_g, st_g, *boxa, R0)
        tol = search_tolerance(_converged_2d(ev, wl), th_o, cand_o | cand_g, wl.grid_step)
        stable, _, _ = oracle.path_conditioning(run, base, tol, keys=oracle.PERTURB_KEYS[:8])
        tie = (m_o < 1.0) | ~stable
        near0 = np.abs(R_o - R0) <= R_REL * np.abs(R_o) + R_ABS
        _, _, k = compare_track_sets(th_o, R_o, cand_o | (near0 & (st_o <= 1)), th_g, R_g, cand_g, tie, keep_o,
                                     src_all[e, :n_tr[e]], tol, wl.grid_step, wl.merge_cells, R0=R0)
        compared += k
    return compared


def test_batch_of_1024_event_workload_search_track_sets(rt):
    wl = WORKLOADS["velo_batch"]
    evs = [make_event(wl, RUN_SEED, e) for e in range(4)]
    # the smeared vertex leaves the slope model few tracks; the origin-vertex
    # variant of the same events gives many
    evs += [make_event(wl, RUN_SEED, e, vertex_sigma=(0, 0, 0)) for e in range(4, 8)]
    compared = _batched_search_sets(rt, wl, evs, 4096)
    assert compared >= 100, compared


def test_batch_of_1024_event_workload_grid_track_sets(rt):
    from paper_1709_08610_gb300.pipeline import GridScanBatch
    wl = WORKLOADS["velo_batch"]
    evs = [make_event(wl, RUN_SEED, e) for e in range(4)]
    b = batch_of(evs)
    gs = GridScanBatch(len(evs), b.hits.shape[0], rt.Grid.of(wl), wl.sigma_grid, wl.R0, max_maxima=8192,
                       max_tracks=4096)
    gs.load(b.hits, b.offsets)
    gs.step()
    # the response grids themselves, from the batch's ordered hits
    out = rt.grid_scan(gs.sorted, gs.offsets, 1, gs.grid, gs.sigma, gs.R0, 8192, store_R=True, boxes=gs.boxes)
    torch.cuda.synchronize()
    # the batch's own maxima are the grid scan's (the first n_max slots of each event)
    assert torch.equal(out["n_max"], gs.maxima["n_max"])
    for e in range(len(evs)):
        n = int(out["n_max"][e])
        assert torch.equal(out["max_idx"][e, :n], gs.maxima["max_idx"][e, :n])
    tr = gs.tracks
    R_o = [oracle.grid_response(ev.hits, 1, wl.grid_lo, wl.grid_step, wl.grid_n, wl.sigma_grid) for ev in evs]
    compared = _grid_sets(rt, wl, evs, out["R"].cpu().numpy(), out, tr, R_o)
    assert compared >= 60, compared


def test_high_multiplicity_batch_search_track_sets(rt):
    wl = WORKLOADS["velo_stress"]
    evs = [make_event(wl, RUN_SEED, e, vertex_sigma=(0, 0, 0)) for e in range(4)]
    assert min(ev.n_hits for ev in evs) > 12288  # beyond what a CTA stages
    compared = _batched_search_sets(rt, wl, evs, 2048)
    assert compared >= 40, compared


def test_high_multiplicity_batch_grid_maxima_on_windows(rt):
    # 2048^2 grids of 4 events; the oracle evaluates 96 x 96 windows around
    # tracks and the maxima strictly inside each window (whose 3 x 3
    # neighbourhood lies in the window) are compared up to near-ties
    wl = WORKLOADS["velo_stress"]
    evs = [make_event(wl, RUN_SEED, e, vertex_sigma=(0, 0, 0)) for e in range(4)]
    b = batch_of(evs)
    hits, offs = torch.from_numpy(b.hits).cuda(), torch.from_numpy(b.offsets).cuda()
    srt, boxes = rt.prepare_hits(hits, offs, 1)
    grid = rt.Grid.of(wl)
    out = rt.grid_scan(srt, offs, 1, grid, wl.sigma_grid, wl.R0, 8192, store_R=True, boxes=boxes)
    R_g = out["R"].cpu().numpy()
    n0, n1 = wl.grid_n
    W = 96
    rng = np.random.default_rng(3)
    checked = 0
    for e, ev in enumerate(evs):
        nm = int(out["n_max"][e])
        got = set(out["max_idx"][e, :nm].cpu().numpy().tolist())
        centres = ev.truth[rng.choice(len(ev.truth), 3, replace=False), :2]
        for c in centres:
            i0 = int(np.clip(np.floor((c[0] - wl.grid_lo[0]) / wl.grid_step[0]) - W // 2, 0, n0 - W))
            i1 = int(np.clip(np.floor((c[1] - wl.grid_lo[1]) / wl.grid_step[1]) - W // 2, 0, n1 - W))
            lo = (wl.grid_lo[0] + i0 * wl.grid_step[0], wl.grid_lo[1] + i1 * wl.grid_step[1])
            R_o = oracle.grid_response(ev.hits, 1, lo, wl.grid_step, (W, W), wl.sigma_grid)
            Rg_w = R_g[e, i1:i1 + W, i0:i0 + W].astype(np.float64)
            tol = R_REL * R_o + R_ABS
            assert np.all(np.abs(Rg_w - R_o) <= tol)
            exp, _, margin = oracle.grid_maxima(R_o, wl.R0, with_margin=True)
            inner = lambda k: 0 < k % W < W - 1 and 0 < k // W < W - 1
            exp_in = {k for k in exp.tolist() if inner(k)}
            got_in = set()
            for k in range(W * W):
                if inner(k) and ((i1 + k // W) * n0 + i0 + k % W) in got:
                    got_in.add(k)
            for k in exp_in ^ got_in:
                assert margin.reshape(-1)[k] <= 2 * tol.reshape(-1)[k], (e, k)
            checked += len(exp_in)
    assert checked >= 12, checked
