"""Refinement of grid maxima (step 4 of the grid algorithm) on the GPU vs the
FP64 oracle, through the C ABI.

The starting points are cell centres of maxima the oracle finds (or, at full
size, the cell the oracle places each MC track in); the GPU path refines them
with retina_refine_maxima and the oracle with refine_maxima.  Tolerances as
for the local search: points whose every oracle decision is robust take the
same status, theta within 1e-3 cell at a converged maximum (more only where
the maximum is so ill-conditioned that the FP32 gradient tolerance moves it
further; 0.05 cell elsewhere) and R within its FP32 tolerance.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import WORKLOADS, make_event, make_toy2d_event

pytestmark = pytest.mark.gpu

R_REL, R_ABS = 1e-5, 1e-6
GH_REL = 1e-4
TH_CELLS = 1e-3


@pytest.fixture(scope="module")
def rt():
    from paper_1709_08610_gb300 import build as rbuild
    rbuild.build()
    from paper_1709_08610_gb300 import retina
    return retina


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _window_maxima(wl, ev, i0, i1, n):
    step = np.asarray(wl.grid_step)
    lo = (wl.grid_lo[0] + i0 * step[0], wl.grid_lo[1] + i1 * step[1])
    R = oracle.grid_response(ev.hits, wl.model, lo, step, n, wl.sigma_grid)
    idx = oracle.grid_maxima(R, wl.R0)
    return lo, step, R, idx, oracle.maxima_centres(idx, lo, step, n)


def _check(wl, ev, sigma, step, th_g, R_g, st_g, th_o, R_o, st_o, m_o):
    """Robust points (every oracle decision at least one tolerance from its
    threshold) take the same status.  Where the oracle's point is a converged
    maximum (negative-definite Hessian, Newton distance <= 0.05 cell) theta
    agrees within 1e-3 cell - or, on an ill-conditioned maximum (the toy's
    ridges), within |H^-1| (1e-4 |g|_abs), the displacement the FP32 gradient
    tolerance (1e-4 of the sum of absolute terms) allows there, if larger -
    and R within its FP32 tolerance plus what that theta difference can
    change, whether or not the last Armijo decisions were ties: near the top
    the updates shrink cubically, and a step the FP32 response cannot resolve
    (an increase below ~1e-6 R, a step below ~1.4e-3 of the one-cell peak
    width) is one either side may take or refuse.  Robust points away from a
    maximum agree within 0.05 cell.  Returns the number of converged points."""
    robust = m_o >= 1.0
    assert np.all(st_g[robust] == st_o[robust])
    n_conv = 0
    for i in np.flatnonzero(st_o <= 1):
        o = oracle.rgh(ev.hits, wl.model, th_o[i], sigma)
        H, g = o["hess"], o["grad"]
        conv = False
        try:
            if np.all(np.linalg.eigvalsh(H) < 0):
                Hi = np.linalg.inv(H)
                conv = np.max(np.abs(Hi @ g) / step) <= 0.05
        except np.linalg.LinAlgError:  # numerically singular: a flat ridge, not a converged peak
            conv = False
        if not conv and not robust[i]:
            continue
        n_conv += conv
        if conv:
            d = np.maximum(TH_CELLS * step, np.abs(Hi) @ (GH_REL * o["grad_abs"]))
        else:
            d = 50 * TH_CELLS * step
        assert np.all(np.abs(th_g[i] - th_o[i]) <= d), (i, conv, (th_g[i] - th_o[i]) / step)
        tol = R_REL * R_o[i] + R_ABS + np.abs(g) @ d + np.abs(H).max() * (d @ d)
        assert abs(R_g[i] - R_o[i]) <= tol, (i, R_g[i], R_o[i], tol)
    return n_conv


@pytest.mark.parametrize("with_boxes", [False, True])
def test_refine_matches_oracle_on_windows(rt, with_boxes):
    # three VELO-like windows of 128 x 128 cells around tracks, plus a toy
    # window; maxima padded to K = 96 rows whose tails must stay untouched
    wl = WORKLOADS["velo"]
    cases = []
    for eid in range(3):
        ev = make_event(wl, 11, eid, vertex_sigma=(0, 0, 0))
        tr = ev.truth[eid * 7 % len(ev.truth), :2]
        i0 = int(np.floor((tr[0] - wl.grid_lo[0]) / wl.grid_step[0])) - 64
        i1 = int(np.floor((tr[1] - wl.grid_lo[1]) / wl.grid_step[1])) - 64
        cases.append((wl, ev, i0, i1, (128, 128)))
    tw = WORKLOADS["toy2d"]
    cases.append((tw, make_toy2d_event(11, 0), 0, 0, tw.grid_n))
    K = 96
    n_total = n_conv = 0
    for wl_c, ev, i0, i1, n in cases:
        lo, step, R, idx, c = _window_maxima(wl_c, ev, i0, i1, n)
        assert 1 <= len(idx) <= K
        th_o, R_o, st_o, m_o = oracle.refine_maxima(ev.hits, wl_c.model, c, wl_c.sigma_grid, lo, step, n)
        theta_c = np.full((1, K, 2), np.nan, np.float32)
        theta_c[0, :len(idx)] = c
        box = rt.Grid(lo=tuple(lo), step=tuple(step), n=tuple(n))
        hits = dev(ev.hits)
        off = dev(np.array([0, ev.n_hits], np.int64))
        boxes = None
        if with_boxes:
            sorted_h = torch.empty_like(hits)
            boxes = torch.empty((int(rt.lib.retina_prepare_hits_box_count(ev.n_hits, 1)), 8), dtype=torch.float32,
                                device="cuda")
            rt.prepare_hits(hits, off, wl_c.model, out=(sorted_h, boxes))
            hits = sorted_h
        out = (torch.full((1, K, 2), -7.0, device="cuda"), torch.full((1, K), -7.0, device="cuda"),
               torch.full((1, K), 9, dtype=torch.uint8, device="cuda"))
        rt.refine_maxima(hits, off, wl_c.model, dev(theta_c), dev(np.array([len(idx)], np.int32)),
                         rt.refine_opts(wl_c.sigma_grid), box, out=out, boxes=boxes)
        th_g, R_g, st_g = (t.cpu().numpy()[0] for t in out)
        m = len(idx)
        assert np.all(th_g[m:] == -7.0) and np.all(R_g[m:] == -7.0) and np.all(st_g[m:] == 9)
        n_conv += _check(wl_c, ev, wl_c.sigma_grid, step, th_g[:m].astype(float), R_g[:m].astype(float), st_g[:m],
                         th_o, R_o, st_o, m_o)
        n_total += m
    assert n_conv >= n_total // 2, (n_conv, n_total)


def test_refine_is_bitwise_the_local_search_from_the_same_points(rt):
    wl = WORKLOADS["velo"]
    ev = make_event(wl, 12, 0, vertex_sigma=(0, 0, 0))
    lo, step, R, idx, c = _window_maxima(wl, ev, 384, 384, (256, 256))
    m = len(idx)
    assert m >= 10
    box = rt.Grid(lo=tuple(lo), step=tuple(step), n=(256, 256))
    opts = rt.refine_opts(wl.sigma_grid)
    hits = dev(ev.hits)
    off = dev(np.array([0, ev.n_hits], np.int64))
    th_r, R_r, st_r = rt.refine_maxima(hits, off, 1, dev(c.astype(np.float32)[None]),
                                       dev(np.array([m], np.int32)), opts, box)
    th_s, R_s, st_s = rt.local_search(hits, off, 1, dev(c.astype(np.float32)[None]), opts, box)
    assert torch.equal(th_r, th_s) and torch.equal(R_r, R_s) and torch.equal(st_r, st_s)


def test_refine_ragged_counts_and_edges(rt):
    # counts 3 (event without hits), 5 (7 hits), -3 (read as 0), 40 > K = 32
    # (clipped to K, full event); rows past the count keep their contents
    wl = WORKLOADS["velo"]
    full = make_event(wl, 13, 0, vertex_sigma=(0, 0, 0))
    parts = [full.hits[:0], full.hits[:7], full.hits[:0], full.hits]
    hits = np.concatenate(parts)
    off = np.concatenate([[0], np.cumsum([len(p) for p in parts])]).astype(np.int64)
    K = 32
    rng = np.random.default_rng(3)
    theta_c = (full.truth[rng.integers(0, len(full.truth), (4, K)), :2]
               + rng.normal(0, 0.3, (4, K, 2)) * 2 ** -10).astype(np.float32)
    counts = np.array([3, 5, -3, 40], np.int32)
    box = rt.Grid.of(wl)
    opts = rt.refine_opts(wl.sigma_grid)
    out = (torch.full((4, K, 2), -7.0, device="cuda"), torch.full((4, K), -7.0, device="cuda"),
           torch.full((4, K), 9, dtype=torch.uint8, device="cuda"))
    rt.refine_maxima(dev(hits), dev(off), 1, dev(theta_c), dev(counts), opts, box, out=out)
    th_g, R_g, st_g = (t.cpu().numpy() for t in out)
    live = [3, 5, 0, K]
    step = np.asarray(wl.grid_step)
    for e in range(4):
        n = live[e]
        assert np.all(th_g[e, n:] == -7.0) and np.all(R_g[e, n:] == -7.0) and np.all(st_g[e, n:] == 9)
        if n == 0:
            continue
        th_o, R_o, st_o, m_o = oracle.refine_maxima(parts[e], 1, theta_c[e, :n], wl.sigma_grid, wl.grid_lo,
                                                    wl.grid_step, wl.grid_n)
        if len(parts[e]) == 0:
            # no hits: R = 0 and g = 0 everywhere, so p = 0 and the trial at t = 1
            # passes (0 >= 0): theta stays, status 0, on both sides
            assert np.all(st_o == 0) and np.all(st_g[e, :n] == 0) and np.all(R_g[e, :n] == 0)
            assert np.all(th_g[e, :n] == theta_c[e, :n])
            continue
        ev_e = full if e == 3 else type(full)(full.model, parts[e], full.labels[:len(parts[e])], full.truth)
        _check(wl, ev_e, wl.sigma_grid, step, th_g[e, :n].astype(float), R_g[e, :n].astype(float), st_g[e, :n],
               th_o, R_o, st_o, m_o)
    # zero counts everywhere are a no-op
    rt.refine_maxima(dev(hits), dev(off), 1, dev(theta_c), dev(np.zeros(4, np.int32)), opts, box, out=out)
    assert np.array_equal(out[2].cpu().numpy(), st_g) and np.array_equal(out[0].cpu().numpy(), th_g)


def test_full_size_grid_scan_then_refine_on_truth_cells(rt):
    # the 1024^2 grid scan as the bench runs it, then the refinement of its
    # maxima; the maxima sitting in the cell the oracle places an MC track in
    # are compared with the oracle's refinement from that cell's centre, and
    # every refined point keeps R >= its maximum's R (Armijo).
    wl = WORKLOADS["velo"]
    ev = make_event(wl, 14, 0, vertex_sigma=(0, 0, 0))
    hits = dev(ev.hits)
    off = dev(np.array([0, ev.n_hits], np.int64))
    sorted_h = torch.empty_like(hits)
    boxes = torch.empty((int(rt.lib.retina_prepare_hits_box_count(ev.n_hits, 1)), 8), dtype=torch.float32,
                        device="cuda")
    rt.prepare_hits(hits, off, 1, out=(sorted_h, boxes))
    box = rt.Grid.of(wl)
    K = 4096
    mx = rt.grid_scan(sorted_h, off, 1, box, wl.sigma_grid, wl.R0, K, boxes=boxes)
    th, R, st = rt.refine_maxima(sorted_h, off, 1, mx["max_theta"], mx["n_max"], rt.refine_opts(wl.sigma_grid), box,
                                 boxes=boxes)
    n = int(mx["n_max"].item())
    assert 50 <= n <= K
    idx_g = mx["max_idx"].cpu().numpy()[0, :n]
    R_max = mx["max_R"].cpu().numpy()[0, :n]
    th_g, R_g, st_g = th.cpu().numpy()[0, :n], R.cpu().numpy()[0, :n], st.cpu().numpy()[0, :n]
    assert np.all(R_g[st_g <= 1] >= R_max[st_g <= 1] * (1 - 1e-5))
    step = np.asarray(wl.grid_step)
    cell = np.floor((ev.truth[:, :2] - np.asarray(wl.grid_lo)) / step).astype(np.int64)
    tidx = cell[:, 1] * wl.grid_n[0] + cell[:, 0]
    pos = {int(v): k for k, v in enumerate(idx_g)}
    hit = [(t, pos[int(v)]) for t, v in enumerate(tidx) if int(v) in pos]
    assert len(hit) >= len(tidx) // 3, (len(hit), len(tidx))
    c = oracle.maxima_centres(tidx[[t for t, _ in hit]], wl.grid_lo, step, wl.grid_n)
    th_o, R_o, st_o, m_o = oracle.refine_maxima(ev.hits, 1, c, wl.sigma_grid, wl.grid_lo, step, wl.grid_n)
    k = np.array([g for _, g in hit])
    n_conv = _check(wl, ev, wl.sigma_grid, step, th_g[k].astype(float), R_g[k].astype(float), st_g[k],
                    th_o, R_o, st_o, m_o)
    assert n_conv >= len(hit) // 2
    # refined estimates sit closer to the MC tracks than the cell centres
    t = ev.truth[[t for t, _ in hit], :2]
    assert np.median(np.abs(th_g[k] - t).max(1)) < 0.5 * np.median(np.abs(c - t).max(1))


def test_grid_batch_with_refinement_replays_and_equals_separate_calls(rt):
    from paper_1709_08610_gb300.pipeline import GridScanBatch
    from synth import batch_of
    wl = WORKLOADS["velo_batch"]
    evs = [make_event(wl, 15, e, vertex_sigma=(0, 0, 0)) for e in range(6)]
    b = batch_of(evs)
    box = rt.Grid.of(wl)
    gb = GridScanBatch(6, b.hits.shape[0], box, wl.sigma_grid, wl.R0, refine_iters=4)
    gb.load(b.hits, b.offsets)
    gb.capture()
    gb.replay()
    torch.cuda.synchronize()
    got = gb.results()
    # the same steps as separate calls
    hits, off = dev(b.hits), dev(b.offsets)
    sorted_h = torch.empty_like(hits)
    boxes = torch.empty_like(gb.boxes)
    rt.prepare_hits(hits, off, 1, out=(sorted_h, boxes))
    mx = rt.grid_scan(sorted_h, off, 1, box, wl.sigma_grid, wl.R0, gb.Km, boxes=boxes)
    th, R, st = rt.refine_maxima(sorted_h, off, 1, mx["max_theta"], mx["n_max"], rt.refine_opts(wl.sigma_grid), box,
                                 boxes=boxes)
    tr = rt.extract_tracks(th, R, st, box, wl.R0, 2.0, gb.K, n_valid=mx["n_max"])
    n = tr["n_tracks"].cpu().numpy()
    for e in range(6):
        assert np.array_equal(got[e], tr["tracks"].cpu().numpy()[e, :n[e]].astype(np.float64))
    # and the refined tracks are nearer the MC truth than the unrefined grid's
    plain = GridScanBatch(6, b.hits.shape[0], box, wl.sigma_grid, wl.R0)
    plain.load(b.hits, b.offsets)
    plain.step()
    torch.cuda.synchronize()
    base = plain.results()

    def resid(found):
        out = []
        for f, ev in zip(found, evs):
            d = np.abs(f[:, None, :] - ev.truth[None, :, :2]).max(-1)
            out.extend(d.min(0)[d.min(0) <= 1e-3])
        return np.median(out)

    assert resid(got) < 0.5 * resid(base)
