"""Exact block skipping (retina_prepare_hits boxes) on the GPU.

A block of 32 hits is skipped only when every one of its terms of Eq. 1 is
exactly zero in float32, so with boxes every kernel must return bitwise what
it returns without boxes on the same (spatially ordered) hits; the prepared
hits must be a permutation of each event's hits, and each box must bound its
block.
"""
import numpy as np
import pytest
import torch

import oracle
from hit_order import documented_order
from synth import WORKLOADS, make_event, batch_of, uniform_seeds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    from paper_1709_08610_gb300 import build as rbuild
    rbuild.build()
    from paper_1709_08610_gb300 import retina
    return retina


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _batch(model):
    if model == 1:
        wl = WORKLOADS["velo"]
        evs = [make_event(wl, 4, 0, vertex_sigma=(0, 0, 0)), make_event(wl, 4, 1, n_tracks=0, noise_frac=0.0),
               make_event(wl, 4, 2, n_tracks=700, vertex_sigma=(0, 0, 0)),  # > 16384 hits: two sort chunks
               make_event(wl, 4, 3, n_tracks=20)]
    else:
        wl = WORKLOADS["toy2d"]
        evs = [make_event(wl, 4, e) for e in range(3)]
    return wl, evs, batch_of(evs)


@pytest.mark.parametrize("model", [0, 1])
def test_prepared_hits_are_a_permutation_with_bounding_boxes(rt, model):
    wl, evs, b = _batch(model)
    srt, boxes = rt.prepare_hits(_dev(b.hits), _dev(b.offsets), model)
    srt, boxes = srt.cpu().numpy(), boxes.cpu().numpy()
    for e in range(len(evs)):
        h0, h1 = b.offsets[e], b.offsets[e + 1]
        a = b.hits[h0:h1]
        s = srt[h0:h1]
        assert np.array_equal(a[np.lexsort(a.T[::-1])], s[np.lexsort(s.T[::-1])])
        base = h0 // 32 + e
        for k in range(0, h1 - h0, 32):
            blk = s[k:k + 32].astype(np.float32)
            bx = boxes[base + k // 32]
            if model == 1:  # slopes (float32 division) and |z|
                u, v, w = blk[:, 0] / blk[:, 2], blk[:, 1] / blk[:, 2], np.abs(blk[:, 2])
            else:
                u, v, w = blk[:, 0], blk[:, 1], np.zeros(len(blk), np.float32)
            assert bx[0] == u.min() and bx[1] == u.max()
            assert bx[2] == v.min() and bx[3] == v.max()
            assert bx[4] == w.min() and bx[5] == w.max()
        if model == 1 and h1 - h0 > 1000:
            # blocks are spatially coherent: slope boxes of layers |z| >= 64 mm are small
            bx = boxes[base:base + (h1 - h0) // 32]
            far = bx[:, 4] >= 64
            side = np.sqrt((bx[far, 1] - bx[far, 0]) * (bx[far, 3] - bx[far, 2]))
            assert np.median(side) <= 0.3, np.median(side)


def test_batch_ordering_is_bitwise_the_per_event_ordering(rt):
    # a batch that fills the GPU many times over is ordered one CTA per event,
    # a single event by a cluster of CTAs: the same keys and total order, so
    # the same sorted hits and boxes, bit for bit (events with two sort chunks
    # and an empty one included)
    wl = WORKLOADS["velo_batch"]
    evs = [make_event(wl, 5, e, vertex_sigma=(0, 0, 0)) for e in range(120)]
    evs[7] = make_event(WORKLOADS["velo"], 5, 7, n_tracks=700, vertex_sigma=(0, 0, 0))
    evs[11] = make_event(WORKLOADS["velo"], 5, 11, n_tracks=0, noise_frac=0.0)
    b = batch_of(evs)
    assert len(evs) * 8 > 4 * torch.cuda.get_device_properties(0).multi_processor_count
    srt, boxes = rt.prepare_hits(_dev(b.hits), _dev(b.offsets), 1)
    srt, boxes = srt.cpu().numpy(), boxes.cpu().numpy()
    for e in (0, 7, 11, 63, 119):
        h0, h1 = b.offsets[e], b.offsets[e + 1]
        s1, b1 = rt.prepare_hits(_dev(b.hits[h0:h1]), _dev(np.array([0, h1 - h0], np.int64)), 1)
        np.testing.assert_array_equal(srt[h0:h1], s1.cpu().numpy())
        nb = (h1 - h0 + 31) // 32
        np.testing.assert_array_equal(boxes[h0 // 32 + e:h0 // 32 + e + nb], b1.cpu().numpy()[:nb])


@pytest.mark.parametrize("flags", [1, 2, 3])
def test_grid_response_with_boxes_is_bitwise_the_full_sum(rt, flags):
    wl, evs, b = _batch(1)
    srt, boxes = rt.prepare_hits(_dev(b.hits), _dev(b.offsets), 1)
    offs = _dev(b.offsets)
    grid = rt.Grid.of(wl) if flags == 2 else rt.Grid((-0.25, -0.2), wl.grid_step, (320, 300))
    R_full = rt.grid_response(srt, offs, 1, grid, wl.sigma_grid, flags=flags)
    R_cull = rt.grid_response(srt, offs, 1, grid, wl.sigma_grid, flags=flags, boxes=boxes)
    assert torch.equal(R_full, R_cull)
    # and the culled grid still matches the oracle on sampled cells
    R = R_cull.cpu().numpy()
    rng = np.random.default_rng(0)
    c0, c1 = oracle.cell_centres(grid.lo, grid.step, grid.n)
    for e in (0, 2):
        idx = np.concatenate([rng.integers(0, R[e].size, 400), np.argsort(R[e].reshape(-1))[-100:]])
        th = np.stack([c0[idx % grid.n[0]], c1[idx // grid.n[0]]], 1)
        R_o = oracle.response(evs[e].hits, 1, th, wl.sigma_grid)
        assert np.all(np.abs(R[e].reshape(-1)[idx] - R_o) <= 1e-5 * R_o + 1e-6)


def test_grid_response_toy_with_boxes_is_bitwise_the_full_sum(rt):
    wl, evs, b = _batch(0)
    srt, boxes = rt.prepare_hits(_dev(b.hits), _dev(b.offsets), 0)
    offs = _dev(b.offsets)
    grid = rt.Grid.of(wl)
    for sigma in (wl.sigma_grid, 0.004):
        R_full = rt.grid_response(srt, offs, 0, grid, sigma)
        R_cull = rt.grid_response(srt, offs, 0, grid, sigma, boxes=boxes)
        assert torch.equal(R_full, R_cull)


@pytest.mark.parametrize("model", [0, 1])
def test_searches_with_boxes_are_bitwise_the_full_search(rt, model):
    wl, evs, b = _batch(model)
    srt, boxes = rt.prepare_hits(_dev(b.hits), _dev(b.offsets), model)
    offs = _dev(b.offsets)
    n = 300
    per = []
    for e, ev in enumerate(evs):  # per event: half uniform seeds, half on true tracks
        uni = uniform_seeds(wl, n // 2, 4, e)
        near = (ev.truth[:, :2][np.arange(n // 2) % len(ev.truth)] if len(ev.truth) else uniform_seeds(wl, n // 2, 5, e))
        per.append(np.concatenate([uni, near.astype(np.float32)]))
    S = np.stack(per).astype(np.float32)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    box = rt.Grid.of(wl)
    full = rt.local_search(srt, offs, model, _dev(S), opts, box)
    cull = rt.local_search(srt, offs, model, _dev(S), opts, box, boxes=boxes)
    for x, y in zip(full, cull):
        assert torch.equal(x, y)
    so = _dev(np.arange(len(evs) + 1, dtype=np.int64) * n)
    bfull = rt.batched_search(srt, offs, model, _dev(S.reshape(-1, 2)), so, opts, box)
    bcull = rt.batched_search(srt, offs, model, _dev(S.reshape(-1, 2)), so, opts, box, boxes=boxes)
    for x, y, z in zip(bfull, bcull, full):
        assert torch.equal(x, y)
        assert torch.equal(x.reshape(z.shape), z)


def test_non_finite_hit_blocks_are_never_skipped(rt):
    wl = WORKLOADS["velo"]
    ev = make_event(wl, 6, 0, vertex_sigma=(0, 0, 0))
    hits = ev.hits.copy()
    hits[17, 0] = np.nan
    offs = _dev(np.array([0, len(hits)], np.int64))
    srt, boxes = rt.prepare_hits(_dev(hits), offs, 1)
    grid = rt.Grid((-0.1, -0.1), wl.grid_step, (64, 64))
    R_full = rt.grid_response(srt, offs, 1, grid, wl.sigma_grid, flags=1)
    R_cull = rt.grid_response(srt, offs, 1, grid, wl.sigma_grid, flags=1, boxes=boxes)
    assert torch.isnan(R_full).all() and torch.isnan(R_cull).all()


def _order_events():
    wl = WORKLOADS["velo"]
    rng = np.random.default_rng(17)
    one_band = np.zeros((20000, 4), np.float32)  # one band, three sorted chunks merged
    one_band[:, 2] = rng.uniform(256, 511, 20000)
    one_band[:, :2] = rng.uniform(-0.4, 0.4, (20000, 2)) * one_band[:, 2:3]
    odd = make_event(wl, 9, 3, n_tracks=300, vertex_sigma=(0, 0, 0)).hits.copy()
    odd[5, 2] = 0.0  # slope of a hit at z = 0: infinite, clamped
    odd[9, 0] = np.nan
    odd[11, 2] = np.nan
    odd[13, 1] = np.inf
    return [make_event(wl, 9, 0, vertex_sigma=(0, 0, 0)).hits,  # one chunk
            make_event(wl, 9, 1, n_tracks=700, vertex_sigma=(0, 0, 0)).hits,  # two chunks merged
            make_event(wl, 9, 2, n_tracks=1500, vertex_sigma=(0, 0, 0)).hits,  # two super-chunks
            one_band, odd, np.zeros((0, 4), np.float32)]


@pytest.mark.parametrize("many", [False, True])
def test_prepared_order_is_the_documented_key(rt, many):
    # few events take the cluster kernel, many the one-CTA-per-event kernel:
    # both give exactly the documented order
    hs = _order_events()
    assert len(hs[2]) > 32768 and len(hs[1]) > 8192
    if many:
        hs = hs + [make_event(WORKLOADS["velo_batch"], 9, e, vertex_sigma=(0, 0, 0)).hits for e in range(90)]
    off = np.concatenate([[0], np.cumsum([len(h) for h in hs])]).astype(np.int64)
    srt, _ = rt.prepare_hits(_dev(np.concatenate(hs)), _dev(off), 1)
    srt = srt.cpu().numpy()
    for e, h in enumerate(hs):
        np.testing.assert_array_equal(srt[off[e]:off[e + 1]], h[documented_order(h, 1)], err_msg="event %d" % e)


def test_prepared_order_toy_is_the_documented_key(rt):
    wl, evs, b = _batch(0)
    srt, _ = rt.prepare_hits(_dev(b.hits), _dev(b.offsets), 0)
    srt = srt.cpu().numpy()
    for e, ev in enumerate(evs):
        h0, h1 = b.offsets[e], b.offsets[e + 1]
        np.testing.assert_array_equal(srt[h0:h1], b.hits[h0:h1][documented_order(b.hits[h0:h1], 0)])
