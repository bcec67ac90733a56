"""High-multiplicity events (~600 tracks, 15 % noise, ~16.5k hits, 2048^2 grid)
on the GPU against the FP64 oracle: hit ordering across sort chunks, the grid
response on sampled cells of the full 2048^2 grid, the batched search from
seeds near tracks and uniform seeds (robust seeds identical branches), and the
learned proposer's 2048 seeds from the oracle's logits."""
import numpy as np
import pytest
import torch

import oracle
from oracle import seednet as sn
from synth import WORKLOADS, batch_of, make_event, uniform_seeds

from test_gpu_parity import R_ABS, R_REL, _check_search, dev

pytestmark = pytest.mark.gpu

WL = WORKLOADS["velo_stress"]


@pytest.fixture(scope="module")
def rt():
    from paper_1709_08610_gb300 import build as rbuild
    rbuild.build()
    from paper_1709_08610_gb300 import retina
    return retina


@pytest.fixture(scope="module")
def evs():
    return [make_event(WL, 21, 0, vertex_sigma=(0, 0, 0)), make_event(WL, 21, 1)]


def test_stress_events_span_sort_chunks_and_grid_matches_oracle(rt, evs):
    b = batch_of(evs)
    assert b.hits.shape[0] / len(evs) > 14000
    srt, boxes = rt.prepare_hits(dev(b.hits), dev(b.offsets), 1)
    offs = dev(b.offsets)
    grid = rt.Grid.of(WL)
    R = rt.grid_response(srt, offs, 1, grid, WL.sigma_grid, boxes=boxes).cpu().numpy()
    R_full = rt.grid_response(srt, offs, 1, grid, WL.sigma_grid).cpu().numpy()
    assert np.array_equal(R, R_full)            # block skipping stays exact
    c0, c1 = oracle.cell_centres(grid.lo, grid.step, grid.n)
    rng = np.random.default_rng(1)
    for e, ev in enumerate(evs):
        flat = R[e].reshape(-1)
        idx = np.concatenate([rng.integers(0, flat.size, 300), np.argsort(flat)[-200:]])
        th = np.stack([c0[idx % grid.n[0]], c1[idx // grid.n[0]]], 1)
        R_o = oracle.response(ev.hits, 1, th, WL.sigma_grid)
        assert np.all(np.abs(flat[idx] - R_o) <= R_REL * R_o + R_ABS)


def test_stress_batched_search_matches_oracle(rt, evs):
    ev = evs[0]
    rng = np.random.default_rng(5)
    near = ev.truth[:, :2][rng.integers(0, len(ev.truth), 300)] + rng.normal(0, 3, (300, 2)) * WL.grid_step[0]
    seeds = np.concatenate([near, uniform_seeds(WL, 100, 21, 0)]).astype(np.float32)
    off = np.array([0, ev.n_hits], np.int64)
    srt, boxes = rt.prepare_hits(dev(ev.hits), dev(off), 1)
    so = dev(np.array([0, len(seeds)], np.int64))
    opts = rt.LsOpts(sigma=tuple(WL.sigma_schedule))
    th_g, R_g, st_g = rt.batched_search(srt, dev(off), 1, dev(seeds), so, opts, rt.Grid.of(WL), boxes=boxes)
    th_o, R_o, st_o, m_o = oracle.local_search(ev.hits, 1, seeds, WL.sigma_schedule, WL.grid_lo, WL.grid_step,
                                               WL.grid_n)
    _, n_conv = _check_search(WL, ev, th_g.cpu().numpy().astype(float), R_g.cpu().numpy().astype(float),
                              st_g.cpu().numpy(), th_o, R_o, st_o, m_o, min_robust=250)
    assert n_conv >= 60  # seeds 3 cells off a track in a 600-track event do not all reach a strict maximum


def test_stress_proposer_2048_seeds_match_oracle(rt, evs):
    from paper_1709_08610_gb300.seednet import DEFAULT_WEIGHTS, read_checkpoint
    _, a = read_checkpoint(DEFAULT_WEIGHTS)
    b = batch_of(evs)
    logits = np.stack([sn.forward(sn.slope_histogram(ev.hits)[1], a["params"])["z"] for ev in evs]).astype(np.float32)
    seeds, cells = rt.topk_seeds(dev(logits), 2048, hits=dev(b.hits), offsets=dev(b.offsets), want_idx=True)
    seeds, cells = seeds.cpu().numpy().astype(np.float64), cells.cpu().numpy()
    for e, ev in enumerate(evs):
        s_o, c_o = sn.propose_seeds(logits[e], ev.hits, 2048)
        np.testing.assert_array_equal(cells[e], c_o)
        assert np.all(np.abs(seeds[e] - s_o) <= 2.0 ** -16 / 256 + 2.0 ** -24 * np.abs(s_o) + 1e-12)
