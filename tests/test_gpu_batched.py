"""Persistent batched search (ragged events and seed counts, one launch) on the GPU.

Its per-seed arithmetic is the per-launch search's, and each lane visits the
hits in the same order, so for the same seeds the two entry points must agree
bit for bit; claim order and launch shape must not change a bit either.
Against the FP64 oracle the per-event comparison is the one used for the
per-launch search (robust decisions: same status; converged maxima within
1e-3 cell).
"""
import numpy as np
import pytest
import torch

import oracle
from hit_order import hilbert
from synth import WORKLOADS, make_event, batch_of, uniform_seeds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    from paper_1709_08610_gb300 import build as rbuild
    rbuild.build()
    from paper_1709_08610_gb300 import retina
    return retina


def _ragged(seed=0):
    wl = WORKLOADS["velo"]
    evs = [make_event(wl, seed, 0, vertex_sigma=(0, 0, 0)),
           make_event(wl, seed, 1, n_tracks=12, vertex_sigma=(0, 0, 0)),
           make_event(wl, seed, 2, n_tracks=0, noise_frac=0.0),           # empty event
           make_event(wl, seed, 3, n_tracks=400, vertex_sigma=(0, 0, 0)),  # > 8192 hits: global tail
           make_event(wl, seed, 4, n_tracks=60)]
    counts = [700, 33, 5, 257, 0]  # ragged, one event without seeds
    rng = np.random.default_rng(seed)
    seeds = []
    for ev, n in zip(evs, counts):
        if len(ev.truth) and n:
            k = n // 2
            near = ev.truth[:, :2][rng.integers(0, len(ev.truth), k)] + rng.normal(0, 3, (k, 2)) * 2 ** -10
            seeds.append(np.concatenate([near, uniform_seeds(wl, n - k, seed, 9)]).astype(np.float32))
        else:
            seeds.append(uniform_seeds(wl, n, seed, 9))
    so = np.zeros(len(evs) + 1, np.int64)
    np.cumsum(counts, out=so[1:])
    return wl, evs, batch_of(evs), np.concatenate(seeds), so


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("update", [0, 1, 2])
def test_batched_matches_per_launch_search_bitwise(rt, update):
    wl, evs, b, seeds, so = _ragged()
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule), update=update)
    box = rt.Grid.of(wl)
    th, R, st = rt.batched_search(_dev(b.hits), _dev(b.offsets), 1, _dev(seeds), _dev(so), opts, box)
    th, R, st = th.cpu().numpy(), R.cpu().numpy(), st.cpu().numpy()
    for e, ev in enumerate(evs):
        s0, s1 = so[e], so[e + 1]
        if s1 == s0:
            continue
        off = np.array([0, ev.n_hits], np.int64)
        t1, R1, st1 = rt.local_search(_dev(ev.hits), _dev(off), 1, _dev(seeds[s0:s1][None]), opts, box)
        np.testing.assert_array_equal(th[s0:s1], t1.cpu().numpy()[0])
        np.testing.assert_array_equal(R[s0:s1], R1.cpu().numpy()[0])
        np.testing.assert_array_equal(st[s0:s1], st1.cpu().numpy()[0])
    assert np.all(R[so[2]:so[3]] == 0.0)  # empty event


@pytest.mark.parametrize("with_boxes", [False, True])
@pytest.mark.parametrize("spw,warps,ctas", [(1, 8, 0), (2, 16, 0), (4, 32, 0), (1, 32, 0), (1, 8, 1)])
def test_batched_results_independent_of_order_and_shape(rt, spw, warps, ctas, with_boxes):
    # one, two or four seeds per warp (shared block tests and hit loads, the
    # union of the seeds' kept blocks): the accepted trials, every sum and the
    # trial counts must agree bit for bit, with exact block skipping on or off;
    # one seed per warp tests the backtracking trials in pairs when the launch
    # has at most two seeds per warp (ctas 0: the whole GPU) and one at a time
    # otherwise (one 8-warp CTA for the ~1000 seeds); four seeds per warp with
    # boxes take the kernel that keeps one kept-block list per update (the
    # batch averages 3.2k hits per event; its 10.3k-hit event tests per pass)
    wl, evs, b, seeds, so = _ragged(1)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    box = rt.Grid.of(wl)
    offs = _dev(b.offsets)
    hits, bx = rt.prepare_hits(_dev(b.hits), offs, 1)
    boxes = bx if with_boxes else None
    S = len(seeds)
    ev_ref = torch.empty(S, dtype=torch.uint8, device="cuda")
    old = (rt.get_option(rt.OPT_BATCH_SEEDS_PER_WARP), rt.get_option(rt.OPT_BATCH_WARPS),
           rt.get_option(rt.OPT_BATCH_CTAS))
    try:
        rt.set_option(rt.OPT_BATCH_SEEDS_PER_WARP, 2)
        ref = rt.batched_search(hits, offs, 1, _dev(seeds), _dev(so), opts, box, n_evals=ev_ref)
        rt.set_option(rt.OPT_BATCH_SEEDS_PER_WARP, spw)
        rt.set_option(rt.OPT_BATCH_WARPS, warps)
        rt.set_option(rt.OPT_BATCH_CTAS, ctas)
        order = _dev(np.array([3, 0, 4, 1, 2], np.int32))
        ev_got = torch.empty(S, dtype=torch.uint8, device="cuda")
        got = rt.batched_search(hits, offs, 1, _dev(seeds), _dev(so), opts, box, order=order, n_evals=ev_got,
                                boxes=boxes)
    finally:
        rt.set_option(rt.OPT_BATCH_SEEDS_PER_WARP, old[0])
        rt.set_option(rt.OPT_BATCH_WARPS, old[1])
        rt.set_option(rt.OPT_BATCH_CTAS, old[2])
    for x, y in zip(ref, got):
        np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())
    np.testing.assert_array_equal(ev_ref.cpu().numpy(), ev_got.cpu().numpy())
    assert ev_ref.max().item() > 3  # some seeds backtrack (3 = one trial per update)


def test_batched_matches_oracle_per_event(rt):
    wl, evs, b, seeds, so = _ragged(2)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    th, R, st = rt.batched_search(_dev(b.hits), _dev(b.offsets), 1, _dev(seeds), _dev(so), opts, rt.Grid.of(wl))
    th, R, st = th.cpu().numpy().astype(float), R.cpu().numpy().astype(float), st.cpu().numpy()
    step = np.asarray(wl.grid_step)
    n_conv = 0
    for e, ev in enumerate(evs):
        s0, s1 = so[e], so[e + 1]
        if s1 == s0:
            continue
        th_o, R_o, st_o, m_o = oracle.local_search(ev.hits, 1, seeds[s0:s1], wl.sigma_schedule, wl.grid_lo,
                                                   wl.grid_step, wl.grid_n)
        rob = m_o >= 1.0
        assert np.all(st[s0:s1][rob] == st_o[rob])
        for i in np.flatnonzero(rob & (st_o <= 2)):
            o = oracle.rgh(ev.hits, 1, th_o[i], wl.sigma_schedule[-1])
            conv = False
            if np.all(np.linalg.eigvalsh(o["hess"]) < 0):
                try:
                    conv = np.max(np.abs(np.linalg.solve(o["hess"], o["grad"])) / step) <= 0.05
                except np.linalg.LinAlgError:
                    conv = False
            n_conv += conv
            d = (1e-3 if conv else 5e-2) * step
            assert np.all(np.abs(th[s0 + i] - th_o[i]) <= d)
    assert n_conv >= 50


def test_batched_search_replays_in_a_cuda_graph(rt):
    wl, evs, b, seeds, so = _ragged(3)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    box = rt.Grid.of(wl)
    hits, offs, sd, sod = _dev(b.hits), _dev(b.offsets), _dev(seeds), _dev(so)
    S = seeds.shape[0]
    out = (torch.empty((S, 2), device="cuda"), torch.empty((S,), device="cuda"),
           torch.empty((S,), dtype=torch.uint8, device="cuda"))
    ws = torch.empty(max(rt.batched_search_workspace_size(len(evs)), 256), dtype=torch.uint8, device="cuda")
    eager = [x.clone() for x in rt.batched_search(hits, offs, 1, sd, sod, opts, box)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up on the capture stream (lazy attribute setup happens here)
        rt.batched_search(hits, offs, 1, sd, sod, opts, box, out=out, ws=ws)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rt.batched_search(hits, offs, 1, sd, sod, opts, box, out=out, ws=ws)
    for _ in range(2):
        for x in out:
            x.zero_()
        g.replay()
        torch.cuda.synchronize()
        for x, y in zip(eager, out):
            np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())


def _hilbert9(S, box):
    """Host restatement of the documented seed key (order-9 Hilbert index in the box)."""
    lo = np.asarray(box.lo, np.float32)
    inv = (1.0 / (np.asarray(box.n, np.float64) * np.asarray(box.step, np.float64))).astype(np.float32)
    q = (S.astype(np.float32) - lo) * inv
    qi = np.where(q > 0, np.where(q < 1, np.floor(q * np.float32(512)).astype(np.int64) & 511, 511), 0)
    return hilbert(qi[:, 0], qi[:, 1], 9)


def test_sorted_seeds_are_a_spatial_permutation_and_search_results_follow_them(rt):
    wl, evs, b, seeds, so = _ragged(4)
    seeds = seeds.copy()
    seeds[3] = np.nan                       # a non-finite point goes last in its event
    box = rt.Grid.of(wl)
    srt, perm = rt.sort_seeds(_dev(seeds), _dev(so), box, want_perm=True)
    srt, perm = srt.cpu().numpy(), perm.cpu().numpy()
    for e in range(len(evs)):
        s0, s1 = so[e], so[e + 1]
        p = perm[s0:s1]
        assert sorted(p.tolist()) == list(range(s0, s1))
        np.testing.assert_array_equal(srt[s0:s1], seeds[p])
        fin = np.isfinite(seeds[p]).all(1)
        key = np.where(fin, _hilbert9(seeds[p], box), 1 << 18) * (1 << 13) + (p - s0)
        assert np.all(np.diff(key) > 0)
    # the search is per seed: on sorted points with two seeds per warp, every
    # result is bitwise the unsorted one-seed-per-warp result of the same point
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    ref = rt.batched_search(_dev(b.hits), _dev(b.offsets), 1, _dev(seeds), _dev(so), opts, box)
    old = rt.get_option(rt.OPT_BATCH_SEEDS_PER_WARP)
    rt.set_option(rt.OPT_BATCH_SEEDS_PER_WARP, 2)
    try:
        got = rt.batched_search(_dev(b.hits), _dev(b.offsets), 1, _dev(srt), _dev(so), opts, box)
    finally:
        rt.set_option(rt.OPT_BATCH_SEEDS_PER_WARP, old)
    for x, y in zip(ref, got):
        x, y = x.cpu().numpy(), y.cpu().numpy()
        np.testing.assert_array_equal(x[perm], y)


def test_sorted_seeds_in_chunks_of_8192(rt):
    """Events with more than 8192 points are ordered chunk by chunk (each chunk
    a spatially sorted permutation of its own rows)."""
    wl = WORKLOADS["velo"]
    box = rt.Grid.of(wl)
    n = [10000, 8192, 1, 0, 20000]
    S = np.concatenate([uniform_seeds(wl, k, 7, e) for e, k in enumerate(n)]).astype(np.float32)
    so = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
    srt, perm = rt.sort_seeds(_dev(S), _dev(so), box, want_perm=True)
    srt, perm = srt.cpu().numpy(), perm.cpu().numpy()
    np.testing.assert_array_equal(srt, S[perm])
    for e in range(len(n)):
        for c0 in range(so[e], so[e + 1], 8192):
            c1 = min(c0 + 8192, so[e + 1])
            p = perm[c0:c1]
            assert sorted(p.tolist()) == list(range(c0, c1))
            key = _hilbert9(S[p], box) * (1 << 13) + (p - c0)
            assert np.all(np.diff(key) > 0)
