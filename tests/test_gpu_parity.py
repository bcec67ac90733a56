"""CUDA path vs the FP64 oracle, through the C ABI (via the thin binding).

Tolerances (from the FP32 arithmetic of the kernels, see the design notes):
  R                 |dR| <= 1e-5 R + 1e-6
  gradient, Hessian |d|  <= 1e-4 * sum of |terms| (cancellation near maxima)
  search points     |dtheta|_inf <= 1e-3 * grid step
Integer / index outputs (grid maxima, extracted tracks) are compared exactly
when both sides see the same float32 inputs; when each side computes its own
responses, points whose oracle decision margin is below the tolerance are
ties, where either outcome is correct, and are excluded and counted.
"""
import numpy as np
import pytest
import torch

import oracle
from parity_rules import candidates, check_conditioned, compare_track_sets, search_tolerance
from synth import WORKLOADS, make_event, make_batch, batch_of, uniform_seeds, make_toy2d_event

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


def velo0(seed, eid, **kw):
    return make_event(WORKLOADS["velo"], seed, eid, vertex_sigma=(0, 0, 0), **kw)


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# Eq. 1 with gradient and Hessian at points
# ---------------------------------------------------------------------------

def _gh_floors(hits, model, sigma):
    """Absolute floors of the gradient / Hessian tolerance: 1e-6 of their
    scale at unit response (one hit at r = sigma), mirroring R's 1e-6 floor;
    below it the oracle keeps double-precision tails that FP32 ex2 flushes."""
    jmax = float(np.max(np.abs(hits[:, 2]))) if model == 1 else max(float(np.max(np.abs(hits[:, 0]))), 1.0)
    k = 1.0 / sigma ** 2
    return 1e-6 * 2 * k * sigma * jmax, 1e-6 * 2 * k * jmax ** 2


@pytest.mark.parametrize("wl_name", ["toy2d", "velo"])
def test_response_grad_hess_match_oracle(rt, wl_name):
    wl = WORKLOADS[wl_name]
    ev = make_event(wl, 5, 1, **({"vertex_sigma": (0, 0, 0)} if wl.model == 1 else {}))
    rng = np.random.default_rng(0)
    near = ev.truth[:64, :2] + rng.normal(0, 1.0, (min(64, len(ev.truth)), 2)) * np.asarray(wl.grid_step)
    far = np.asarray(wl.grid_lo) + rng.uniform(0, 1, (64, 2)) * np.asarray(wl.grid_n) * np.asarray(wl.grid_step)
    pts = np.concatenate([near, far]).astype(np.float32)
    off = np.array([0, ev.n_hits], np.int64)
    for sigma in sorted(set(wl.sigma_schedule) | {wl.sigma_grid}):
        gf, hf = _gh_floors(ev.hits, wl.model, sigma)
        out = rt.response(dev(ev.hits), dev(off), wl.model, dev(pts[None]), sigma).cpu().numpy()[0].astype(float)
        for i, th in enumerate(pts.astype(float)):
            o = oracle.rgh(ev.hits, wl.model, th, sigma)
            assert abs(out[i, 0] - o["R"]) <= R_REL * o["R"] + R_ABS, (sigma, i)
            assert np.all(np.abs(out[i, 1:3] - o["grad"]) <= GH_REL * o["grad_abs"].sum() + gf), (sigma, i)
            Hg = np.array([out[i, 3], out[i, 4], out[i, 4], out[i, 5]])
            assert np.all(np.abs(Hg - o["hess"].reshape(-1)) <= GH_REL * o["hess_abs"].sum() + hf), (sigma, i)


# ---------------------------------------------------------------------------
# Eq. 2 on the grid
# ---------------------------------------------------------------------------

def _window(wl, i0, i1, n0, n1):
    lo = (wl.grid_lo[0] + i0 * wl.grid_step[0], wl.grid_lo[1] + i1 * wl.grid_step[1])
    return lo, tuple(wl.grid_step), (n0, n1)


@pytest.mark.parametrize("flags", [0, 1])
def test_grid_response_toy_full_grid(rt, flags):
    wl = WORKLOADS["toy2d"]
    ev = make_event(wl, 0, 3)
    R_o = oracle.grid_response(ev.hits, 0, wl.grid_lo, wl.grid_step, wl.grid_n, wl.sigma_grid)
    off = np.array([0, ev.n_hits], np.int64)
    out = rt.grid_scan(dev(ev.hits), dev(off), 0, rt.Grid.of(wl), wl.sigma_grid, wl.R0, 4096, flags=flags,
                       store_R=True)
    R_g = out["R"].cpu().numpy()[0].astype(float)
    assert np.all(np.abs(R_g - R_o) <= R_REL * R_o + R_ABS)


@pytest.mark.parametrize("flags", [1, 2, 3])
@pytest.mark.parametrize("shape", [(192, 160), (131, 67), (256, 256)])
def test_grid_response_velo_window_ragged(rt, flags, shape):
    # windows spanning several tiles with ragged edges, three ragged events (one empty)
    wl = WORKLOADS["velo"]
    evs = [velo0(1, 0), make_event(wl, 1, 1, n_tracks=40), velo0(1, 2, n_tracks=0, noise_frac=0.0)]
    b = batch_of(evs)
    lo, step, n = _window(wl, 400, 430, *shape)
    grid = rt.Grid(lo, step, n)
    out = rt.grid_scan(dev(b.hits), dev(b.offsets), 1, grid, wl.sigma_grid, wl.R0, 1024, flags=flags, store_R=True)
    R_g = out["R"].cpu().numpy().astype(float)
    for e, ev in enumerate(evs):
        R_o = oracle.grid_response(ev.hits, 1, lo, step, n, wl.sigma_grid)
        assert np.all(np.abs(R_g[e] - R_o) <= R_REL * R_o + R_ABS), (e, np.max(np.abs(R_g[e] - R_o)))
    assert np.all(R_g[2] == 0.0)
    assert out["n_max"].cpu().numpy()[2] == 0


@pytest.mark.parametrize("flags", [1, 2, 3])
def test_grid_response_full_size_sampled(rt, flags):
    # the full 1024^2 slope grid of the single-event workload, in the bench's
    # launch configuration; 3000 sampled cells against the oracle one by one
    wl = WORKLOADS["velo"]
    ev = make_event(wl, 0, 0)
    off = np.array([0, ev.n_hits], np.int64)
    out = rt.grid_scan(dev(ev.hits), dev(off), 1, rt.Grid.of(wl), wl.sigma_grid, wl.R0, 8192, flags=flags,
                       store_R=True)
    R_g = out["R"].cpu().numpy()[0].astype(float)
    rng = np.random.default_rng(1)
    idx = rng.integers(0, R_g.size, 3000)
    # add the cells around the largest responses
    idx = np.concatenate([idx, np.argsort(R_g.reshape(-1))[-500:]])
    i0, i1 = idx % wl.grid_n[0], idx // wl.grid_n[0]
    c0, c1 = oracle.cell_centres(wl.grid_lo, wl.grid_step, wl.grid_n)
    R_o = oracle.response(ev.hits, 1, np.stack([c0[i0], c1[i1]], 1), wl.sigma_grid)
    got = R_g.reshape(-1)[idx]
    assert np.all(np.abs(got - R_o) <= R_REL * R_o + R_ABS)
    # every R is in [0, N]
    assert R_g.min() >= 0 and R_g.max() <= ev.n_hits


def test_grid_response_wide_tiles_on_a_batch(rt):
    # a batch large enough for the 128 x 256 tensor-core tiles (the launch
    # rule takes them from 8 x 152 tiles of 128 x 128 on), on a 1024 x 600
    # window: the last tile column is ragged (88 cells); 3 of the 32 events
    # against the oracle on sampled cells and the cells around the peaks
    wl = WORKLOADS["velo_batch"]
    evs = [make_event(wl, 3, e, vertex_sigma=(0, 0, 0)) for e in range(32)]
    b = batch_of(evs)
    n = (1024, 600)
    lo = (wl.grid_lo[0], wl.grid_lo[1] + 200 * wl.grid_step[1])
    grid = rt.Grid(lo, wl.grid_step, n)
    R = torch.empty((len(evs), n[1], n[0]), dtype=torch.float32, device="cuda")
    ws = torch.empty(max(rt.grid_response_workspace_size(len(evs), 1, grid), 1), dtype=torch.uint8, device="cuda")
    offs = dev(b.offsets)
    srt, bx = rt.prepare_hits(dev(b.hits), offs, 1)  # the bench's path: ordered hits, exact block skipping
    rt.grid_response(srt, offs, 1, grid, wl.sigma_grid, R_out=R, ws=ws, boxes=bx)
    R_g = R.cpu().numpy().astype(float)
    c0, c1 = oracle.cell_centres(lo, wl.grid_step, n)
    rng = np.random.default_rng(2)
    for e in (0, 17, 31):
        idx = np.concatenate([rng.integers(0, n[0] * n[1], 1500), np.argsort(R_g[e].reshape(-1))[-300:],
                              np.arange(n[0] * (n[1] - 1), n[0] * n[1])[::7]])  # the ragged last rows
        i0, i1 = idx % n[0], idx // n[0]
        R_o = oracle.response(evs[e].hits, 1, np.stack([c0[i0], c1[i1]], 1), wl.sigma_grid)
        got = R_g[e].reshape(-1)[idx]
        assert np.all(np.abs(got - R_o) <= R_REL * R_o + R_ABS), (e, np.max(np.abs(got - R_o)))


# ---------------------------------------------------------------------------
# grid maxima: exact on identical float32 inputs, tie-aware end to end
# ---------------------------------------------------------------------------

def test_grid_maxima_exact_on_identical_inputs(rt):
    wl = WORKLOADS["velo"]
    lo, step, n = _window(wl, 380, 400, 300, 260)
    evs = [velo0(2, e) for e in range(3)]
    Rs = [f32(oracle.grid_response(ev.hits, 1, lo, step, n, wl.sigma_grid)) for ev in evs]
    # a quantised copy creates many exact ties, exercising the index tie rule
    Rs.append(np.round(Rs[0] * 4) / 4)
    Rs.append(np.zeros_like(Rs[0]))
    grid = rt.Grid(lo, step, n)
    K = 64
    out = rt.grid_maxima(dev(np.stack(Rs).astype(np.float32)), grid, 3.0, K)
    n_max = out["n_max"].cpu().numpy()
    idx = out["max_idx"].cpu().numpy()
    th = out["max_theta"].cpu().numpy()
    Rm = out["max_R"].cpu().numpy()
    c0, c1 = oracle.cell_centres(lo, step, n)
    for e, R in enumerate(Rs):
        exp_idx = oracle.grid_maxima(R, float(np.float32(3.0)))
        assert n_max[e] == len(exp_idx)
        k = min(K, len(exp_idx))
        assert idx[e, :k].tolist() == exp_idx[:k].tolist()
        np.testing.assert_array_equal(th[e, :k, 0], c0[exp_idx[:k] % n[0]].astype(np.float32))
        np.testing.assert_array_equal(th[e, :k, 1], c1[exp_idx[:k] // n[0]].astype(np.float32))
        np.testing.assert_array_equal(Rm[e, :k], R.reshape(-1)[exp_idx[:k]].astype(np.float32))
    assert n_max[3] > K  # truncation exercised
    assert n_max[4] == 0


@pytest.mark.parametrize("n,K", [((100, 100), 64), ((150, 150), 3000), ((1024, 600), 5000), ((1024, 600), 16)])
def test_grid_maxima_exact_on_noise_many_maxima(rt, n, K):
    """Seeded noise grids hold ~cells/9 strict maxima: the ordering of 1-4k
    candidates and, past 4096 per event, the exact whole-grid fallback."""
    rng = np.random.default_rng(n[0] * 7 + K)
    Rs = [rng.uniform(0, 1, (n[1], n[0])).astype(np.float32) for _ in range(2)]
    Rs[1] = np.round(Rs[1] * 8) / 8  # exact ties
    grid = rt.Grid((-0.5, -0.5), (2.0 ** -10, 2.0 ** -10), n)
    out = rt.grid_maxima(dev(np.stack(Rs).astype(np.float32)), grid, 0.25, K)
    n_max, idx = out["n_max"].cpu().numpy(), out["max_idx"].cpu().numpy()
    Rm = out["max_R"].cpu().numpy()
    for e, R in enumerate(Rs):
        exp_idx = oracle.grid_maxima(R, 0.25)
        assert n_max[e] == len(exp_idx)
        k = min(K, len(exp_idx))
        assert idx[e, :k].tolist() == exp_idx[:k].tolist()
        np.testing.assert_array_equal(Rm[e, :k], R.reshape(-1)[exp_idx[:k]])


@pytest.mark.parametrize("flags", [1, 2, 3])
def test_grid_scan_maxima_match_oracle_up_to_ties(rt, flags):
    wl = WORKLOADS["velo"]
    lo, step, n = _window(wl, 300, 300, 384, 384)
    ev = velo0(3, 0)
    off = np.array([0, ev.n_hits], np.int64)
    out = rt.grid_scan(dev(ev.hits), dev(off), 1, rt.Grid(lo, step, n), wl.sigma_grid, wl.R0, 4096, flags=flags)
    got = set(out["max_idx"].cpu().numpy()[0, :out["n_max"].item()].tolist())
    R_o = oracle.grid_response(ev.hits, 1, lo, step, n, wl.sigma_grid)
    exp, cnt, margin = oracle.grid_maxima(R_o, wl.R0, with_margin=True)
    exp = set(exp.tolist())
    assert len(exp) >= 5
    tol = R_REL * R_o.reshape(-1) + R_ABS
    for c in got ^ exp:
        assert margin.reshape(-1)[c] <= 2 * tol[c], c


def test_grid_scan_toy_matches_oracle(rt):
    wl = WORKLOADS["toy2d"]
    for eid in range(8):
        ev = make_event(wl, 0, eid)
        off = np.array([0, ev.n_hits], np.int64)
        out = rt.grid_scan(dev(ev.hits), dev(off), 0, rt.Grid.of(wl), wl.sigma_grid, wl.R0, 4096)
        got = set(out["max_idx"].cpu().numpy()[0, :out["n_max"].item()].tolist())
        R_o = oracle.grid_response(ev.hits, 0, wl.grid_lo, wl.grid_step, wl.grid_n, wl.sigma_grid)
        exp, cnt, margin = oracle.grid_maxima(R_o, wl.R0, with_margin=True)
        tol = R_REL * R_o.reshape(-1) + R_ABS
        for c in got ^ set(exp.tolist()):
            assert margin.reshape(-1)[c] <= 2 * tol[c]


# ---------------------------------------------------------------------------
# local search (Algorithm 1 + truncated Newton)
# ---------------------------------------------------------------------------

def _search_both(rt, wl, ev, seeds, sigma=None, update=0):
    sig = tuple(wl.sigma_schedule if sigma is None else sigma)
    off = np.array([0, ev.n_hits], np.int64)
    th_g, R_g, st_g = rt.local_search(dev(ev.hits), dev(off), wl.model, dev(seeds[None]),
                                      rt.LsOpts(sigma=sig, update=update), rt.Grid.of(wl))
    th_o, R_o, st_o, m_o = oracle.local_search(ev.hits, wl.model, seeds, sig, wl.grid_lo, wl.grid_step, wl.grid_n,
                                               update=update)
    return (th_g.cpu().numpy()[0].astype(float), R_g.cpu().numpy()[0].astype(float), st_g.cpu().numpy()[0],
            th_o, R_o, st_o, m_o)


def _check_search(wl, ev, th_g, R_g, st_g, th_o, R_o, st_o, m_o, min_robust):
    """Seeds whose every oracle decision is robust (margin >= 1) must take the
    same branches: identical status; theta within 1e-3 cell where the oracle's
    point is a converged maximum (negative-definite Hessian and Newton
    distance |H^-1 g| <= 0.05 cell at sigma_q).  Away from a maximum the end
    point is not defined to that precision (on a ridge R is flat along it and
    the remaining Newton steps amplify FP32 rounding), so there theta must
    agree to 0.05 cell; R within its FP32 tolerance plus the change the
    allowed theta difference can cause, |g| dtheta + |H| dtheta^2, g and H
    being the oracle's own at its point."""
    robust = m_o >= 1.0
    assert robust.sum() >= min_robust, robust.sum()
    assert np.all(st_g[robust] == st_o[robust])
    step = np.asarray(wl.grid_step)
    sq = wl.sigma_schedule[-1]
    n_conv = 0
    for i in np.flatnonzero(robust & (st_o <= 2)):
        o = oracle.rgh(ev.hits, wl.model, th_o[i], sq)
        H, g = o["hess"], o["grad"]
        conv = False
        if np.all(np.linalg.eigvalsh(H) < 0):
            try:
                conv = np.max(np.abs(np.linalg.solve(H, g)) / step) <= 0.05
            except np.linalg.LinAlgError:
                conv = False
        n_conv += conv
        d = (TH_CELLS if conv else 50 * TH_CELLS) * step
        dth = np.abs(th_g[i] - th_o[i])
        assert np.all(dth <= d), (i, conv, dth / step, R_o[i])
        tol = R_REL * R_o[i] + R_ABS + np.abs(g) @ d + np.abs(H).max() * (d @ d)
        assert abs(R_g[i] - R_o[i]) <= tol, (i, R_g[i], R_o[i], tol)
    return robust, n_conv


def test_local_search_toy_matches_oracle(rt):
    wl = WORKLOADS["toy2d"]
    for eid in range(4):
        ev = make_event(wl, 0, eid)
        seeds = uniform_seeds(wl, wl.n_seeds, 0, eid)
        res = _search_both(rt, wl, ev, seeds)
        _, n_conv = _check_search(wl, ev, *res, min_robust=100)
        assert n_conv >= 1


@pytest.mark.parametrize("spw", [1, 2, 4])
def test_local_search_velo_matches_oracle(rt, spw):
    wl = WORKLOADS["velo"]
    ev = velo0(0, 0)
    # seeds near tracks (alive everywhere) plus uniform ones; count not a multiple of a block
    rng = np.random.default_rng(4)
    near = ev.truth[:, :2][rng.integers(0, len(ev.truth), 700)] + rng.normal(0, 3, (700, 2)) * 2 ** -10
    seeds = np.concatenate([near, uniform_seeds(wl, 301, 0, 0)]).astype(np.float32)
    old = rt.get_option(rt.OPT_LS_SEEDS_PER_WARP)
    rt.set_option(rt.OPT_LS_SEEDS_PER_WARP, spw)
    try:
        res = _search_both(rt, wl, ev, seeds)
    finally:
        rt.set_option(rt.OPT_LS_SEEDS_PER_WARP, old)
    _, n_conv = _check_search(wl, ev, *res, min_robust=600)
    assert n_conv >= 100


def _converged_2d(ev, wl):
    step = np.asarray(wl.grid_step)
    sq = wl.sigma_schedule[-1]

    def at(th):
        o = oracle.rgh(ev.hits, wl.model, th, sq)
        H, g = o["hess"], o["grad"]
        if not np.all(np.linalg.eigvalsh(H) < 0):
            return None
        try:
            if np.max(np.abs(np.linalg.solve(H, g)) / step) > 0.05:
                return None
        except np.linalg.LinAlgError:  # numerically singular: a flat ridge, not a converged peak
            return None
        return g, H, o["grad_abs"]
    return at


@pytest.mark.parametrize("update", [1, 2])
@pytest.mark.parametrize("wl_name", ["toy2d", "velo"])
def test_local_search_alternative_updates_match_oracle(rt, update, wl_name):
    # steepest ascent (1): the robust-decision parity of the truncated Newton
    # search.  Newton with a modified Hessian (2): a shifted step solves a
    # system of condition >= 1e3, which can amplify float32 rounding, so the
    # paths are classified by the oracle's perturbed replicas first
    # (check_conditioned): point-wise parity on every robust, well-conditioned
    # seed; the rest are counted and checked for validity
    wl = WORKLOADS[wl_name]
    if wl_name == "velo":
        ev = velo0(0, 2)
        rng = np.random.default_rng(6)
        near = ev.truth[:, :2][rng.integers(0, len(ev.truth), 500)] + rng.normal(0, 3, (500, 2)) * 2 ** -10
        seeds = np.concatenate([near, uniform_seeds(wl, 201, 0, 2)]).astype(np.float32)
    else:
        ev = make_event(wl, 0, 5)
        seeds = uniform_seeds(wl, wl.n_seeds, 0, 5)
    res = _search_both(rt, wl, ev, seeds, update=update)
    if update == 1:
        _check_search(wl, ev, *res, min_robust=len(seeds) // 4)
        return
    th_g, R_g, st_g = res[:3]
    sig = tuple(wl.sigma_schedule)

    def run(pt):
        return oracle.local_search(ev.hits, wl.model, seeds, sig, wl.grid_lo, wl.grid_step, wl.grid_n,
                                   update=update, perturb=pt)

    # the oracle ends 165 (velo) / 15 (toy) robust, well-conditioned seeds at converged maxima
    check_conditioned(th_g, R_g, st_g, res[3:], run, wl.grid_step, _converged_2d(ev, wl),
                      lambda th: oracle.response(ev.hits, wl.model, [th], sig[-1])[0],
                      min_firm_conv=120 if wl_name == "velo" else 10)


def test_local_search_svelo_matches_oracle(rt):
    # the paper's own sVELO geometry (20 disks, p_hit 0.5, Poisson(250) noise)
    wl = WORKLOADS["svelo"]
    ev = make_event(wl, 0, 0)
    rng = np.random.default_rng(7)
    near = ev.truth[:, :2][rng.integers(0, len(ev.truth), 600)] + rng.normal(0, 3, (600, 2)) * 2 ** -10
    seeds = np.concatenate([near, uniform_seeds(wl, 301, 0, 0)]).astype(np.float32)
    res = _search_both(rt, wl, ev, seeds)
    _, n_conv = _check_search(wl, ev, *res, min_robust=400)  # the oracle finds 447 robust, 179 converged
    assert n_conv >= 150


def test_local_search_hits_beyond_shared_memory(rt):
    # hits past the staged capacity are read from global memory: same results
    wl = WORKLOADS["velo"]
    ev = velo0(0, 1)
    rng = np.random.default_rng(5)
    seeds = (ev.truth[:, :2][rng.integers(0, len(ev.truth), 300)] + rng.normal(0, 2, (300, 2)) * 2 ** -10)
    seeds = seeds.astype(np.float32)
    old = rt.get_option(rt.OPT_LS_SMEM_HITS)
    rt.set_option(rt.OPT_LS_SMEM_HITS, 1000)
    try:
        res = _search_both(rt, wl, ev, seeds)
    finally:
        rt.set_option(rt.OPT_LS_SMEM_HITS, old)
    _check_search(wl, ev, *res, min_robust=250)


def test_local_search_edge_cases(rt):
    wl = WORKLOADS["velo"]
    box = rt.Grid.of(wl)
    seeds = np.array([[0.01, -0.02], [0.6, 0.0], [0.499, 0.3]], np.float32)
    # empty event, single-hit event, an event with one hit on the first seed's line
    e0 = np.zeros((0, 4), np.float32)
    e1 = np.array([[5.0, -3.0, 100.0, 0.0]], np.float32)
    e2 = np.array([[0.01 * 200.0 + 0.02, -0.02 * 200.0, 200.0, 0.0]], np.float32)
    hits = np.concatenate([e0, e1, e2])
    off = np.array([0, 0, 1, 2], np.int64)
    S = np.stack([seeds] * 3)
    th, R, st = rt.local_search(dev(hits), dev(off), 1, dev(S), rt.LsOpts(), box)
    th, R, st = th.cpu().numpy(), R.cpu().numpy(), st.cpu().numpy()
    for e, eh in enumerate([e0, e1, e2]):
        th_o, R_o, st_o, m_o = oracle.local_search(eh, 1, seeds, (0.3, 0.175, 0.05), wl.grid_lo, wl.grid_step,
                                                   wl.grid_n)
        # empty event: R = 0, points unmoved; the seed outside the box is flagged
        if e == 0:
            assert np.all(R[e] == 0) and np.all(th[e] == seeds)
        np.testing.assert_array_equal(st[e][[1]], [2])
        rob = m_o >= 1
        assert np.all(st[e][rob] == st_o[rob])
        assert np.all(np.abs(R[e][rob] - R_o[rob]) <= R_REL * R_o[rob] + R_ABS)
    # malformed offsets (decreasing, beyond n_hits) are clamped, not read out of bounds
    bad = np.array([0, 2, 1, 99], np.int64)
    th, R, st = rt.local_search(dev(hits), dev(bad), 1, dev(S), rt.LsOpts(), box)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(R.cpu().numpy()))


# ---------------------------------------------------------------------------
# extraction: exact on identical inputs
# ---------------------------------------------------------------------------

def test_extract_tracks_exact_on_oracle_points(rt):
    wl = WORKLOADS["velo"]
    E = 3
    thetas, Rs, sts = [], [], []
    for e in range(E):
        ev = velo0(7, e)
        rng = np.random.default_rng(e)
        near = ev.truth[:, :2][rng.integers(0, len(ev.truth), 600)] + rng.normal(0, 4, (600, 2)) * 2 ** -10
        seeds = np.concatenate([near, uniform_seeds(wl, 424, 7, e)]).astype(np.float32)
        th_o, R_o, st_o, m_o = oracle.local_search(ev.hits, 1, seeds, wl.sigma_schedule, wl.grid_lo, wl.grid_step,
                                                   wl.grid_n)
        thetas.append(th_o.astype(np.float32))
        Rs.append(R_o.astype(np.float32))
        sts.append(st_o)
    th, R, st = np.stack(thetas), np.stack(Rs), np.stack(sts)
    R0 = float(np.float32(wl.R0))
    K = 512
    out = rt.extract_tracks(dev(th), dev(R), dev(st), rt.Grid.of(wl), R0, wl.merge_cells, K)
    n_tr = out["n_tracks"].cpu().numpy()
    src = out["track_src"].cpu().numpy()
    for e in range(E):
        keep = oracle.extract_tracks(th[e], R[e], st[e], wl.grid_lo, wl.grid_step, wl.grid_n, R0, wl.merge_cells)
        assert len(keep) >= 10
        assert n_tr[e] == len(keep)
        assert src[e, :len(keep)].tolist() == keep.tolist()
        np.testing.assert_array_equal(out["tracks"].cpu().numpy()[e, :len(keep)], th[e][keep])


def test_extract_tracks_exact_random_clusters_and_edges(rt):
    # dense random clusters with exact R ties, points on the box edges and on
    # the merge distance, n_valid, K truncation and an all-rejected event
    rng = np.random.default_rng(11)
    lo, step, n = (-1.0, -1.0), (2 ** -6, 2 ** -6), (128, 128)
    E, P = 6, 3000
    centres = rng.uniform(-1.0, 1.0, (E, 60, 2))
    th = centres[np.arange(E)[:, None], rng.integers(0, 60, (E, P))] + rng.normal(0, 2 * step[0], (E, P, 2))
    th = np.round(th / (step[0] / 8)) * (step[0] / 8)  # on a lattice: exact merge-distance hits
    th[:, :20, 0] = -1.0                               # on the lower box edge (inside)
    th[:, 20:40, 1] = 1.0                              # on the upper box edge (outside)
    R = rng.integers(0, 40, (E, P)).astype(np.float32)
    st = rng.integers(0, 4, (E, P)).astype(np.uint8)
    R[3] = 0.0
    th = th.astype(np.float32)
    # events 2, 4 and 5 keep at most 64 candidates (one warp decides them)
    nv = np.array([P, 2500, 17, P, 100, 140], np.int32)
    n_cand = []
    for K in (100, 8):
        out = rt.extract_tracks(dev(th), dev(R), dev(st), rt.Grid(lo, step, n), 5.0, 2.0, K, n_valid=dev(nv))
        n_tr = out["n_tracks"].cpu().numpy()
        src = out["track_src"].cpu().numpy()
        for e in range(E):
            m = nv[e]
            keep = oracle.extract_tracks(th[e, :m], R[e, :m], st[e, :m], lo, step, n, 5.0, 2.0)
            assert n_tr[e] == len(keep)
            k = min(K, len(keep))
            assert src[e, :k].tolist() == keep[:k].tolist()
        assert n_tr[0] > K and n_tr[3] == 0
    for e in (4, 5):
        m = nv[e]
        ok = (st[e, :m] <= 1) & (R[e, :m] >= 5.0) & np.all((th[e, :m] >= -1.0) & (th[e, :m] < 1.0), axis=1)
        n_cand.append(int(ok.sum()))
    assert 32 < n_cand[0] <= 64 and 32 < n_cand[1] <= 64, n_cand  # both halves of the warp's ranks
    assert n_tr[4] > 8  # truncation at K inside the one-warp path


# ---------------------------------------------------------------------------
# whole paths at the single-event workload's full size
# ---------------------------------------------------------------------------

def _search_sets(rt, wl, ev, seeds):
    """One event's search at full size through the CUDA path and the oracle,
    both extracted; the found-track sets compared up to near-ties
    (compare_track_sets).  Ties: seeds with an oracle decision within
    tolerance, or whose path the oracle's perturbed replicas do not pin to the
    comparison tolerance."""
    th_g, R_g, st_g, th_o, R_o, st_o, m_o = _search_both(rt, wl, ev, seeds)
    R0 = float(np.float32(wl.R0))
    box = (wl.grid_lo, wl.grid_step, wl.grid_n)
    tr = rt.extract_tracks(dev(th_g[None].astype(np.float32)), dev(R_g[None].astype(np.float32)), dev(st_g[None]),
                           rt.Grid.of(wl), R0, wl.merge_cells, 4096)
    ng = tr["n_tracks"].item()
    src_g = tr["track_src"].cpu().numpy()[0, :ng]
    keep_o = oracle.extract_tracks(th_o, R_o, st_o, *box, R0, wl.merge_cells)
    cand_o = candidates(th_o, R_o, st_o, *box, R0)
    cand_g = candidates(th_g, R_g, st_g, *box, R0)
    # near-R0 items count as candidates for the component analysis on both sides
    near0 = np.abs(R_o - R0) <= R_REL * np.abs(R_o) + R_ABS
    tol = search_tolerance(_converged_2d(ev, wl), th_o, cand_o | cand_g, wl.grid_step)
    sig = tuple(wl.sigma_schedule)

    def run(pt):
        return oracle.local_search(ev.hits, wl.model, seeds, sig, *box, perturb=pt)

    stable, _, _ = oracle.path_conditioning(run, (th_o, R_o, st_o, m_o), tol, keys=oracle.PERTURB_KEYS[:8])
    tie = (m_o < 1.0) | ~stable
    comps, tied, compared = compare_track_sets(th_o, R_o, cand_o | (near0 & (st_o <= 1)), th_g, R_g, cand_g, tie,
                                               keep_o, src_g, tol, wl.grid_step, wl.merge_cells, R0=R0)
    return len(keep_o), ng, comps, tied, compared


@pytest.mark.parametrize("wl_name,vertex", [("toy2d", None), ("velo", "smeared"), ("velo", "origin")])
def test_search_and_extract_full_size_track_sets(rt, wl_name, vertex):
    # the single-event search at its full size (256 seeds on the toy, 8192 on
    # the VELO-like event), event seeds 0-7: track sets equal up to near-ties
    wl = WORKLOADS[wl_name]
    kw = {"vertex_sigma": (0, 0, 0)} if vertex == "origin" else {}
    total = 0
    for eid in range(8):
        ev = make_event(wl, 0, eid, **kw)
        seeds = uniform_seeds(wl, wl.n_seeds, 0, eid)
        n_o, n_g, comps, tied, compared = _search_sets(rt, wl, ev, seeds)
        total += compared
    # the smeared-vertex events' slope-model searches find almost nothing (a
    # two-slope line through the origin cannot fit a displaced vertex)
    assert total >= (40 if wl_name == "toy2d" else (1 if vertex == "smeared" else 200)), total


def _grid_sets(rt, wl, ev_list, R_g_all, mx, tr, Ro_list):
    """Grid maxima and extracted grid tracks of several events against the
    oracle's: the maxima sets may differ only at cells whose oracle margin
    (distance of R to R0 or to a neighbour's R) is within twice R's
    tolerance; the extracted sets are compared up to near-ties."""
    n0, n1 = wl.grid_n
    c0, c1 = oracle.cell_centres(wl.grid_lo, wl.grid_step, wl.grid_n)
    R0 = float(np.float32(wl.R0))
    compared = 0
    for e, ev in enumerate(ev_list):
        R_o = Ro_list[e]
        nm = int(mx["n_max"][e])
        idx_g = mx["max_idx"][e, :nm].cpu().numpy().astype(np.int64)
        exp, cnt, margin = oracle.grid_maxima(R_o, wl.R0, with_margin=True)
        tolc = (R_REL * R_o + R_ABS).reshape(-1)
        diff = set(idx_g.tolist()) ^ set(exp.tolist())
        for c in diff:
            assert margin.reshape(-1)[c] <= 2 * tolc[c], (e, c)
        cells = np.array(sorted(set(idx_g.tolist()) | set(exp.tolist())), dtype=np.int64)
        pos = np.stack([c0[cells % n0], c1[cells // n0]], 1)
        Rg = R_g_all[e].reshape(-1)[cells].astype(np.float64)
        Ro = R_o.reshape(-1)[cells]
        cand_o = np.isin(cells, exp)
        cand_g = np.isin(cells, idx_g)
        tie = np.array([margin.reshape(-1)[c] <= 2 * tolc[c] for c in cells], dtype=bool)
        keep_o = oracle.extract_tracks(pos[cand_o], Ro[cand_o], None, wl.grid_lo, wl.grid_step, wl.grid_n, R0,
                                       wl.merge_cells)
        keep_o = np.flatnonzero(cand_o)[keep_o]
        nt = int(tr["n_tracks"][e])
        src = tr["track_src"][e, :nt].cpu().numpy()
        keep_g = np.searchsorted(cells, idx_g[src])
        tol = np.full((len(cells), 2), 1e-9) * np.asarray(wl.grid_step)
        _, _, k = compare_track_sets(pos, Ro, cand_o, pos, Rg, cand_g, tie, keep_o, keep_g, tol, wl.grid_step,
                                     wl.merge_cells, R0=R0)
        compared += k
    return compared


@pytest.mark.parametrize("wl_name", ["toy2d", "velo"])
def test_grid_scan_full_size_track_sets(rt, wl_name):
    # the whole grid (200^2 toy, 1024^2 VELO-like) of event seeds 0-7 against
    # the oracle's whole grid: maxima and extracted tracks
    wl = WORKLOADS[wl_name]
    evs = [make_event(wl, 0, eid) for eid in range(8)]
    K, KT = 8192, 4096
    compared = 0
    for ev in evs:
        off = np.array([0, ev.n_hits], np.int64)
        out = rt.grid_scan(dev(ev.hits), dev(off), wl.model, rt.Grid.of(wl), wl.sigma_grid, wl.R0, K, store_R=True)
        nm = out["n_max"].item()
        assert 0 < nm <= K
        tr = rt.extract_tracks(out["max_theta"], out["max_R"], None, rt.Grid.of(wl), float(np.float32(wl.R0)),
                               wl.merge_cells, KT, n_valid=out["n_max"])
        R_o = oracle.grid_response(ev.hits, wl.model, wl.grid_lo, wl.grid_step, wl.grid_n, wl.sigma_grid)
        compared += _grid_sets(rt, wl, [ev], out["R"].cpu().numpy(), out, tr, [R_o])
    assert compared >= (50 if wl_name == "toy2d" else 150), compared


# ---------------------------------------------------------------------------
# beyond the shared-memory sizes: more points than 8192 per event, events
# with more hits than a CTA stages
# ---------------------------------------------------------------------------

def test_extract_tracks_exact_beyond_8192_points(rt):
    rng = np.random.default_rng(21)
    lo, step, n = (-1.0, -1.0), (2 ** -7, 2 ** -7), (256, 256)
    E, P = 3, 20000
    centres = rng.uniform(-1.0, 1.0, (E, 300, 2))
    th = centres[np.arange(E)[:, None], rng.integers(0, 300, (E, P))] + rng.normal(0, 2 * step[0], (E, P, 2))
    th = (np.round(th / (step[0] / 8)) * (step[0] / 8)).astype(np.float32)
    R = rng.integers(0, 60, (E, P)).astype(np.float32)
    st = rng.integers(0, 3, (E, P)).astype(np.uint8)
    nv = np.array([P, 15000, 9000], np.int32)
    for K in (4000, 50):
        out = rt.extract_tracks(dev(th), dev(R), dev(st), rt.Grid(lo, step, n), 5.0, 2.0, K, n_valid=dev(nv))
        n_tr = out["n_tracks"].cpu().numpy()
        src = out["track_src"].cpu().numpy()
        for e in range(E):
            m = nv[e]
            keep = oracle.extract_tracks(th[e, :m], R[e, :m], st[e, :m], lo, step, n, 5.0, 2.0)
            assert n_tr[e] == len(keep) > 100
            k = min(K, len(keep))
            assert src[e, :k].tolist() == keep[:k].tolist()


def test_search_and_extract_on_an_event_beyond_25k_hits_with_12288_points(rt):
    # a high-multiplicity event with 1200 tracks (~33k hits: more than a CTA
    # stages) and 12288 starting points around its tracks (more than the
    # shared-memory extraction holds) through the batched search and the
    # workspace extraction: found-track set equal to the oracle's up to near-ties
    from paper_1709_08610_gb300.pipeline import BatchTracker
    wl = WORKLOADS["velo_stress"]
    ev = make_event(wl, 23, 0, vertex_sigma=(0, 0, 0), n_tracks=1200)
    assert ev.n_hits > 25000
    rng = np.random.default_rng(8)
    S = 12288
    seeds = (ev.truth[:, :2][rng.integers(0, len(ev.truth), S)] + rng.normal(0, 3, (S, 2)) * wl.grid_step[0])
    seeds = seeds.astype(np.float32)
    box = rt.Grid.of(wl)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    tr = BatchTracker(1, ev.n_hits, S, box, opts, wl.R0, max_tracks=4096, sort_seeds=True, seeds_per_warp=2,
                      warps=32, smem_hits=12288)
    tr.load(ev.hits, np.array([0, ev.n_hits], np.int64), seeds[None])
    tr.step()
    torch.cuda.synchronize()
    th_g, R_g, st_g = (x.cpu().numpy() for x in tr.search_out)
    th_g, R_g = th_g.astype(float), R_g.astype(float)
    ss = tr.seeds_sorted.cpu().numpy()
    nt = int(tr.tracks["n_tracks"][0])
    assert 0 < nt <= 4096
    src = tr.tracks["track_src"][0, :nt].cpu().numpy()
    R0 = float(np.float32(wl.R0))
    boxa = (wl.grid_lo, wl.grid_step, wl.grid_n)

    def run(pt):
        return oracle.local_search(ev.hits, 1, ss, wl.sigma_schedule, *boxa, perturb=pt)

    th_o, R_o, st_o, m_o = base = run(None)
    keep_o = oracle.extract_tracks(th_o, R_o, st_o, *boxa, R0, wl.merge_cells)
    cand_o = candidates(th_o, R_o, st_o, *boxa, R0)
    cand_g = candidates(th_g, R_g, st_g, *boxa, R0)
    assert cand_g.sum() > 8192  # the extraction's candidates exceed shared memory
    tol = search_tolerance(_converged_2d(ev, wl), th_o, cand_o | cand_g, wl.grid_step)
    stable, _, _ = oracle.path_conditioning(run, base, tol, keys=oracle.PERTURB_KEYS[:4])
    near0 = np.abs(R_o - R0) <= R_REL * np.abs(R_o) + R_ABS
    _, _, compared = compare_track_sets(th_o, R_o, cand_o | (near0 & (st_o <= 1)), th_g, R_g, cand_g,
                                        (m_o < 1.0) | ~stable, keep_o, src, tol, wl.grid_step, wl.merge_cells, R0=R0)
    assert compared >= 500, compared
