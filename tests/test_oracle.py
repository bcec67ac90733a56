"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these tests re-types the oracle's formulas: they use hand-worked
examples (tests/golden), closed forms, finite differences, least squares
(numpy.linalg.lstsq), library local-maximum filters (scipy.ndimage) and brute
force, chosen so that a dropped term, a flipped sign, a wrong index or a
transposed operand anywhere in the oracle breaks at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from synth import WORKLOADS, make_event, make_toy2d_event, close_tracks_event, uniform_seeds
from synth.events import TOY_PLANES_X

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))
E1, E4 = math.exp(-1.0), math.exp(-4.0)


def _c(coeffs):
    return coeffs[0] + coeffs[1] * E1 + coeffs[2] * E4


# --------------------------------------------------------------------------
# Eq. 1 and its derivatives
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", GOLD["response"], ids=lambda c: c["name"])
def test_worked_example_response_grad_hess(case):
    hits = np.array(case["hits"], dtype=np.float32)
    out = oracle.rgh(hits, case["model"], case["theta"], case["sigma"])
    assert out["R"] == pytest.approx(_c(case["R"]), rel=1e-14)
    for a in range(2):
        assert out["grad"][a] == pytest.approx(_c(case["grad"][a]), rel=1e-12, abs=1e-9)
        for b in range(2):
            assert out["hess"][a, b] == pytest.approx(_c(case["hess"][a][b]), rel=1e-12, abs=1e-6)
    # R alone agrees with R from the derivative routine
    assert oracle.response(hits, case["model"], [case["theta"]], case["sigma"])[0] == pytest.approx(out["R"], rel=1e-15)


@pytest.mark.parametrize("model", [0, 1])
def test_single_hit_closed_form(model):
    # one hit displaced by exactly d in the measured coordinate: R = exp(-d^2 / sigma^2)
    sigma = 0.125
    for d in [0.0, 0.0625, 0.125, 0.25, 0.5]:
        if model == 0:
            hits = np.array([[3.0, 0.25 * 3.0 - 0.5 + d, 0, 0]], np.float32)
            th = [0.25, -0.5]
        else:
            hits = np.array([[0.25 * 64.0 + d, -0.5 * 64.0, 64.0, 0]], np.float32)
            th = [0.25, -0.5]
        R = oracle.response(hits, model, [th], sigma)[0]
        assert R == pytest.approx(math.exp(-(d / sigma) ** 2), rel=1e-14)


@pytest.mark.parametrize("model", [0, 1])
def test_all_hits_on_pattern_gives_R_equal_N_and_closed_form_hessian(model):
    # hits exactly on the pattern: R = N, grad = 0, Hess = -(2 / sigma^2) sum J^T J
    th = np.array([0.25, -0.125])
    sigma = 0.3
    if model == 0:
        xs = np.arange(1, 11, dtype=np.float64)
        hits = np.stack([xs, th[0] * xs + th[1], 0 * xs, 0 * xs], 1).astype(np.float32)
        JtJ = np.array([[np.sum(xs * xs), np.sum(xs)], [np.sum(xs), len(xs)]])
    else:
        zs = np.array([-128.0, -32.0, 16.0, 64.0, 256.0, 512.0])
        hits = np.stack([th[0] * zs, th[1] * zs, zs, 0 * zs], 1).astype(np.float32)
        JtJ = np.eye(2) * np.sum(zs * zs)
    out = oracle.rgh(hits, model, th, sigma)
    assert out["R"] == len(hits)
    np.testing.assert_array_equal(out["grad"], [0.0, 0.0])
    np.testing.assert_allclose(out["hess"], -(2.0 / sigma ** 2) * JtJ, rtol=1e-14)


@pytest.mark.parametrize("wl_name", ["toy2d", "velo"])
def test_bounds_and_permutation_invariance(wl_name):
    wl = WORKLOADS[wl_name]
    ev = make_event(wl, 7, 3)
    rng = np.random.default_rng(0)
    th = np.asarray(wl.grid_lo) + rng.uniform(0, 1, (64, 2)) * np.asarray(wl.grid_n) * np.asarray(wl.grid_step)
    R = oracle.response(ev.hits, wl.model, th, wl.sigma_grid)
    assert np.all(R >= 0) and np.all(R <= ev.n_hits)
    perm = rng.permutation(ev.n_hits)
    R2 = oracle.response(ev.hits[perm], wl.model, th, wl.sigma_grid)
    np.testing.assert_allclose(R2, R, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("wl_name", ["toy2d", "velo"])
def test_gradient_and_hessian_match_central_differences(wl_name):
    wl = WORKLOADS[wl_name]
    ev = make_event(wl, 1, 0, **({"vertex_sigma": (0, 0, 0)} if wl.model == 1 else {}))
    sigma = wl.sigma_schedule[0]
    # points near true tracks, where R and its derivatives are far from underflow
    rng = np.random.default_rng(5)
    pts = ev.truth[:6, :2] + rng.normal(0, 0.5, (6, 2)) * np.asarray(wl.grid_step)
    for th in pts:
        out = oracle.rgh(ev.hits, wl.model, th, sigma)
        h = 1e-4 * np.asarray(wl.grid_step)
        g_fd = np.zeros(2)
        H_fd = np.zeros((2, 2))
        for a in range(2):
            ea = np.zeros(2)
            ea[a] = h[a]
            Rp = oracle.response(ev.hits, wl.model, [th + ea], sigma)[0]
            Rm = oracle.response(ev.hits, wl.model, [th - ea], sigma)[0]
            g_fd[a] = (Rp - Rm) / (2 * h[a])
            gp = oracle.rgh(ev.hits, wl.model, th + ea, sigma)["grad"]
            gm = oracle.rgh(ev.hits, wl.model, th - ea, sigma)["grad"]
            H_fd[:, a] = (gp - gm) / (2 * h[a])
        scale_g = out["grad_abs"].sum()
        scale_H = out["hess_abs"].sum()
        assert np.max(np.abs(g_fd - out["grad"])) <= 1e-6 * scale_g
        assert np.max(np.abs(H_fd - out["hess"])) <= 1e-6 * scale_H
        assert out["hess"][0, 1] == out["hess"][1, 0]


# --------------------------------------------------------------------------
# Grid maxima and cluster selection
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", GOLD["grid_maxima"], ids=lambda c: "R0=%g" % c["R0"])
def test_worked_example_grid_maxima(case):
    R = np.array(case["R"], dtype=np.float64)
    idx = oracle.grid_maxima(R, case["R0"])
    assert idx.tolist() == case["expected"]


def test_grid_maxima_agree_with_library_maximum_filter():
    ndi = pytest.importorskip("scipy.ndimage")
    wl = WORKLOADS["velo"]
    ev = make_event(wl, 0, 4, vertex_sigma=(0, 0, 0))
    # a 192 x 160 window of the slope grid (continuous data: no exact ties)
    lo = (wl.grid_lo[0] + 400 * wl.grid_step[0], wl.grid_lo[1] + 420 * wl.grid_step[1])
    R = oracle.grid_response(ev.hits, wl.model, lo, wl.grid_step, (192, 160), wl.sigma_grid)
    assert len(np.unique(R)) == R.size
    mx = ndi.maximum_filter(R, size=3, mode="constant", cval=-np.inf)
    expect = np.flatnonzero((R == mx) & (R >= 3.0))
    assert len(expect) >= 3
    assert oracle.grid_maxima(R, 3.0).tolist() == expect.tolist()


@pytest.mark.parametrize("case", GOLD["extract_tracks"], ids=lambda c: "m=%g" % c["merge_cells"])
def test_worked_example_extract_tracks(case):
    b = case["box"]
    keep = oracle.extract_tracks(np.array(case["theta"]), np.array(case["R"], float), np.array(case["status"]),
                                 b["lo"], b["step"], b["n"], case["R0"], case["merge_cells"])
    assert keep.tolist() == case["expected"]


def test_extract_tracks_invariants_on_random_points():
    rng = np.random.default_rng(3)
    lo, step, n = (-1.0, -1.0), (0.0625, 0.0625), (32, 32)
    th = rng.uniform(-1.1, 1.1, (600, 2))
    R = rng.integers(0, 50, 600).astype(float)  # many exact ties in R
    st = rng.integers(0, 4, 600).astype(np.uint8)
    m = 2.0
    keep = oracle.extract_tracks(th, R, st, lo, step, n, 10.0, m)
    hi = np.asarray(lo) + np.asarray(n) * np.asarray(step)
    cand = np.flatnonzero((st <= 1) & (R >= 10.0) & np.all((th >= lo) & (th < hi), axis=1))
    assert set(keep.tolist()) <= set(cand.tolist())
    dist = lambda i, j: np.max(np.abs(th[i] - th[j]) / np.asarray(step))
    # kept points are pairwise at least m apart and visited by (R desc, index asc)
    for a in range(len(keep)):
        for b in range(a + 1, len(keep)):
            assert dist(keep[a], keep[b]) >= m
            assert (R[keep[a]], -keep[a]) > (R[keep[b]], -keep[b])
    # every rejected candidate lies within m of a kept point ranked before it
    for c in set(cand.tolist()) - set(keep.tolist()):
        assert any(dist(c, k) < m and (R[k], -k) > (R[c], -c) for k in keep)


# --------------------------------------------------------------------------
# Local search: truncated Newton (Section 3) inside Algorithm 1
# --------------------------------------------------------------------------

def test_large_sigma_newton_step_lands_on_least_squares_fit_toy():
    # For residuals r << sigma, R ~ N - sum r^2 / sigma^2 is quadratic, so a
    # full Newton step lands on the least-squares line fit up to O(delta (r/sigma)^2).
    # The start is chosen so the CG forcing test needs the second iteration
    # (gradient with equal components along both eigenvectors of J^T J).
    ev = make_toy2d_event(11, 0, n_tracks=1, noise_frac=0.0)
    x = ev.hits[:, 0].astype(np.float64)
    y = ev.hits[:, 1].astype(np.float64)
    A = np.stack([x, np.ones_like(x)], 1)
    ls = np.linalg.lstsq(A, y, rcond=None)[0]
    w, V = np.linalg.eigh(A.T @ A)
    sigma = 1.0
    for c in (0.04, -0.06, 0.08):
        start = ls + c * V[:, 0] + c * (w[0] / w[1]) * V[:, 1]
        s32 = np.array([start], np.float32)
        th, R, st, m = oracle.local_search(ev.hits, 0, s32, [sigma], (-1, -1), (1e-3, 1e-3), (2000, 2000),
                                           step_cap_cells=1e9)
        assert st[0] == 0
        delta = np.max(np.abs(s32[0] - ls))
        rmax = np.max(np.abs(A @ s32[0].astype(float) - y))
        assert np.max(np.abs(th[0] - ls)) < 2.0 * delta * (rmax / sigma) ** 2


def test_large_sigma_newton_step_lands_on_least_squares_fit_velo():
    # Same limit for the slope model: the least-squares slope per axis is
    # sum(z x) / sum(z^2); J^T J = sum z^2 I is isotropic.
    ev = make_event(WORKLOADS["velo"], 12, 0, n_tracks=1, noise_frac=0.0, vertex_sigma=(0, 0, 0))
    h = ev.hits.astype(np.float64)
    ls = np.array([np.sum(h[:, 2] * h[:, 0]), np.sum(h[:, 2] * h[:, 1])]) / np.sum(h[:, 2] ** 2)
    sigma = 5.0
    for off in ((1e-3, -5e-4), (-8e-4, 2e-4)):
        s32 = np.array([ls + np.asarray(off)], np.float32)
        th, R, st, m = oracle.local_search(ev.hits, 1, s32, [sigma], (-0.5, -0.5), (2 ** -10,) * 2, (1024, 1024),
                                           step_cap_cells=1e9)
        assert st[0] == 0
        delta = np.max(np.abs(s32[0] - ls))
        r = np.concatenate([h[:, 0] - s32[0, 0] * h[:, 2], h[:, 1] - s32[0, 1] * h[:, 2]])
        assert np.max(np.abs(th[0] - ls)) < 2.0 * delta * (np.max(np.abs(r)) / sigma) ** 2


def test_newton_converges_quadratically_on_noiseless_track():
    # Noiseless single VELO track through the origin.  Inside the peak (start
    # at ~0.1 of its width w = sigma / z_rms) each truncated Newton step
    # satisfies err_next <= 2 err^2 / w (a Gaussian peak is even in fact
    # cubic there); 1e-9 covers the float32 rounding of the hits.
    zs = np.array([-300.0 + 42.0 * p for p in range(26)])
    t = np.array([0.07, -0.045])
    hits = np.stack([t[0] * zs, t[1] * zs, zs, 0 * zs], 1).astype(np.float32)
    sigma = 0.3
    w = sigma / math.sqrt(np.mean(zs ** 2))
    seeds = np.array([t + np.array([0.08, -0.05]) * w], np.float32)
    errs = [np.max(np.abs(seeds[0] - t))]
    for q in range(1, 4):
        th, R, st, m = oracle.local_search(hits, 1, seeds, [sigma] * q, (-0.5, -0.5), (2 ** -10,) * 2, (1024, 1024))
        assert st[0] == 0
        errs.append(np.max(np.abs(th[0] - t)))
    for k in range(3):
        assert errs[k + 1] <= 2.0 * errs[k] ** 2 / w + 1e-9
    assert errs[1] < 0.05 * errs[0]
    assert errs[3] < 1e-8


@pytest.mark.parametrize("c1", [1e-4, 0.3, 0.6])
def test_negative_curvature_takes_capped_steepest_ascent_and_armijo_by_brute_force(c1):
    # one hit; a start in the convex tail of its Gaussian has d^T H d > 0 along g,
    # so the direction is g itself, capped to step_cap_cells; the accepted step is
    # the first of 1, 1/2, 1/4 ... passing the sufficient-increase test.
    sigma = 0.25
    hits = np.array([[0.0, 0.0, 0.0, 0.0]], np.float32)  # toy: y = 0 at x = 0 -> constrains beta only
    hits = np.array([[1.0, 0.0, 0.0, 0.0], [2.0, 0.0, 0.0, 0.0]], np.float32)
    start = np.array([0.0, 0.3], np.float64)  # beta = 0.3 > sigma / sqrt(2): convex tail
    step = (2 ** -8, 2 ** -8)
    out = oracle.rgh(hits, 0, start, sigma)
    g = out["grad"]
    assert g @ out["hess"] @ g > 0
    cap = 4.0
    p = g * cap / np.max(np.abs(g) / np.asarray(step))
    R0 = out["R"]
    t_expect = None
    for h in range(9):
        t = 0.5 ** h
        Rt = oracle.response(hits, 0, [start + t * p], sigma)[0]
        if Rt >= R0 + c1 * t * (g @ p):
            t_expect = t
            break
    assert t_expect is not None
    th, R, st, m = oracle.local_search(hits, 0, np.array([start], np.float32), [sigma], (-1, -1), step, (512, 512),
                                       step_cap_cells=cap, c1=c1)
    np.testing.assert_allclose(th[0], start.astype(np.float32).astype(float) + t_expect * p, rtol=0, atol=1e-12)


@pytest.mark.parametrize("c1", [1e-4, 0.3, 0.6, 0.9])
def test_newton_overshoot_backtracks_by_armijo_brute_force(c1):
    # One VELO hit, seed offset along t_x only: g = (g0, 0) and H is diagonal,
    # so the first CG iteration is the exact 1D Newton step p = (-g0/H00, 0).
    # From 0.3 peak widths the step overshoots (increase ratio ~0.41), so the
    # accepted t depends on c1; the expected t is found by brute force.
    hits = np.array([[12.5, -25.0, 100.0, 0.0]], np.float32)
    sigma = 0.25
    w = sigma / 100.0
    start = np.array([0.125 + 0.3 * w, -0.25])
    s32 = np.array([start], np.float32)
    th0 = s32[0].astype(np.float64)
    out = oracle.rgh(hits, 1, th0, sigma)
    g, H = out["grad"], out["hess"]
    assert g[1] == 0 and H[0, 1] == 0 and H[0, 0] < 0
    p = np.array([-g[0] / H[0, 0], 0.0])
    t_expect = None
    for h in range(9):
        t = 0.5 ** h
        if oracle.response(hits, 1, [th0 + t * p], sigma)[0] >= out["R"] + c1 * t * (g @ p):
            t_expect = t
            break
    th, R, st, m = oracle.local_search(hits, 1, s32, [sigma], (-0.5, -0.5), (2 ** -10,) * 2, (1024, 1024),
                                       step_cap_cells=1e9, c1=c1)
    if t_expect is None:
        assert st[0] == 1 and np.all(th[0] == th0)
    else:
        assert st[0] == 0
        np.testing.assert_allclose(th[0], th0 + t_expect * p, rtol=0, atol=1e-15)
    assert {1e-4: 1.0, 0.3: 1.0, 0.6: 0.5, 0.9: 0.125}[c1] == t_expect


def _one_velo_hit_start(offset_widths):
    hits = np.array([[12.5, -25.0, 100.0, 0.0]], np.float32)
    sigma = 0.25
    w = sigma / 100.0
    s32 = np.array([[0.125 + offset_widths * w, -0.25]], np.float32)
    return hits, sigma, w, s32, s32[0].astype(np.float64)


def _armijo_t(hits, model, th0, p, sigma, c1, R0, g):
    for h in range(9):
        t = 0.5 ** h
        if oracle.response(hits, model, [th0 + t * p], sigma)[0] >= R0 + c1 * t * (g @ p):
            return t
    return None


@pytest.mark.parametrize("c1", [1e-4, 0.3])
def test_steepest_ascent_takes_the_capped_gradient(c1):
    # Inside the peak (0.3 widths off along t_x, where the truncated Newton
    # direction would be the Newton step) the steepest-ascent update moves
    # along grad R itself, scaled down to the step cap, by the first
    # step length passing the Armijo test (found by brute force).
    hits, sigma, w, s32, th0 = _one_velo_hit_start(0.3)
    step = (2 ** -10, 2 ** -10)
    out = oracle.rgh(hits, 1, th0, sigma)
    g = out["grad"]
    cap = 0.25
    p = g * cap / np.max(np.abs(g) / np.asarray(step))
    t = _armijo_t(hits, 1, th0, p, sigma, c1, out["R"], g)
    assert t is not None
    th, R, st, m = oracle.local_search(hits, 1, s32, [sigma], (-0.5, -0.5), step, (1024, 1024),
                                       step_cap_cells=cap, c1=c1, update=1)
    assert st[0] == 0
    np.testing.assert_allclose(th[0], th0 + t * p, rtol=0, atol=1e-15)
    # the truncated Newton direction differs here (it is -H^-1 g, not along g scaled)
    th_n, _, _, _ = oracle.local_search(hits, 1, s32, [sigma], (-0.5, -0.5), step, (1024, 1024),
                                        step_cap_cells=1e9, c1=c1)
    assert not np.allclose(th_n[0], th[0])


@pytest.mark.parametrize("c1", [1e-4, 0.6])
@pytest.mark.parametrize("model", [0, 1])
def test_modified_newton_is_the_newton_step_where_the_peak_is_concave(c1, model):
    # -Hess R positive definite (inside the peak): no shift, p = -H^-1 g
    # (numpy.linalg.solve), then Armijo by brute force.  Slope model: one hit
    # (diagonal Hessian); 2D toy: a noiseless line seen at x = 1..10, whose
    # Hessian couples the two parameters.
    if model == 1:
        hits, sigma, w, s32, th0 = _one_velo_hit_start(0.3)
        lo, step, n = (-0.5, -0.5), (2 ** -10,) * 2, (1024, 1024)
    else:
        xs = np.arange(1, 11, dtype=np.float64)
        hits = np.stack([xs, 0.1 * xs - 0.2, 0 * xs, 0 * xs], 1).astype(np.float32)
        sigma = 0.05
        s32 = np.array([[0.1 + 0.002, -0.2 - 0.006]], np.float32)
        th0 = s32[0].astype(np.float64)
        lo, step, n = (-1, -1), (2 ** -8,) * 2, (512, 512)
    out = oracle.rgh(hits, model, th0, sigma)
    g, H = out["grad"], out["hess"]
    assert np.all(np.linalg.eigvalsh(-H) > 0)
    assert model == 1 or abs(H[0, 1]) > 0.5 * np.sqrt(H[0, 0] * H[1, 1])
    p = np.linalg.solve(-H, g)
    t = _armijo_t(hits, model, th0, p, sigma, c1, out["R"], g)
    th, R, st, m = oracle.local_search(hits, model, s32, [sigma], lo, step, n,
                                       step_cap_cells=1e9, c1=c1, update=2)
    if t is None:
        assert st[0] == 1 and np.all(th[0] == th0)
    else:
        np.testing.assert_allclose(th[0], th0 + t * p, rtol=0, atol=1e-14)


def test_modified_newton_in_a_rank_one_convex_tail_is_the_capped_gradient_step():
    # One toy hit: Hess R = e (4k^2 r^2 - 2k) v v^T with v = (x, 1), so in the
    # convex tail (4 k r^2 > 2) -H has eigenvalues (mu1 < 0, 0) with g along v.
    # The shift leaves eigenvalue delta along v, so p = g / delta points along
    # g and, being far longer than the cap, is capped: exactly the
    # steepest-ascent update (worked by hand from the definitions).
    hits = np.array([[2.0, 0.0, 0.0, 0.0]], np.float32)
    sigma = 0.25
    start = np.array([[0.05, 0.3]], np.float32)
    th0 = start[0].astype(np.float64)
    out = oracle.rgh(hits, 0, th0, sigma)
    r = 0.0 - th0[0] * 2.0 - th0[1]
    assert 4 * r * r / sigma ** 2 > 2
    step = (2 ** -8, 2 ** -8)
    args = (hits, 0, start, [sigma], (-1, -1), step, (512, 512))
    th2, R2, st2, _ = oracle.local_search(*args, step_cap_cells=2.0, update=2)
    th1, R1, st1, _ = oracle.local_search(*args, step_cap_cells=2.0, update=1)
    np.testing.assert_allclose(th2[0], th1[0], rtol=0, atol=1e-12)
    assert st1[0] == st2[0] == 0 and R2[0] > out["R"]


@pytest.mark.parametrize("update", [1, 2])
def test_alternative_updates_on_a_noiseless_track(update):
    # Modified Newton converges quadratically inside the peak (it is Newton
    # there); steepest ascent converges too, linearly at best.  Both never
    # lower R at a fixed bandwidth (Armijo).
    zs = np.array([-300.0 + 42.0 * p for p in range(26)])
    t = np.array([0.07, -0.045])
    hits = np.stack([t[0] * zs, t[1] * zs, zs, 0 * zs], 1).astype(np.float32)
    sigma = 0.3
    w = sigma / math.sqrt(np.mean(zs ** 2))
    seeds = np.array([t + np.array([0.08, -0.05]) * w], np.float32)
    errs, Rs = [np.max(np.abs(seeds[0] - t))], [oracle.response(hits, 1, seeds.astype(float), sigma)[0]]
    qs = (1, 2, 3) if update == 2 else (2, 4, 8)
    for q in qs:
        th, R, st, m = oracle.local_search(hits, 1, seeds, [sigma] * q, (-0.5, -0.5), (2 ** -10,) * 2, (1024, 1024),
                                           step_cap_cells=0.5, update=update)
        errs.append(np.max(np.abs(th[0] - t)))
        Rs.append(R[0])
    assert all(b >= a * (1 - 1e-15) for a, b in zip(Rs, Rs[1:]))
    if update == 2:
        for k in range(3):
            assert errs[k + 1] <= 2.0 * errs[k] ** 2 / w + 1e-9
        assert errs[3] < 1e-8
    else:
        assert errs[-1] < 0.2 * errs[0]


@pytest.mark.parametrize("update", [0, 1, 2])
def test_every_update_never_lowers_R_at_a_fixed_bandwidth(update):
    wl = WORKLOADS["velo"]
    ev = make_event(wl, 8, 0, vertex_sigma=(0, 0, 0))
    rng = np.random.default_rng(8)
    seeds = (ev.truth[rng.integers(0, len(ev.truth), 200), :2] + rng.normal(0, 3, (200, 2)) * 2 ** -10)
    seeds = seeds.astype(np.float32)
    sigma = 0.175
    R0 = oracle.response(ev.hits, 1, seeds.astype(float), sigma)
    th, R, st, m = oracle.local_search(ev.hits, 1, seeds, [sigma] * 3, wl.grid_lo, wl.grid_step, wl.grid_n,
                                       update=update)
    ok = st <= 1
    assert ok.sum() >= 190
    assert np.all(R[ok] >= R0[ok] * (1 - 1e-12))
    assert np.mean(R[ok] > R0[ok]) > 0.9


def test_search_maxima_agree_with_brute_force_fine_grid():
    # tiny event (3 tracks, ~30 hits): every converged point with R >= R0 is a
    # local maximum of R to within a fine-grid step around it.
    ev = make_toy2d_event(21, 0, n_tracks=3, noise_frac=0.1)
    wl = WORKLOADS["toy2d"]
    sigma = 0.02
    seeds = uniform_seeds(wl, 512, 21, 0)
    # the toy's ridge is ill-conditioned: run 12 rounds of 8 updates each
    for _ in range(12):
        th, R, st, m = oracle.local_search(ev.hits, 0, seeds, [sigma] * 8, wl.grid_lo, wl.grid_step, wl.grid_n)
        seeds = th.astype(np.float32)
    keep = oracle.extract_tracks(th, R, st, wl.grid_lo, wl.grid_step, wl.grid_n, 5.0, 2.0)
    # stationary points among the kept ones (the rest are still crawling along a ridge)
    stat = [k for k in keep if np.all(np.abs(oracle.rgh(ev.hits, 0, th[k], sigma)["grad"]) <= 1e-9 *
                                       oracle.rgh(ev.hits, 0, th[k], sigma)["grad_abs"].sum())]
    assert len(stat) >= 3
    fine = 1e-5
    for k in stat:
        c = th[k]
        lo = (c[0] - 50.5 * fine, c[1] - 50.5 * fine)
        Rf = oracle.grid_response(ev.hits, 0, lo, (fine, fine), (101, 101), sigma)
        i1, i0 = np.unravel_index(np.argmax(Rf), Rf.shape)
        best = np.array([lo[0] + (i0 + 0.5) * fine, lo[1] + (i1 + 0.5) * fine])
        assert np.max(np.abs(best - c)) <= 1.0 * fine
        assert Rf.max() <= R[k] * (1 + 1e-9)


def test_grid_maxima_near_search_maxima():
    # Grid-scan maxima at or above R0 mostly lie within one cell of the
    # continuous maximum the Newton search reaches from them (a discrete
    # maximum on a ridge need not), and the search never lowers R (Armijo).
    wl = WORKLOADS["velo"]
    ev = make_event(wl, 3, 0, vertex_sigma=(0, 0, 0))
    tr = ev.truth[np.argsort(np.abs(ev.truth[:, 0]) + np.abs(ev.truth[:, 1]))[0], :2]
    i0 = int(np.floor((tr[0] - wl.grid_lo[0]) / wl.grid_step[0])) - 48
    i1 = int(np.floor((tr[1] - wl.grid_lo[1]) / wl.grid_step[1])) - 48
    lo = (wl.grid_lo[0] + i0 * wl.grid_step[0], wl.grid_lo[1] + i1 * wl.grid_step[1])
    n = (96, 96)
    R = oracle.grid_response(ev.hits, 1, lo, wl.grid_step, n, wl.sigma_grid)
    idx = oracle.grid_maxima(R, wl.R0)
    assert len(idx) >= 1
    c0, c1 = oracle.cell_centres(lo, wl.grid_step, n)
    gth = np.stack([c0[idx % n[0]], c1[idx // n[0]]], 1)
    th, Rs, st, m = oracle.local_search(ev.hits, 1, gth.astype(np.float32), [wl.sigma_grid] * 8, wl.grid_lo,
                                        wl.grid_step, wl.grid_n)
    d = np.max(np.abs(th - gth) / np.asarray(wl.grid_step), axis=1)
    assert np.all(st <= 1)
    assert np.mean(d <= 1.0) >= 0.9
    assert np.all(Rs >= R.reshape(-1)[idx] * (1 - 1e-12))


# --------------------------------------------------------------------------
# Step 4 of the grid algorithm: parameter estimates refined from the maxima
# --------------------------------------------------------------------------

def _noiseless_track(model, offset_cells):
    """Hits exactly on one track whose parameters sit offset_cells from the
    centre of grid cell (37, 21) of a 64 x 64 window; returns (hits, truth,
    lo, step, n, sigma)."""
    if model == 1:
        wl = WORKLOADS["velo"]
        zs = np.array([-300.0 + 42.0 * p for p in range(26)])
    else:
        wl = WORKLOADS["toy2d"]
        zs = np.asarray(TOY_PLANES_X, dtype=np.float64)
    step = np.asarray(wl.grid_step)
    lo = np.array([wl.grid_lo[0] + 400 * step[0], wl.grid_lo[1] + 40 * step[1]]) if model == 1 else \
        np.array([wl.grid_lo[0] + 70 * step[0], wl.grid_lo[1] + 60 * step[1]])
    n = (64, 64)
    t = lo + (np.array([37, 21]) + 0.5 + np.asarray(offset_cells)) * step
    if model == 1:
        hits = np.stack([t[0] * zs, t[1] * zs, zs, 0 * zs], 1).astype(np.float32)
    else:
        hits = np.stack([zs, t[0] * zs + t[1], 0 * zs, 0 * zs], 1).astype(np.float32)
    return hits, t, lo, step, n, wl.sigma_grid


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("offset", [(0.3, -0.22), (-0.41, 0.12), (0.0, 0.0)])
def test_refinement_recovers_noiseless_track_exactly(model, offset):
    # All hits on one track: R is largest, and equals the number of hits, at
    # the track's parameters (Eq. 1 with s = 0 for every hit).  Slope model:
    # the grid's only maximum is the cell holding the track, offset from its
    # centre by the chosen fraction of a cell.  2D toy: the peak is a ridge
    # (the planes are all at x > 0), on which the grid can have several
    # discrete maxima; the highest is refined.  The refined estimate lands on
    # the track to the float32 rounding of the hits, with R = N.
    hits, t, lo, step, n, sigma = _noiseless_track(model, offset)
    N = hits.shape[0]
    R = oracle.grid_response(hits, model, lo, step, n, sigma)
    idx = oracle.grid_maxima(R, 0.5 * N)
    if model == 1:
        assert list(idx) == [21 * n[0] + 37]
    idx = idx[[int(np.argmax(R.reshape(-1)[idx]))]]
    c = oracle.maxima_centres(idx, lo, step, n)
    if model == 1:
        np.testing.assert_allclose((t - c[0]) / step, offset, atol=1e-9)
    iters = 4 if model == 1 else 8
    th, Rr, st, m = oracle.refine_maxima(hits, model, c, sigma, lo, step, n, iters=iters)
    assert st[0] == 0
    assert np.max(np.abs(th[0] - t)) <= 1e-8
    assert Rr[0] == pytest.approx(N, rel=1e-8)
    if np.any(c[0] != t):
        assert Rr[0] > R.reshape(-1)[idx[0]]


def test_refinement_never_lowers_R_and_respects_the_cap():
    # Every update accepts only an Armijo increase (or stays): R at the
    # refined point >= R at the cell centre; each of the iters steps is at most
    # step_cap_cells cells in the infinity norm.
    wl = WORKLOADS["velo"]
    ev = make_event(wl, 5, 1, vertex_sigma=(0, 0, 0))
    lo = (wl.grid_lo[0] + 448 * wl.grid_step[0], wl.grid_lo[1] + 448 * wl.grid_step[1])
    n = (128, 128)
    R = oracle.grid_response(ev.hits, 1, lo, wl.grid_step, n, wl.sigma_grid)
    idx = oracle.grid_maxima(R, wl.R0)
    assert len(idx) >= 3
    c = oracle.maxima_centres(idx, lo, wl.grid_step, n)
    for iters, cap in ((1, 0.25), (3, 0.5), (4, 1.0)):
        th, Rr, st, m = oracle.refine_maxima(ev.hits, 1, c, wl.sigma_grid, lo, wl.grid_step, n, iters=iters,
                                             step_cap_cells=cap)
        assert np.all(st <= 2)
        assert np.all(Rr >= R.reshape(-1)[idx] * (1 - 1e-12))
        d = np.max(np.abs(th - c) / np.asarray(wl.grid_step), axis=1)
        assert np.all(d <= iters * cap * (1 + 1e-9)), d


def test_refined_maxima_agree_with_brute_force_fine_grid():
    # On a noisy event, each refined estimate that is a converged maximum
    # (negative-definite Hessian) is where R peaks on a fine grid of 1/32
    # cell around it, and R there is not exceeded by any fine-grid point.
    wl = WORKLOADS["velo"]
    ev = make_event(wl, 3, 0, vertex_sigma=(0, 0, 0))
    tr = ev.truth[np.argsort(np.abs(ev.truth[:, 0]) + np.abs(ev.truth[:, 1]))[0], :2]
    i0 = int(np.floor((tr[0] - wl.grid_lo[0]) / wl.grid_step[0])) - 32
    i1 = int(np.floor((tr[1] - wl.grid_lo[1]) / wl.grid_step[1])) - 32
    step = np.asarray(wl.grid_step)
    lo = (wl.grid_lo[0] + i0 * step[0], wl.grid_lo[1] + i1 * step[1])
    n = (64, 64)
    R = oracle.grid_response(ev.hits, 1, lo, step, n, wl.sigma_grid)
    idx = oracle.grid_maxima(R, wl.R0)
    c = oracle.maxima_centres(idx, lo, step, n)
    th, Rr, st, m = oracle.refine_maxima(ev.hits, 1, c, wl.sigma_grid, lo, step, n, iters=4)
    fine = step / 32
    n_conv = 0
    for k in range(len(idx)):
        o = oracle.rgh(ev.hits, 1, th[k], wl.sigma_grid)
        if st[k] != 0 or not np.all(np.linalg.eigvalsh(o["hess"]) < 0):
            continue
        n_conv += 1
        flo = (th[k][0] - 32.5 * fine[0], th[k][1] - 32.5 * fine[1])
        Rf = oracle.grid_response(ev.hits, 1, flo, fine, (65, 65), wl.sigma_grid)
        j1, j0 = np.unravel_index(np.argmax(Rf), Rf.shape)
        best = np.array([flo[0] + (j0 + 0.5) * fine[0], flo[1] + (j1 + 0.5) * fine[1]])
        assert np.all(np.abs(best - th[k]) <= fine * (1 + 1e-9)), (k, (best - th[k]) / fine)
        assert Rf.max() <= Rr[k] * (1 + 1e-9)
    assert n_conv >= 10
    # the estimate of the chosen track is closer to it than its cell centre
    k = int(np.argmin(np.max(np.abs(c - tr) / step, axis=1)))
    assert np.max(np.abs(th[k] - tr)) < np.max(np.abs(c[k] - tr))


def test_figure2_close_tracks_split_and_merge():
    # Figure 2: small sigma splits each smeared track into several clusters of
    # activated units, sigma comparable to the smear resolves the two tracks,
    # large sigma merges them into one cluster.
    ndi = pytest.importorskip("scipy.ndimage")
    lo, step, n = (0.0, -0.2), (2 ** -9, 2 ** -9), (256, 256)
    for seed in range(3):
        ev = close_tracks_event(seed)
        counts = {}
        for sigma in (1e-3, 1e-2, 1e-1):
            R = oracle.grid_response(ev.hits, 0, lo, step, n, sigma)
            counts[sigma] = ndi.label(R >= 0.5 * R.max(), structure=np.ones((3, 3)))[1]
        assert counts[1e-3] > 4
        assert counts[1e-2] == 2
        assert counts[1e-1] == 1


def test_oracle_option_ranges_are_enforced():
    h = np.zeros((1, 4), np.float32)
    with pytest.raises(ValueError):
        oracle.local_search(h, 1, np.zeros((1, 2), np.float32), [0.3], (0, 0), (1, 1), (2, 2), update=3)
    with pytest.raises(ValueError):
        oracle.refine_maxima(h, 1, np.zeros((1, 2)), 0.3, (0, 0), (1, 1), (2, 2), iters=0)
    with pytest.raises(ValueError):
        oracle.local_search4(h, np.zeros((1, 4), np.float32), [0.3] * 9, (1, 1, 1, 1))


# --------------------------------------------------------------------------
# perturbed replicas (path conditioning of the parity tests)
# --------------------------------------------------------------------------

def test_splitmix64_matches_its_published_outputs():
    # SplitMix64 (Steele, Lea & Flood 2014) from state 0: its first outputs
    assert oracle.splitmix64(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = [oracle.perturb_u(k, i, j, c) for k in (1, 2) for i in range(50) for j in range(3) for c in range(6)]
    assert all(-1.0 <= x < 1.0 for x in u)
    assert abs(np.mean(u)) < 0.1 and 0.25 < np.var(u) < 0.42  # ~ U[-1, 1): variance 1/3
    assert oracle.perturb_u(7, 3, 1, 2) == oracle.perturb_u(7, 3, 1, 2) != oracle.perturb_u(8, 3, 1, 2)


@pytest.mark.parametrize("update", [0, 2])
def test_level_zero_replica_is_the_plain_search(update):
    wl = WORKLOADS["velo"]
    ev = make_event(wl, 0, 3, vertex_sigma=(0, 0, 0))
    seeds = uniform_seeds(wl, 64, 0, 3)
    args = (ev.hits, 1, seeds, wl.sigma_schedule, wl.grid_lo, wl.grid_step, wl.grid_n)
    base = oracle.local_search(*args, update=update)
    zero = oracle.local_search(*args, update=update, perturb=(0.0, 12345))
    for a, b in zip(base, zero):
        assert np.array_equal(a, b)
    one = oracle.local_search(*args, update=update, perturb=(1.0, 12345))
    assert not np.array_equal(base[0], one[0])  # the displacement reaches the path


def test_replicas_split_at_a_symmetric_saddle_and_agree_on_a_clean_peak():
    # two noiseless tracks at slopes (+-a, 0): the midpoint (0, 0) has an exactly
    # zero gradient by symmetry, so the unperturbed search stays there, while
    # replicas whose gradient is displaced within its tolerance leave it towards
    # either track - an ill-conditioned path; a seed near one track converges
    # onto it in every replica - a well-conditioned one
    a = 2.0 ** -8
    z = np.array([-300.0 + 42.0 * p for p in range(26)])
    hits = np.concatenate([np.stack([s * a * z, 0 * z, z, 0 * z], 1) for s in (1.0, -1.0)]).astype(np.float32)
    lo, step, n = (-0.5, -0.5), (2.0 ** -10, 2.0 ** -10), (1024, 1024)
    sig = (0.3, 0.175, 0.05)
    seeds = np.array([[0.0, 0.0], [a + 2 ** -12, 2 ** -12]], np.float32)

    def run(pt):
        return oracle.local_search(hits, 1, seeds, sig, lo, step, n, perturb=pt)

    base = run(None)
    # the gradient there is zero up to rounding (~1e-13): the search stays at the saddle
    assert np.max(np.abs(base[0][0])) < 1e-12
    assert np.max(np.abs(base[0][1] - [a, 0.0])) < 1e-6
    stable, ends, sts = oracle.path_conditioning(run, base, 1e-3 * np.asarray(step))
    assert stable.tolist() == [False, True]
    assert np.all(np.max(np.abs(ends[:, 1] - base[0][1]), axis=1) < 1e-6)
    # replicas leave the saddle for both tracks
    assert ends[:, 0, 0].min() < -0.9 * a and ends[:, 0, 0].max() > 0.9 * a
