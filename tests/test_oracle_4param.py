"""Pins of the four-parameter track model of the oracle (x0, y0, t_x, t_y):
the track crosses the layer z at (x0 + t_x z, y0 + t_y z).  Checked against
the pinned two-parameter slope model, translation invariance, closed forms on
the track, central differences and the convergence of the Newton search."""
import math

import numpy as np
import pytest

import oracle
from synth import WORKLOADS, make_event

ZS = np.array([-300.0 + 42.0 * p for p in range(26)])


def _event():
    return make_event(WORKLOADS["velo"], 21, 0, vertex_sigma=(0, 0, 0)).hits


@pytest.mark.parametrize("sigma", [0.05, 0.3])
def test_reduces_to_the_slope_model_through_the_origin(sigma):
    h = _event()
    rng = np.random.default_rng(0)
    for t in rng.uniform(-0.2, 0.2, (5, 2)):
        a = oracle.rgh4(h, [0.0, 0.0, t[0], t[1]], sigma)
        b = oracle.rgh(h, 1, t, sigma)
        assert a["R"] == pytest.approx(b["R"], rel=1e-13, abs=1e-300)
        np.testing.assert_allclose(a["grad"][2:], b["grad"], rtol=1e-12, atol=1e-12 * b["grad_abs"].sum())
        np.testing.assert_allclose(a["hess"][2:, 2:], b["hess"], rtol=1e-12, atol=1e-12 * b["hess_abs"].sum())


def test_an_offset_equals_shifting_the_hits():
    # R(x0, y0, t; hits) = R(0, 0, t; hits - (x0, y0)): the offsets enter only through the residual
    h = _event()[:400].astype(np.float64)
    x0, y0, t = 0.75, -0.5, (0.03, -0.02)
    hs = h.copy()
    hs[:, 0] -= x0
    hs[:, 1] -= y0
    a = oracle.rgh4(h.astype(np.float32), [x0, y0, t[0], t[1]], 0.3)
    # float32 hits on both sides: compare through the shifted float32 copy's exact values
    a2 = oracle.rgh4(hs.astype(np.float32), [0.0, 0.0, t[0], t[1]], 0.3)
    assert a["R"] == pytest.approx(a2["R"], rel=1e-6)
    np.testing.assert_allclose(a["grad"], a2["grad"], rtol=1e-4, atol=1e-6 * a["grad_abs"].sum())


def test_on_the_track_R_is_N_gradient_zero_and_hessian_closed_form():
    # dyadic parameters and integer layers: every hit is exact in float32, so
    # every residual is exactly zero
    x0, y0, tx, ty = 0.375, -0.25, 0.0625, -0.03125
    h = np.stack([x0 + tx * ZS, y0 + ty * ZS, ZS, 0 * ZS], 1).astype(np.float32)
    assert np.all(h[:, 0].astype(np.float64) == x0 + tx * ZS)
    th = np.array([x0, y0, tx, ty])
    sigma = 0.3
    k = 1.0 / sigma ** 2
    out = oracle.rgh4(h, th, sigma)
    z = ZS
    assert out["R"] == len(ZS)
    assert np.all(out["grad"] == 0.0)
    JJ = np.array([[len(z), 0, z.sum(), 0], [0, len(z), 0, z.sum()],
                   [z.sum(), 0, (z * z).sum(), 0], [0, z.sum(), 0, (z * z).sum()]])
    np.testing.assert_allclose(out["hess"], -2 * k * JJ, rtol=1e-13)


def test_gradient_and_hessian_match_central_differences():
    h = _event()
    rng = np.random.default_rng(2)
    sigma = 0.3
    for _ in range(4):
        th = np.array([rng.normal(0, 0.05), rng.normal(0, 0.05), rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1)])
        out = oracle.rgh4(h, th, sigma)
        steps = np.array([1e-5, 1e-5, 2e-8, 2e-8])
        for a in range(4):
            e = np.zeros(4)
            e[a] = steps[a]
            fd = (oracle.response4(h, th + e, sigma) - oracle.response4(h, th - e, sigma)) / (2 * steps[a])
            assert fd == pytest.approx(out["grad"][a], rel=1e-4, abs=1e-6 * out["grad_abs"].sum())
            gp = oracle.rgh4(h, th + e, sigma)["grad"]
            gm = oracle.rgh4(h, th - e, sigma)["grad"]
            np.testing.assert_allclose((gp - gm) / (2 * steps[a]), out["hess"][a], rtol=1e-3,
                                       atol=1e-5 * out["hess_abs"].sum())


def test_search_recovers_a_track_from_a_displaced_vertex():
    # a noiseless track from a vertex at z = 60 mm (x0 = -t_x 60, ...): the slope
    # model through the origin cannot reach R = N, the four-parameter search does.
    # Offsets and slopes are strongly coupled (the layers are not centred on
    # z = 0), so the truncated CG resolves the stiff slope directions first and
    # the offsets a few updates later; R never decreases.
    x0, y0, tx, ty = -0.07 * 60.0 + 0.2, 0.045 * 60.0 - 0.1, 0.07, -0.045
    h = np.stack([x0 + tx * ZS, y0 + ty * ZS, ZS, 0 * ZS], 1).astype(np.float32)
    truth = np.array([x0, y0, tx, ty])
    sigma = 0.3
    scale = (0.05, 0.05, 2 ** -10, 2 ** -10)
    start = truth + np.array([0.02, -0.015, 4e-5, -3e-5])
    seeds = start.astype(np.float32)[None]
    errs = [np.max(np.abs(seeds[0] - truth) / scale)]
    Rs = [oracle.response4(h, seeds[0].astype(np.float64), sigma)]
    for q in range(1, 7):
        th, R, st, m = oracle.local_search4(h, seeds, [sigma] * q, scale)
        assert st[0] == 0
        errs.append(np.max(np.abs(th[0] - truth) / scale))
        Rs.append(R[0])
    assert all(b >= a for a, b in zip(Rs, Rs[1:]))
    assert errs[3] < 0.05 * errs[0] and errs[6] < 1e-5
    assert Rs[-1] == pytest.approx(len(ZS), rel=1e-9)
    # the two-parameter model's best over a fine slope grid stays well below N
    R2 = oracle.grid_response(h, 1, (tx - 0.01, ty - 0.01), (1e-4, 1e-4), (200, 200), sigma)
    assert R2.max() < 0.8 * len(ZS)


def test_search_steps_never_lower_R_at_a_fixed_bandwidth():
    h = _event()
    ev_truth = make_event(WORKLOADS["velo"], 21, 0, vertex_sigma=(0, 0, 0)).truth
    rng = np.random.default_rng(4)
    t = ev_truth[rng.integers(0, len(ev_truth), 100), :2] + rng.normal(0, 2e-3, (100, 2))
    seeds = np.concatenate([rng.normal(0, 0.05, (100, 2)), t], 1).astype(np.float32)
    R0 = np.array([oracle.response4(h, s.astype(np.float64), 0.175) for s in seeds])
    th, R, st, m = oracle.local_search4(h, seeds, [0.175] * 3, (0.05, 0.05, 2 ** -10, 2 ** -10))
    ok = st <= 1
    assert ok.sum() >= 95
    assert np.all(R[ok] >= R0[ok] * (1 - 1e-12))


def test_reference_plane_is_a_reparametrisation():
    # (x0, y0) at z_ref is (x0 - t_x z_ref, y0 - t_y z_ref) at z = 0: same R, and
    # the slope derivatives at fixed reference offsets follow the chain rule
    h = _event()
    th = np.array([0.3, -0.2, 0.04, -0.03])
    zr = 225.0
    th0 = np.array([th[0] - th[2] * zr, th[1] - th[3] * zr, th[2], th[3]])
    a = oracle.rgh4(h, th, 0.3, zref=zr)
    b = oracle.rgh4(h, th0, 0.3)
    assert a["R"] == pytest.approx(b["R"], rel=1e-12)
    # d/dt_x at fixed x0(z_ref) = d/dt_x at fixed x0(0) + d/dx0 * d x0(0)/d t_x = g_t - z_ref g_x0
    np.testing.assert_allclose(a["grad"][:2], b["grad"][:2], rtol=1e-9, atol=1e-9 * b["grad_abs"].sum())
    np.testing.assert_allclose(a["grad"][2:], b["grad"][2:] - zr * b["grad"][:2], rtol=1e-7,
                               atol=1e-9 * b["grad_abs"].sum() * zr)


def test_centred_reference_plane_decouples_and_converges():
    # z_ref = the layers' mean z: sum (z - z_ref) = 0 on a full track, so the
    # Hessian on the track is block-diagonal.  In units of about one peak width
    # per parameter the scaled Newton-CG moves offsets and slopes together;
    # its forcing tolerance (1/2 of |g| while |g| > 1/4) makes the early steps
    # inexact, so the error falls geometrically (here by 0.63, 0.30, 0.30, 0.14,
    # ... per update) before the last steps land on the track
    zr = float(ZS.mean())
    x0, y0, tx, ty = 0.375, -0.25, 0.0625, -0.03125
    h = np.stack([x0 + tx * (ZS - zr), y0 + ty * (ZS - zr), ZS, 0 * ZS], 1).astype(np.float32)
    out = oracle.rgh4(h, [x0, y0, tx, ty], 0.3, zref=zr)
    assert out["R"] == len(ZS)
    assert abs(out["hess"][0, 2]) <= 1e-12 * abs(out["hess"][2, 2])
    assert abs(out["hess"][1, 3]) <= 1e-12 * abs(out["hess"][3, 3])
    scale = (0.25, 0.25, 2 ** -10, 2 ** -10)
    start = np.array([[x0 + 0.04, y0 - 0.03, tx + 6e-4, ty - 5e-4]], np.float32)
    errs = [np.max(np.abs(start[0] - [x0, y0, tx, ty]) / scale)]
    for q in range(1, 9):
        th, R, st, m = oracle.local_search4(h, start, [0.3] * q, scale, zref=zr)
        assert st[0] == 0
        errs.append(np.max(np.abs(th[0] - [x0, y0, tx, ty]) / scale))
    assert all(b <= 0.7 * a for a, b in zip(errs[:6], errs[1:7]))
    assert errs[8] < 1e-4


# --------------------------------------------------------------------------
# starting points from hit pairs, and four-parameter cluster / select
# --------------------------------------------------------------------------

def _axis_event():
    """Five noiseless tracks from points on the z axis, with well separated
    azimuths, seen on two layers, plus three noise hits on them."""
    za, zb = 500.0, 700.0
    vz = np.array([-40.0, 0.0, 25.0, 60.0, -80.0])
    phi = np.array([0.3, 1.5, 2.7, 3.9, 5.1])
    tan = np.array([0.05, 0.08, 0.11, 0.03, 0.14])
    t = np.stack([tan * np.cos(phi), tan * np.sin(phi)], 1)
    hits = []
    for z in (za, zb):
        for k in range(5):
            hits.append([t[k, 0] * (z - vz[k]), t[k, 1] * (z - vz[k]), z, 0.0])
    hits += [[30.0, -20.0, za, 0.0], [-45.0, 10.0, zb, 0.0], [5.0, 55.0, zb, 0.0]]
    return np.asarray(hits, np.float32), t, vz, (za, zb)


def _axis_distance_by_sampling(hi, hj):
    """Closest transverse distance of the line through two hits to the z axis
    and its z, by sampling the line densely (independent of a closed form)."""
    s = np.linspace(-20.0, 20.0, 400001)
    p = hi[None, :3] + s[:, None] * (hj[:3] - hi[:3])[None, :]
    d = np.hypot(p[:, 0], p[:, 1])
    k = int(np.argmin(d))
    return d[k], p[k, 2]


def test_pair_seeds_keep_exactly_the_lines_through_the_axis():
    hits, t, vz, (za, zb) = _axis_event()
    zref = 225.0
    seeds, cnt = oracle.pair_seeds4(hits, [(za, zb)], 0.5, 0.3, (-250.0, 250.0), zref)
    # brute force over all pairs in order: kept iff the sampled line passes within
    # d_max of the axis at -250 <= z <= 250 (no pair lies near either cut)
    expect = []
    for i in np.flatnonzero(hits[:, 2] == za):
        for j in np.flatnonzero(hits[:, 2] == zb):
            d, zc = _axis_distance_by_sampling(hits[i].astype(np.float64), hits[j].astype(np.float64))
            assert abs(d - 0.3) > 0.05 and abs(abs(zc) - 250.0) > 5.0
            if d <= 0.3 and -250.0 <= zc <= 250.0:
                expect.append((i, j))
    assert cnt == len(expect) == 5
    # each kept line is a track: (x0, y0) = t (zref - vz) at zref, slopes t
    truth = np.concatenate([t * (zref - vz)[:, None], t], 1)
    for (i, j), s in zip(expect, seeds):
        k = i  # the k-th track's hit on the first layer is hit k
        np.testing.assert_allclose(s, truth[k], rtol=1e-5, atol=1e-4)


def test_pair_seeds_cuts_and_order():
    hits, t, vz, (za, zb) = _axis_event()
    # no z window: nothing; a layer pair listed twice: the same seeds twice, in order
    s0, c0 = oracle.pair_seeds4(hits, [(za, zb)], 0.5, 0.3, (-1.0, 1.0), 225.0)
    assert c0 == 1  # only the track from vz = 0 comes closest inside |z| <= 1
    s1, c1 = oracle.pair_seeds4(hits, [(za, zb), (za, zb)], 0.5, 0.3, (-250.0, 250.0), 225.0)
    s2, c2 = oracle.pair_seeds4(hits, [(za, zb)], 0.5, 0.3, (-250.0, 250.0), 225.0)
    assert c1 == 2 * c2 and np.array_equal(s1[:c2], s2) and np.array_equal(s1[c2:], s2)
    # a wider distance cut keeps a superset; the layer tolerance selects the layers
    _, c3 = oracle.pair_seeds4(hits, [(za, zb)], 0.5, 50.0, (-1e4, 1e4), 225.0)
    assert c3 > c2
    _, c4 = oracle.pair_seeds4(hits, [(za + 10.0, zb)], 0.5, 0.3, (-250.0, 250.0), 225.0)
    assert c4 == 0
    # capacity: the count is not clamped
    s5, c5 = oracle.pair_seeds4(hits, [(za, zb)], 0.5, 0.3, (-250.0, 250.0), 225.0, cap=2)
    assert c5 == 5 and len(s5) == 2 and np.array_equal(s5, s2[:2])


UNITS4 = (0.25, 0.25, 2.0 ** -10, 2.0 ** -10)


def test_extract4_reduces_to_the_slope_extraction_when_offsets_agree():
    # equal offsets: a conflict is decided by the slopes alone, as in the
    # (pinned) two-parameter extraction on a grid of the same steps
    rng = np.random.default_rng(3)
    n = 600
    sl = rng.uniform(-0.05, 0.05, (n, 2))
    sl = np.round(sl / 2 ** -12) * 2 ** -12
    R = rng.integers(5, 40, n).astype(np.float64)
    st = rng.integers(0, 3, n).astype(np.uint8)
    th4 = np.concatenate([np.full((n, 2), 7.5), sl], 1)
    lo, step, nn = (-0.5, -0.5), (2.0 ** -10, 2.0 ** -10), (1024, 1024)
    k4 = oracle.extract_tracks4(th4, R, st, lo, step, nn, UNITS4, 10.0, 2.0)
    k2 = oracle.extract_tracks(sl, R, st, lo, step, nn, 10.0, 2.0)
    assert len(k4) > 20 and k4.tolist() == k2.tolist()


def test_extract4_invariants_and_offsets_separate_tracks():
    rng = np.random.default_rng(4)
    n = 800
    centres = np.concatenate([rng.uniform(-20, 20, (40, 2)), rng.uniform(-0.1, 0.1, (40, 2))], 1)
    th = centres[rng.integers(0, 40, n)] + rng.normal(0, 1, (n, 4)) * np.array([0.3, 0.3, 1e-3, 1e-3])
    R = rng.uniform(0, 30, n)
    lo, step, nn = (-0.5, -0.5), (2.0 ** -10, 2.0 ** -10), (1024, 1024)
    keep = oracle.extract_tracks4(th, R, None, lo, step, nn, UNITS4, 5.0, 2.0)
    u = np.asarray(UNITS4)
    cand = np.flatnonzero(R >= 5.0)
    kept = th[keep]
    # no two kept points conflict; every rejected candidate conflicts with a kept one of >= R
    d = np.max(np.abs(kept[:, None] - kept[None]) / u, axis=2)
    np.fill_diagonal(d, np.inf)
    assert np.all(d >= 2.0)
    for i in set(cand.tolist()) - set(keep.tolist()):
        dd = np.max(np.abs(kept - th[i]) / u, axis=1)
        assert np.any((dd < 2.0) & (R[keep] >= R[i]))
    # two points with the same slopes but offsets 1 mm apart are two tracks
    two = np.array([[0.0, 0.0, 0.01, 0.02], [1.0, 0.0, 0.01, 0.02]])
    assert len(oracle.extract_tracks4(two, [9.0, 8.0], None, lo, step, nn, UNITS4, 5.0, 2.0)) == 2
    assert len(oracle.extract_tracks4(two * [1, 1, 1, 1] + [[0, 0, 0, 0], [-0.6, 0, 0, 0]], [9.0, 8.0], None, lo,
                                      step, nn, UNITS4, 5.0, 2.0)) == 1
