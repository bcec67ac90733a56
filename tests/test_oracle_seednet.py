"""Pins of the FP64 seed-net oracle (learned seed proposer) against libraries,
closed forms and finite differences."""
import math

import numpy as np
import pytest

from oracle import seednet as sn
from synth import WORKLOADS, make_event, seednet_init_params


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 10, 5000), rng.uniform(-1e-3, 1e-3, 1000),
                        np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0])]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).float().numpy().astype(np.float64)
    np.testing.assert_array_equal(sn.bf16(x), ref)
    # straight from double: against the same rounding applied to values exactly representable in float32
    np.testing.assert_array_equal(sn.bf16_exact(x.astype(np.float64)), ref)
    assert sn.bf16_exact(1 + 2 ** -9) == 1.0 and sn.bf16_exact(1 + 3 * 2 ** -9) == 1 + 2 ** -7


def test_histogram_matches_numpy_histogram2d_away_from_edges():
    wl = WORKLOADS["velo"]
    ev = make_event(wl, 2, 0, vertex_sigma=(0, 0, 0))
    counts, feat = sn.slope_histogram(ev.hits)
    h = ev.hits.astype(np.float64)
    keep = np.abs(h[:, 2]) >= 50
    u, v = h[keep, 0] / h[keep, 2], h[keep, 1] / h[keep, 2]
    edges = np.linspace(-0.5, 0.5, 65)
    # drop hits within 1e-6 of a bin edge (where float32 and float64 binning may differ)
    near = lambda t: np.min(np.abs(t[:, None] - edges[None, :]), axis=1) < 1e-6
    ok = ~(near(u) | near(v))
    ref, _, _ = np.histogram2d(v[ok], u[ok], bins=[edges, edges])
    # the oracle's counts restricted to the same hits
    sub = ev.hits[np.flatnonzero(keep)[ok]]
    counts_ok, _ = sn.slope_histogram(sub)
    np.testing.assert_array_equal(counts_ok, ref.astype(np.int64))
    assert counts.sum() >= counts_ok.sum() and counts.sum() > 1000
    np.testing.assert_array_equal(feat, sn.bf16(np.log1p(counts.astype(np.float32))))


def test_histogram_zmin_and_range():
    hits = np.array([[0.1 * 60, 0.0, 60.0, 0], [0.1 * 40, 0.0, 40.0, 0],   # |z| < 50 dropped
                     [0.6 * 100, 0.0, 100.0, 0], [-0.5 * 100, -0.5 * 100, 100.0, 0],
                     [0.4999 * 200, 0.0, -200.0, 0]], np.float32)
    counts, _ = sn.slope_histogram(hits)
    assert counts.sum() == 3
    assert counts[32, 38] == 1            # u = 0.1 -> bin floor(0.6 * 64) = 38, v = 0 -> 32
    assert counts[0, 0] == 1              # (-0.5, -0.5) is the lower edge, inside
    assert counts[32, 0] == 1             # x / z = -0.4999 with z < 0


def test_forward_matches_scipy_correlate():
    ss = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    feat = sn.bf16(rng.uniform(0, 3, (64, 64)))
    p = seednet_init_params(3)
    f = sn.forward(feat, p, rounding=False)
    P = sn.unpack(p)
    a1 = np.stack([ss.correlate2d(feat, P["W1"][o, 0], mode="same") + P["b1"][o] for o in range(16)])
    np.testing.assert_allclose(f["a1"], a1, rtol=1e-12, atol=1e-12)
    h1 = np.maximum(a1, 0)
    a2 = np.stack([sum(ss.correlate2d(h1[i], P["W2"][o, i], mode="same") for i in range(16)) + P["b2"][o]
                   for o in range(32)])
    np.testing.assert_allclose(f["a2"], a2, rtol=1e-12, atol=1e-10)
    z = np.tensordot(P["W3"], np.maximum(a2, 0), axes=1) + P["b3"]
    np.testing.assert_allclose(f["z"], z, rtol=1e-12, atol=1e-10)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(2)
    feats = [sn.bf16(rng.uniform(0, 2, (64, 64))) for _ in range(2)]
    labels = [(rng.uniform(0, 1, (64, 64)) < 0.02).astype(np.float64) for _ in range(2)]
    p = seednet_init_params(4).astype(np.float64)
    pw = sn.pos_weight(np.stack(labels))

    def loss(q):
        fw = [sn.forward(x, q, rounding=False) for x in feats]
        return np.mean([sn.bce_loss(f["z"], y, pw) for f, y in zip(fw, labels)])

    fw = [sn.forward(x, p, rounding=False) for x in feats]
    g = sn.backward(fw, labels, p, pw, rounding=False)
    idx = np.concatenate([rng.integers(0, 144, 6), 144 + np.arange(3), rng.integers(160, 4768, 10),
                          4768 + np.arange(3), 4800 + np.arange(4), [4832]])
    h = 1e-5
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (loss(p + e) - loss(p - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_bce_and_pos_weight_closed_forms():
    y = np.zeros((4, 4))
    y[0, 0] = 1
    assert sn.pos_weight(y) == 15.0
    assert sn.pos_weight(np.zeros((20, 20))) == 100.0      # no positives: clamped
    z = np.zeros((4, 4))
    # at z = 0 every term is log 2; mean = (pw * 1 + 15) log 2 / 16
    assert sn.bce_loss(z, y, 15.0) == pytest.approx((15.0 + 15.0) * math.log(2) / 16, rel=1e-14)


def test_adam_first_steps_closed_form():
    g = np.array([0.5, -2.0, 1e-3])
    p0 = np.array([1.0, 1.0, 1.0])
    p1, m, v = sn.adam(p0, g, np.zeros(3), np.zeros(3), 1, lr=0.1)
    # step 1: m_hat = g, v_hat = g^2 -> p1 = p0 - lr g / (|g| + eps)
    np.testing.assert_allclose(p1, p0 - 0.1 * g / (np.abs(g) + 1e-8), rtol=1e-15)
    # step 2 with the same gradient: m_hat = g, v_hat = g^2 again
    p2, m, v = sn.adam(p1, g, m, v, 2, lr=0.1)
    np.testing.assert_allclose(p2, p1 - 0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_top_k_ties_and_cell_centres():
    z = np.zeros(64 * 64)
    z[[5, 70, 4095]] = 3.0
    z[[100, 7]] = 2.0  # tie: 7 before 100
    order, seeds = sn.top_k(z, 5)
    assert order.tolist() == [5, 70, 4095, 7, 100]
    np.testing.assert_allclose(seeds[0], [-0.5 + 5.5 / 64, -0.5 + 0.5 / 64])
    np.testing.assert_allclose(seeds[2], [0.5 - 0.5 / 64, 0.5 - 0.5 / 64])


def _hits_at(points, rng):
    """Hits whose float32 slopes are exactly the given (u, v) (z a power of two)."""
    rows = []
    for a, b in points:
        z = float(rng.choice([-256.0, 64.0, 128.0, 512.0]))
        rows.append((a * z, b * z, z, 0.0))
    return np.array(rows, dtype=np.float32)


def test_propose_seeds_splits_cells_into_dense_sub_cells():
    # constructed event: cell A holds two tracks in different sub-cells (5 and 4 hits) plus one
    # noise hit in a third sub-cell; cell B holds 2 hits in one sub-cell and 1 in another (none
    # reaches n_min = 3: one seed at the fuller sub-cell); cell C is empty; the rest of the
    # cells rank below.  Expected seeds follow from the construction alone.
    rng = np.random.default_rng(9)
    w, ws = 1.0 / 64, 1.0 / 256
    A, B, C = (10, 20), (30, 31), (5, 5)                     # (row, col)

    def pt(cell, sr, sc, fr, fc):                           # point at fraction (fr, fc) of sub-cell (sr, sc)
        r, c = cell
        return (-0.5 + (4 * c + sc + fc) * ws, -0.5 + (4 * r + sr + fr) * ws)

    t1 = [pt(A, 0, 1, 0.30 + 0.01 * k, 0.40) for k in range(5)]
    t2 = [pt(A, 3, 2, 0.60, 0.70 - 0.02 * k) for k in range(4)]
    nz = [pt(A, 2, 0, 0.5, 0.5)]
    b1 = [pt(B, 1, 1, 0.2, 0.2), pt(B, 1, 1, 0.4, 0.6)]
    b2 = [pt(B, 2, 3, 0.5, 0.5)]
    pts = t1 + t2 + nz + b1 + b2
    H = _hits_at(pts, rng)
    H = np.concatenate([H, np.array([[1.0, 1.0, 10.0, 0.0]], np.float32)])   # |z| < zmin: ignored
    exact = np.stack([H[:-1, 0] / H[:-1, 2], H[:-1, 1] / H[:-1, 2]], 1).astype(np.float64)
    logits = np.full(4096, -9.0)
    logits[A[0] * 64 + A[1]] = 3.0
    logits[B[0] * 64 + B[1]] = 2.0
    logits[C[0] * 64 + C[1]] = 1.0
    seeds, cells = sn.propose_seeds(logits, H[rng.permutation(len(H))], K=6, n_min=3)
    assert list(cells) == [A[0] * 64 + A[1]] * 2 + [B[0] * 64 + B[1]] + [C[0] * 64 + C[1]] + [0, 1]
    np.testing.assert_allclose(seeds[0], exact[0:5].mean(0), rtol=0, atol=1e-15)   # 5 hits first
    np.testing.assert_allclose(seeds[1], exact[5:9].mean(0), rtol=0, atol=1e-15)
    np.testing.assert_allclose(seeds[2], exact[10:12].mean(0), rtol=0, atol=1e-15)
    assert tuple(seeds[3]) == (-0.5 + 5.5 * w, -0.5 + 5.5 * w)                      # empty: centre
    assert tuple(seeds[4]) == (-0.5 + 0.5 * w, -0.5 + 0.5 * w)                      # next cells by index
    # K cuts inside a cell; n_min = 1 gives every non-empty sub-cell, fullest first
    s2, c2 = sn.propose_seeds(logits, H, K=1)
    assert len(s2) == 1 and c2[0] == A[0] * 64 + A[1]
    s3, _ = sn.propose_seeds(logits, H, K=5, n_min=1)
    np.testing.assert_allclose(s3[2], exact[9], atol=1e-15)                          # the lone noise hit
    np.testing.assert_allclose(s3[3], exact[10:12].mean(0), atol=1e-15)
    np.testing.assert_allclose(s3[4], exact[12], atol=1e-15)
    # sub-cells refine the histogram's cells exactly, including hits on cell edges
    edge = _hits_at([(-0.5 + 7 * w, -0.5 + 9 * w), (-0.5 + 7 * w - ws / 2, 0.0)], rng)
    counts, _ = sn.slope_histogram(edge)
    lg = np.zeros(4096)
    _, ce = sn.propose_seeds(lg - np.arange(4096) * 1e-3 + 10 * counts.reshape(-1), edge, K=2, n_min=1)
    assert sorted(ce) == sorted(np.flatnonzero(counts.reshape(-1)))
