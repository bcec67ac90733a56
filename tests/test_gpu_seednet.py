"""Learned seed proposer on the GPU against the FP64 oracle (oracle/seednet.py).

Histogram: counts exact, features bitwise.  Network: the
kernels round the same quantities to bfloat16 as the oracle, but from float32
sums where the oracle rounds double sums, so a stored activation can differ
by one bfloat16 step where a sum sits within float32 error of a rounding
boundary.  The logit bound below propagates that worst case layer by layer
(every activation one step off, plus float32 summation error), and the
fraction of activations not bitwise equal to the oracle's must stay small.
Gradients: relative L2 error per parameter block and an elementwise bound in
units of the block's sum of |terms|.  Top-K: bit-exact indices on float32
logits with ties, NaN and signed zeros; seeds within float32 rounding.
"""
import math
import os
import tempfile

import numpy as np
import pytest
import torch

from oracle import seednet as sn
from synth import WORKLOADS, batch_of, make_event, seednet_init_params

pytestmark = pytest.mark.gpu

U7 = 2.0 ** -7      # one bfloat16 step, relative to the value's magnitude (8 significant bits)


@pytest.fixture(scope="module")
def rt():
    from paper_1709_08610_gb300 import build as rbuild
    rbuild.build()
    from paper_1709_08610_gb300 import retina
    return retina


@pytest.fixture(params=[0, 1], ids=["cuda_cores", "tensor_cores"])
def conv2_path(rt, request):
    """The second convolution on the FP32 CUDA cores or the tcgen05 tensor cores."""
    old = rt.get_option(rt.OPT_SEEDNET_TC)
    rt.set_option(rt.OPT_SEEDNET_TC, request.param)
    rt.device_error(reset=True)
    yield request.param
    torch.cuda.synchronize()
    rt.set_option(rt.OPT_SEEDNET_TC, old)
    assert rt.device_error() == 0


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _f(t):
    return t.float().cpu().numpy().astype(np.float64)


def _events(n=3, v0=True):
    wl = WORKLOADS["velo"]
    vs = (0, 0, 0) if v0 else (0.05, 0.05, 50.0)
    return [make_event(wl, 11, e, vertex_sigma=vs) for e in range(n)]


def _special_hits():
    """Bin edges, the range ends, |z| at and below zmin, negative z, z = 0 and NaN."""
    w = 1.0 / 64
    rows = []
    for k in (0, 1, 31, 32, 63):
        u = -0.5 + k * w                       # exactly on the lower edge of bin k
        rows += [(u * 128.0, 0.1 * 128.0, 128.0), (u * -256.0, -0.2 * -256.0, -256.0)]
    rows += [(0.5 * 64.0, 0.0, 64.0),          # u = 0.5: outside [lo, hi)
             (-0.5 * 64.0, -0.5 * 64.0, 64.0),  # u = v = -0.5: bin (0, 0)
             (1.0, 1.0, 50.0), (1.0, 1.0, -50.0), (1.0, 1.0, 49.99),
             (1.0, 1.0, 0.0), (float("nan"), 1.0, 100.0), (1.0, 1.0, float("nan"))]
    return np.array([(a, b, c, 0.0) for a, b, c in rows], dtype=np.float32)


# ---------------------------------------------------------------------------
# S7: histogram
# ---------------------------------------------------------------------------

def test_slope_histogram_is_exact(rt):
    evs = _events(3, v0=False) + _events(1)
    hits = [e.hits for e in evs] + [np.zeros((0, 4), np.float32), _special_hits()]
    offs = np.zeros(len(hits) + 1, np.int64)
    offs[1:] = np.cumsum([len(h) for h in hits])
    H = np.concatenate(hits)
    feat, cnt = rt.slope_histogram(_dev(H), _dev(offs), counts=True)
    feat, cnt = _f(feat), cnt.cpu().numpy()
    for e, h in enumerate(hits):
        c_o, f_o = sn.slope_histogram(h)
        np.testing.assert_array_equal(cnt[e], c_o)
        np.testing.assert_array_equal(feat[e], f_o)
    # the special event: bin edges land in the upper bin, u = 0.5 and |z| < 50 are dropped
    c_s = cnt[len(hits) - 1]
    assert c_s.sum() == 13 and c_s[0, 0] == 1
    # order independence
    perm = np.concatenate([offs[i] + np.random.default_rng(i).permutation(len(h)) for i, h in enumerate(hits)])
    feat2, cnt2 = rt.slope_histogram(_dev(H[perm]), _dev(offs), counts=True)
    assert np.array_equal(cnt2.cpu().numpy(), cnt) and np.array_equal(_f(feat2), feat)


def test_histogram_feature_of_every_small_count_is_the_oracles(rt):
    # one event per count c = 0..511, all c hits in one cell: bf16(log1pf(c)) vs numpy's float32 log1p
    n = 512
    hits = np.concatenate([np.tile(np.array([[1.0, 1.0, 100.0, 0.0]], np.float32), (c, 1)) for c in range(n)])
    offs = np.concatenate([[0], np.cumsum(np.arange(n))]).astype(np.int64)
    feat = _f(rt.slope_histogram(_dev(hits), _dev(offs)))
    r, c = 32, 32  # slope 0.01 -> bin 32 of 64 over [-0.5, 0.5)
    np.testing.assert_array_equal(feat[:, r, c], sn.bf16(np.log1p(np.arange(n, dtype=np.float32))))


# ---------------------------------------------------------------------------
# S8: forward
# ---------------------------------------------------------------------------

def _abs_conv(x, W):
    return sn._conv_same(np.abs(x), np.abs(W))


def _bounds(fw, params):
    """Worst-case |gpu - oracle| of h1, h2 and the logits when every stored
    activation may be one bfloat16 step off and a float32 sum of n terms
    carries n 2^-24 times the sum of their magnitudes."""
    P = sn.unpack(params)
    W1, W2, W3 = sn.bf16(P["W1"]), sn.bf16(P["W2"]), sn.bf16(P["W3"])
    b1, b2, b3 = sn.bf16(P["b1"]), sn.bf16(P["b2"]), sn.bf16(P["b3"])
    k = 1.0 + 2.0 ** -8   # |relu(a)| <= k |bf16(relu(a))|
    A1 = _abs_conv(fw["x"], W1) + np.abs(b1)[:, None, None]
    e1 = 10 * 2.0 ** -24 * A1
    E1 = 1.01 * (e1 + U7 * (k * np.abs(fw["h1"]) + e1))
    A2 = _abs_conv(np.abs(fw["h1"]) + E1, W2) + np.abs(b2)[:, None, None]
    e2 = _abs_conv(E1, W2) + 145 * 2.0 ** -24 * A2
    E2 = 1.01 * (e2 + U7 * (k * np.abs(fw["h2"]) + e2))
    Az = np.einsum("o,orc->rc", np.abs(W3), np.abs(fw["h2"]) + E2) + abs(b3)
    Ez = 1.01 * (np.einsum("o,orc->rc", np.abs(W3), E2) + 33 * 2.0 ** -24 * Az)
    return E1, E2, Ez


def _logit_bound(fw, params):
    return _bounds(fw, params)[2]


@pytest.mark.parametrize("pseed,scale", [(7, 1.0), (8, 3.0)])
def test_forward_matches_oracle(rt, conv2_path, pseed, scale):
    evs = _events(3)
    b = batch_of(evs)
    feat = rt.slope_histogram(_dev(b.hits), _dev(b.offsets))
    params = seednet_init_params(pseed)
    params[:4832] *= np.float32(scale)
    logits, h1, h2 = rt.seednet_forward(feat, _dev(params), want_h2=True)
    logits, h1, h2 = _f(logits), _f(h1), _f(h2)
    n_h1 = n_h2 = 0
    for e, ev in enumerate(evs):
        _, f_o = sn.slope_histogram(ev.hits)
        fw = sn.forward(f_o, params)
        E1, E2, Ez = _bounds(fw, params)
        assert np.all(np.abs(h1[e] - fw["h1"]) <= E1)
        assert np.all(np.abs(h2[e] - fw["h2"]) <= E2)
        assert np.all(np.abs(logits[e] - fw["z"]) <= Ez), np.max(np.abs(logits[e] - fw["z"]) - Ez)
        n_h1 += np.count_nonzero(h1[e] != fw["h1"])
        n_h2 += np.count_nonzero(h2[e] != fw["h2"])
    # activations differ only where a sum sits at a rounding boundary
    assert n_h1 <= 1e-3 * h1.size and n_h2 <= 1e-2 * h2.size, (n_h1 / h1.size, n_h2 / h2.size)


# ---------------------------------------------------------------------------
# S10: training step
# ---------------------------------------------------------------------------

def _labels(evs):
    """1 at the cells of the events' true slopes (a seeded, structured label map)."""
    y = np.zeros((len(evs), 64, 64), np.uint8)
    for e, ev in enumerate(evs):
        t = ev.truth[:, :2]
        c = np.floor((t + 0.5) * 64).astype(int)
        ok = (c >= 0).all(1) & (c < 64).all(1)
        y[e, c[ok, 1], c[ok, 0]] = 1
    return y


def _grad_abs_scale(fws, labels, params, pw):
    """Per parameter, the sum of |terms| its gradient sums (built from the oracle's forward)."""
    P = sn.unpack(params)
    W2, W3 = np.abs(sn.bf16(P["W2"])), np.abs(sn.bf16(P["W3"]))
    N = sum(f["z"].size for f in fws)
    g = {k: np.zeros_like(np.asarray(v, dtype=np.float64)) for k, v in P.items()}
    g["b3"] = 0.0
    for f, y in zip(fws, labels):
        y = y.astype(np.float64)
        sg = 1 / (1 + np.exp(-f["z"]))
        dz = np.abs(pw * y * (sg - 1) + (1 - y) * sg) / N
        g["W3"] += np.einsum("rc,orc->o", dz, f["h2"])
        g["b3"] += dz.sum()
        d2 = dz[None] * W3[:, None, None] * (f["h2"] > 0)
        hp = np.pad(f["h1"], ((0, 0), (1, 1), (1, 1)))
        for dy in range(3):
            for dx in range(3):
                g["W2"][:, :, dy, dx] += np.einsum("orc,irc->oi", d2, hp[:, dy:dy + 64, dx:dx + 64])
        g["b2"] += d2.sum((1, 2))
        dp = np.pad(d2, ((0, 0), (1, 1), (1, 1)))
        d1 = np.zeros((16, 64, 64))
        for dy in range(3):
            for dx in range(3):
                d1 += np.einsum("oi,orc->irc", W2[:, :, dy, dx], dp[:, 2 - dy:66 - dy, 2 - dx:66 - dx])
        d1 *= f["h1"] > 0
        xp = np.pad(f["x"][0], 1)
        for dy in range(3):
            for dx in range(3):
                g["W1"][:, 0, dy, dx] += np.einsum("orc,rc->o", d1, xp[dy:dy + 64, dx:dx + 64])
        g["b1"] += d1.sum((1, 2))
    return sn.pack(g)


BLOCKS = dict(W1=(0, 144), b1=(144, 160), W2=(160, 4768), b2=(4768, 4800), W3=(4800, 4832), b3=(4832, 4833))


def test_train_step_gradient_and_loss_match_oracle(rt, conv2_path):
    evs = _events(4)
    b = batch_of(evs)
    feat = rt.slope_histogram(_dev(b.hits), _dev(b.offsets))
    y = _labels(evs)
    params = seednet_init_params(9)
    p_d, m_d, v_d = _dev(params.copy()), torch.zeros(4833, device="cuda"), torch.zeros(4833, device="cuda")
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(4833, device="cuda")
    lr = 1e-3
    rt.seednet_train_step(feat, _dev(y), p_d, m_d, v_d, 1, lr=lr, loss=loss, grad=grad)
    fws = [sn.forward(sn.slope_histogram(ev.hits)[1], params) for ev in evs]
    pw = sn.pos_weight(y)
    L_o = sn.bce_loss(np.stack([f["z"] for f in fws]), y, pw)
    g_o = sn.backward(fws, list(y), params, pw)
    g = _f(grad)
    assert abs(loss.item() - L_o) <= 1e-5 * L_o
    A = _grad_abs_scale(fws, list(y), params, pw)
    for name, (i, j) in BLOCKS.items():
        d = g[i:j] - g_o[i:j]
        assert np.linalg.norm(d) <= 1e-3 * np.linalg.norm(g_o[i:j]) + 1e-12, (name, np.linalg.norm(d) / np.linalg.norm(g_o[i:j]))
        assert np.all(np.abs(d) <= 2e-3 * A[i:j] + 1e-12), (name, np.max(np.abs(d) / (A[i:j] + 1e-30)))
    # the Adam update on the GPU gradient: step 1 moves each weight by lr g / (|g| + eps)
    p_new = _f(p_d)
    ref = params.astype(np.float64) - lr * g / (np.abs(g) + 1e-8)
    assert np.all(np.abs(p_new - ref) <= 2.0 ** -22 * np.abs(ref) + 1e-6 * lr)
    # and it moves in the oracle gradient's direction wherever the two gradients are resolved
    big = np.abs(g_o) > 1e-2 * np.max(np.abs(g_o))
    assert np.all(np.sign(p_new - params)[big] == -np.sign(g_o[big]))


def test_adam_matches_oracle(rt):
    """Float32 Adam vs double: m = b1 m + (1 - b1) g can cancel, so its error is
    bounded by float32 rounding of the magnitudes it sums (M below), not of m;
    the parameter error follows through m_hat / (sqrt(v_hat) + eps)."""
    rng = np.random.default_rng(3)
    p = rng.normal(0, 1, 4833)
    m = np.zeros(4833)
    v = np.zeros(4833)
    M = np.zeros(4833)
    tol_p = np.zeros(4833)
    p_d, m_d, v_d = _dev(p.astype(np.float32)), torch.zeros(4833, device="cuda"), torch.zeros(4833, device="cuda")
    p = p.astype(np.float32).astype(np.float64)
    # the kernel receives the hyper-parameters as float32: the oracle gets the same numbers
    lr, b1, b2, eps = (float(np.float32(x)) for x in (1e-2, 0.9, 0.999, 1e-8))
    u = 2.0 ** -24
    for step in range(1, 6):
        g = (rng.normal(0, 1, 4833) * 10.0 ** rng.uniform(-7, 1, 4833)).astype(np.float32)
        rt.seednet_adam(p_d, m_d, v_d, _dev(g), step, lr=lr, betas=(b1, b2), eps=eps)
        p, m, v = sn.adam(p, g.astype(np.float64), m, v, step, lr=lr, b1=b1, b2=b2, eps=eps)
        M = b1 * M + (1 - b1) * np.abs(g)
        tol_m = 4 * step * u * M
        assert np.all(np.abs(_f(m_d) - m) <= tol_m)
        np.testing.assert_allclose(_f(v_d), v, rtol=8 * step * u, atol=0)
        den = np.sqrt(v / (1 - b2 ** step)) + eps
        c1 = 1 / (1 - b1 ** step)
        tol_p += 2 * u * np.abs(p) + lr * (c1 * tol_m + 8 * u * c1 * np.abs(m)) / den
        assert np.all(np.abs(_f(p_d) - p) <= tol_p + 1e-7 * lr)


def test_train_steps_are_deterministic_and_resume_bitwise(rt, tmp_path):
    from paper_1709_08610_gb300 import seednet as snet
    evs = _events(4)
    b = batch_of(evs)
    feat = rt.slope_histogram(_dev(b.hits), _dev(b.offsets))
    y = _dev(_labels(evs))

    def run(n, state=None):
        st = state or snet.TrainState.fresh(seednet_init_params(2), "cuda")
        for _ in range(n):
            st.step(feat, y)
        return st

    a = run(6)
    b1 = run(3)
    path = os.path.join(tmp_path, "ck.seednet")
    b1.save(path, meta={"note": "test"})
    b2 = snet.TrainState.load(path, "cuda")
    assert b2.n_steps == 3
    b2 = run(3, b2)
    for x, z in ((a.params, b2.params), (a.m, b2.m), (a.v, b2.v)):
        assert torch.equal(x, z)
    assert a.last_loss == b2.last_loss
    # a few steps on a fixed batch lower the loss
    c = run(40)
    assert c.last_loss < a.losses[0]


# ---------------------------------------------------------------------------
# S9: top-K
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("K", [1, 512, 4096])
def test_topk_is_exact_with_ties_nan_and_signed_zeros(rt, K):
    rng = np.random.default_rng(K)
    z = (np.round(rng.normal(0, 2, (3, 4096)) * 4) / 4).astype(np.float32)  # many equal values
    z[0, rng.integers(0, 4096, 40)] = np.nan
    z[1, :100] = -0.0
    z[1, 100:200] = 0.0
    z[2, 7] = np.inf
    z[2, 9] = -np.inf
    seeds, idx = rt.topk_seeds(_dev(z), K, want_idx=True)
    seeds, idx = seeds.cpu().numpy(), idx.cpu().numpy()
    for e in range(3):
        order, s_o = sn.top_k(z[e], K)
        np.testing.assert_array_equal(idx[e], order)
        np.testing.assert_array_equal(seeds[e], s_o.astype(np.float32))


def _check_proposal(seeds, cells, s_o, c_o):
    """Cells bit-exact; seeds within float32 rounding of the sub-cell mean
    (in-sub-cell positions from float32 t = (u - lo) 256, error <= 2^-17 of a
    sub-cell each, plus the final float32 rounding)."""
    np.testing.assert_array_equal(cells, c_o)
    assert np.all(np.abs(seeds - s_o) <= 2.0 ** -16 / 256 + 2.0 ** -24 * np.abs(s_o) + 1e-12)


@pytest.mark.parametrize("K,n_min", [(512, 3), (64, 1), (4096, 3)])
def test_proposed_seeds_match_oracle(rt, K, n_min):
    evs = _events(3) + [make_event(WORKLOADS["velo"], 11, 9, n_tracks=0, noise_frac=0.0)]  # one empty event
    hits = [e.hits for e in evs] + [_special_hits()]
    offs = np.concatenate([[0], np.cumsum([len(h) for h in hits])]).astype(np.int64)
    H = np.concatenate(hits)
    # host-made logits from the oracle's counts: busy cells first, then a fixed ramp, with exact ties
    ramp = np.round(1e-3 * np.arange(4096)[::-1].reshape(64, 64), 1)
    logits = np.stack([np.log1p(sn.slope_histogram(h)[0]) + ramp for h in hits]).astype(np.float32)
    seeds, cells = rt.topk_seeds(_dev(logits), K, hits=_dev(H), offsets=_dev(offs), min_sub_hits=n_min,
                                 want_idx=True)
    seeds, cells = seeds.cpu().numpy().astype(np.float64), cells.cpu().numpy()
    for e, h in enumerate(hits):
        s_o, c_o = sn.propose_seeds(logits[e], h, K, n_min=n_min)
        _check_proposal(seeds[e], cells[e], s_o, c_o)
    # hits in any order give the same seeds bitwise
    perm = np.concatenate([offs[i] + np.random.default_rng(7 + i).permutation(len(h)) for i, h in enumerate(hits)])
    seeds2 = rt.topk_seeds(_dev(logits), K, hits=_dev(H[perm]), offsets=_dev(offs), min_sub_hits=n_min)
    assert np.array_equal(seeds2.cpu().numpy().astype(np.float64), seeds)


# ---------------------------------------------------------------------------
# full size: 1024 ragged events (the batched workload's shapes), sampled
# ---------------------------------------------------------------------------

def test_proposer_at_full_batch_size(rt, conv2_path):
    wl = WORKLOADS["velo_batch"]
    evs = [make_event(wl, 12, e, vertex_sigma=(0, 0, 0)) for e in range(1024)]
    b = batch_of(evs)
    hits, offs = _dev(b.hits), _dev(b.offsets)
    feat, cnt = rt.slope_histogram(hits, offs, counts=True)
    params = seednet_init_params(5)
    logits = rt.seednet_forward(feat, _dev(params))
    cnt, lg = cnt.cpu().numpy(), logits.cpu().numpy()
    sample = list(range(0, 1024, 97))
    z_o = {}
    for e in sample:
        c_o, f_o = sn.slope_histogram(evs[e].hits)
        np.testing.assert_array_equal(cnt[e], c_o)
        fw = sn.forward(f_o, params)
        assert np.all(np.abs(lg[e] - fw["z"]) <= _logit_bound(fw, params))
        z_o[e] = fw["z"].astype(np.float32)
        lg[e] = z_o[e]  # the sampled events' rows: the oracle's logits, read by both sides
    seeds, cells = rt.topk_seeds(_dev(lg), 512, hits=hits, offsets=offs, want_idx=True)
    seeds, cells = seeds.cpu().numpy().astype(np.float64), cells.cpu().numpy()
    for e in sample:
        s_o, c_o = sn.propose_seeds(z_o[e], evs[e].hits, 512)
        _check_proposal(seeds[e], cells[e], s_o, c_o)
