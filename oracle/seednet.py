"""FP64 oracle of the learned seed proposer - TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the bench's CPU-baseline leg use this
module; it shares no code with the CUDA path.  Plain numpy, double precision,
written as the definitions read:

* slope_histogram - counts of hit slopes (x/z, y/z) on a regular 64 x 64 grid
  over [lo, hi)^2, hits with |z| >= zmin only; feature = bf16(log1p(count)).
  The bin of a hit is decided in float32, as the kernel decides it: u = x / z,
  bin = floor((u - lo) * (n / (hi - lo))).
* forward - conv 3x3 (1 -> 16) + ReLU, conv 3x3 (16 -> 32) + ReLU, 1x1
  (32 -> 1): 'same' zero padding, stride 1, cross-correlation; weights and
  activations rounded to bfloat16 (round to nearest even), sums in double.
* bce_loss / backward - binary cross-entropy with logits, positive weight
  pw = min(100, #negative / max(#positive, 1)) over the batch, mean over all
  pixels; gradients by the chain rule, the gradient images rounded to
  bfloat16 where the kernels store them.
* adam - Adam (Kingma & Ba) with bias correction.
* top_k - the K largest logits per event (ties: lower index first), seeds at
  the cell centres.
* propose_seeds - the seeds of the learned proposer: walk the cells by
  decreasing logit; each cell splits into 4 x 4 sub-cells and gives one seed
  per sub-cell holding at least n_min of its hits (most hits first) at the
  mean slope of those hits; a cell with no such sub-cell gives one seed at its
  most populated sub-cell's mean, an empty cell its centre; stop at K seeds.
  Only the first R_MAX ranked cells are split; later ones give their centre.

Parameter vector layout (4833 values): W1 [16,1,3,3] at 0, b1 [16] at 144,
W2 [32,16,3,3] at 160, b2 [32] at 4768, W3 [32] at 4800, b3 at 4832.
"""
from __future__ import annotations

import numpy as np

NB = 64
C1, C2 = 16, 32
N_PARAMS = 4833
OFF = dict(W1=0, b1=144, W2=160, b2=4768, W3=4800, b3=4832)


def unpack(p: np.ndarray) -> dict:
    p = np.asarray(p, dtype=np.float64)
    return dict(W1=p[0:144].reshape(C1, 1, 3, 3), b1=p[144:160], W2=p[160:4768].reshape(C2, C1, 3, 3),
                b2=p[4768:4800], W3=p[4800:4832], b3=p[4832])


def pack(d: dict) -> np.ndarray:
    return np.concatenate([d["W1"].reshape(-1), d["b1"].reshape(-1), d["W2"].reshape(-1), d["b2"].reshape(-1),
                           d["W3"].reshape(-1), np.atleast_1d(d["b3"]).reshape(-1)]).astype(np.float64)


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    Goes through float32 first (exact for float32 inputs; for doubles the
    kernels' own float32 sums are what gets rounded)."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(a), out, a.astype(np.float64))


def bf16_exact(x) -> np.ndarray:
    """Round a float64 straight to the nearest bfloat16 (ties to even)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
    scaled = np.ldexp(m, 8)                  # 8 significant bits
    r = np.round(scaled)                     # numpy rounds half to even
    return np.where(x == 0, 0.0, np.ldexp(r, e - 8))


def _binned_slopes(hits, lo, hi, nb, zmin):
    """(u, v, u_bin, v_bin) of the hits slope_histogram counts (same float32 rule)."""
    h = np.asarray(hits, dtype=np.float32)
    x, y, z = h[:, 0], h[:, 1], h[:, 2]
    keep = np.abs(z) >= np.float32(zmin)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = (x / z).astype(np.float32)
        v = (y / z).astype(np.float32)
        scale = np.float32(nb / (hi - lo))
        bu = np.floor((u - np.float32(lo)) * scale)
        bv = np.floor((v - np.float32(lo)) * scale)
        ok = keep & np.isfinite(bu) & np.isfinite(bv) & (bu >= 0) & (bu < nb) & (bv >= 0) & (bv < nb)
    return u[ok], v[ok], bu[ok].astype(np.int64), bv[ok].astype(np.int64)


def slope_histogram(hits: np.ndarray, lo: float = -0.5, hi: float = 0.5, nb: int = NB, zmin: float = 50.0):
    """(counts int64 [nb, nb] indexed [v_bin, u_bin], feature float64 (bf16 values))."""
    _, _, bu, bv = _binned_slopes(hits, lo, hi, nb, zmin)
    counts = np.zeros((nb, nb), dtype=np.int64)
    np.add.at(counts, (bv, bu), 1)
    return counts, bf16(np.log1p(counts.astype(np.float32)))


def _conv_same(x: np.ndarray, W: np.ndarray) -> np.ndarray:
    """'same' 3x3 cross-correlation: out[o, r, c] = sum_{i,dy,dx} W[o,i,dy,dx] x[i, r+dy-1, c+dx-1]."""
    Ci, H, Wd = x.shape
    xp = np.zeros((Ci, H + 2, Wd + 2))
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((W.shape[0], H, Wd))
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("oi,irc->orc", W[:, :, dy, dx], xp[:, dy:dy + H, dx:dx + Wd])
    return out


def _ident(x):
    return np.asarray(x, dtype=np.float64)


def forward(feat: np.ndarray, params: np.ndarray, rounding: bool = True) -> dict:
    """One event's forward pass; feat [64, 64] (bf16 values).  rounding=False
    drops every bfloat16 rounding (a smooth function, for derivative checks)."""
    P = unpack(params)
    rp, ra = (bf16, bf16_exact) if rounding else (_ident, _ident)
    W1, W2, W3 = rp(P["W1"]), rp(P["W2"]), rp(P["W3"])
    b1, b2, b3 = rp(P["b1"]), rp(P["b2"]), rp(P["b3"])
    x = np.asarray(feat, dtype=np.float64)[None]
    a1 = _conv_same(x, W1) + b1[:, None, None]
    h1 = ra(np.maximum(a1, 0.0))
    a2 = _conv_same(h1, W2) + b2[:, None, None]
    h2 = ra(np.maximum(a2, 0.0))
    z = np.einsum("o,orc->rc", W3, h2) + b3
    return dict(x=x, a1=a1, h1=h1, a2=a2, h2=h2, z=z)


def pos_weight(labels: np.ndarray) -> float:
    y = np.asarray(labels)
    npos = int(np.count_nonzero(y))
    nneg = y.size - npos
    return float(min(100.0, nneg / max(npos, 1)))


def softplus(t):
    return np.logaddexp(0.0, t)


def bce_loss(z: np.ndarray, y: np.ndarray, pw: float) -> float:
    """mean over pixels of pw y softplus(-z) + (1 - y) softplus(z)."""
    z = np.asarray(z, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return float(np.mean(pw * y * softplus(-z) + (1.0 - y) * softplus(z)))


def backward(fw_list, labels, params: np.ndarray, pw: float, rounding: bool = True) -> np.ndarray:
    """Gradient of bce_loss(mean over the batch) w.r.t. the parameter vector.

    The kernels store dL/d(pre-activation) of both convolutions as bfloat16;
    so does this oracle, at the same points (rounding=False: no rounding,
    the exact gradient of the smooth forward(rounding=False))."""
    P = unpack(params)
    rp, ra = (bf16, bf16_exact) if rounding else (_ident, _ident)
    W2, W3 = rp(P["W2"]), rp(P["W3"])
    n_px = sum(f["z"].size for f in fw_list)
    g = {k: np.zeros_like(np.asarray(v, dtype=np.float64)) for k, v in P.items()}
    g["b3"] = 0.0
    for f, y in zip(fw_list, labels):
        y = np.asarray(y, dtype=np.float64)
        sig = 1.0 / (1.0 + np.exp(-f["z"]))
        dz = (pw * y * (sig - 1.0) + (1.0 - y) * sig) / n_px           # dL/dz [64, 64]
        g["W3"] += np.einsum("rc,orc->o", dz, f["h2"])
        g["b3"] += dz.sum()
        d2 = ra(dz[None] * W3[:, None, None] * (f["h2"] > 0))  # dL/da2, stored bf16
        hp = np.zeros((C1, 66, 66))
        hp[:, 1:-1, 1:-1] = f["h1"]
        for dy in range(3):
            for dx in range(3):
                g["W2"][:, :, dy, dx] += np.einsum("orc,irc->oi", d2, hp[:, dy:dy + 64, dx:dx + 64])
        g["b2"] += d2.sum(axis=(1, 2))
        # dL/dh1 = transposed convolution of d2 with W2
        dp = np.zeros((C2, 66, 66))
        dp[:, 1:-1, 1:-1] = d2
        dh1 = np.zeros((C1, 64, 64))
        for dy in range(3):
            for dx in range(3):
                dh1 += np.einsum("oi,orc->irc", W2[:, :, dy, dx], dp[:, 2 - dy:66 - dy, 2 - dx:66 - dx])
        d1 = ra(dh1 * (f["h1"] > 0))                            # dL/da1, stored bf16
        xp = np.zeros((1, 66, 66))
        xp[:, 1:-1, 1:-1] = f["x"]
        for dy in range(3):
            for dx in range(3):
                g["W1"][:, 0, dy, dx] += np.einsum("orc,rc->o", d1, xp[0, dy:dy + 64, dx:dx + 64])
        g["b1"] += d1.sum(axis=(1, 2))
    return pack(g)


def adam(params, grad, m, v, step: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns (params, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def top_k(logits: np.ndarray, K: int, lo: float = -0.5, hi: float = 0.5, nb: int = NB):
    """Indices (v_bin * nb + u_bin) of the K largest logits (ties: lower
    index first) and the seeds (u, v) at their cell centres."""
    z = np.asarray(logits, dtype=np.float64).reshape(-1)
    order = np.lexsort((np.arange(z.size), -z))[:K]
    w = (hi - lo) / nb
    seeds = np.stack([lo + (order % nb + 0.5) * w, lo + (order // nb + 0.5) * w], 1)
    return order, seeds


SUB = 4          # sub-cells per cell and axis
R_MAX = 1024     # ranked cells that are split into sub-cells


def propose_seeds(logits: np.ndarray, hits: np.ndarray, K: int, lo: float = -0.5, hi: float = 0.5,
                  nb: int = NB, zmin: float = 50.0, n_min: int = 3):
    """(seeds float64 [K, 2], cell index [K]) of the learned proposer.

    Sub-cell of a hit: floor of t = (u - lo) * (4 s) in float32, s =
    float32(nb / (hi - lo)) - four times the histogram's own t, so the cell
    is exactly the histogram's bin and the sub-cell refines it."""
    z = np.asarray(logits, dtype=np.float64).reshape(-1)
    order = np.lexsort((np.arange(z.size), -z))
    h = np.asarray(hits, dtype=np.float32)
    keep = np.abs(h[:, 2]) >= np.float32(zmin)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = (h[:, 0] / h[:, 2]).astype(np.float32)
        v = (h[:, 1] / h[:, 2]).astype(np.float32)
        s4 = np.float32(nb / (hi - lo)) * np.float32(SUB)
        fu = np.floor((u - np.float32(lo)) * s4)
        fv = np.floor((v - np.float32(lo)) * s4)
        nf = nb * SUB
        ok = keep & np.isfinite(fu) & np.isfinite(fv) & (fu >= 0) & (fu < nf) & (fv >= 0) & (fv < nf)
    u, v = u[ok].astype(np.float64), v[ok].astype(np.float64)
    fu, fv = fu[ok].astype(np.int64), fv[ok].astype(np.int64)
    cell = (fv // SUB) * nb + fu // SUB
    sub = (fv % SUB) * SUB + fu % SUB
    w = (hi - lo) / nb
    seeds, cells = [], []
    for r, c in enumerate(order):
        if len(seeds) == K:
            break
        centre = (lo + (c % nb + 0.5) * w, lo + (c // nb + 0.5) * w)
        if r >= R_MAX:
            seeds.append(centre)
            cells.append(c)
            continue
        mine = cell == c
        cnt = np.bincount(sub[mine], minlength=SUB * SUB)
        ranked = sorted(range(SUB * SUB), key=lambda q: (-cnt[q], q))
        chosen = [q for q in ranked if cnt[q] >= n_min]
        if not chosen and cnt.max() >= 1:
            chosen = ranked[:1]
        if not chosen:
            seeds.append(centre)
            cells.append(c)
            continue
        for q in chosen:
            if len(seeds) == K:
                break
            sel = mine & (sub == q)
            seeds.append((u[sel].mean(), v[sel].mean()))
            cells.append(c)
    return np.array(seeds, dtype=np.float64).reshape(-1, 2), np.array(cells, dtype=np.int64)
