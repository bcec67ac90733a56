"""Train the learned seed proposer on generated VELO-like events, on the GPU.

    python -m paper_1709_08610_gb300.train_seednet --events 100000 --epochs 3 \\
        --out paper_1709_08610_gb300/weights/seednet_velo.ckpt

Data: VELO-like single events (150 tracks, 26 layers, 90 % layer efficiency,
10 % noise, 0.01 mm hit smear) with every track from the origin - the
slope model's own hypothesis class; with a vertex smeared by N(0, 50 mm) in z
a track's hits leave the origin line by millimetres, far beyond sigma, and the
method finds almost none of them.  Run seed 1000, event ids 0 .. N-1, drawn
by a pool of host processes.

Labels: 1 at each 64 x 64 slope cell holding a maximum the plain grid method
finds - Eq. 2 on the 1024 x 1024 grid at the grid sigma, strict local maxima
above R0 (retina_grid_scan, the parity-tested GPU path) - else 0.

Training: the library's kernels only (histogram, forward, backward, Adam);
contiguous batches of i.i.d. events, Adam lr 1e-3, betas (0.9, 0.999),
eps 1e-8, deterministic.  The checkpoint's JSON header records the recipe, the
loss curve and a held-out evaluation (see ``evaluate``).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import time
from typing import Dict, List

import numpy as np

RUN_SEED_TRAIN = 1000
RUN_SEED_EVAL = 2000
V0 = (0.0, 0.0, 0.0)


def _gen(job):
    """Host worker: one chunk of events -> (hits, offsets, truth slopes)."""
    from synth import WORKLOADS, make_event
    name, run_seed, lo, hi = job
    wl = WORKLOADS[name]
    evs = [make_event(wl, run_seed, e, vertex_sigma=V0) for e in range(lo, hi)]
    offs = np.zeros(len(evs) + 1, np.int64)
    offs[1:] = np.cumsum([e.n_hits for e in evs])
    return (np.concatenate([e.hits for e in evs]), offs, [e.truth[:, :2].copy() for e in evs])


def generate(name: str, run_seed: int, n: int, chunk: int, workers: int):
    """Yield chunks of generated events, drawn in a spawn pool (no fork after CUDA)."""
    jobs = [(name, run_seed, a, min(a + chunk, n)) for a in range(0, n, chunk)]
    if workers <= 1:
        for j in jobs:
            yield _gen(j)
        return
    with mp.get_context("spawn").Pool(workers) as pool:
        for out in pool.imap(_gen, jobs):
            yield out


def cells_of(theta: np.ndarray, lo: float = -0.5, hi: float = 0.5, nb: int = 64) -> np.ndarray:
    """Linear cell index (row * nb + col) of slope points, -1 outside the box."""
    c = np.floor((np.asarray(theta, dtype=np.float64) - lo) * (nb / (hi - lo))).astype(np.int64)
    ok = np.all((c >= 0) & (c < nb), axis=-1)
    return np.where(ok, c[..., 1] * nb + c[..., 0], -1)


def build_dataset(n: int, chunk: int, workers: int, device="cuda"):
    """features bf16 [n, 64, 64] and labels uint8 [n, 64, 64] on the device."""
    import torch
    from synth import WORKLOADS
    from . import retina as rt
    wl = WORKLOADS["velo"]
    grid = rt.Grid.of(wl)
    feats = torch.empty((n, 64, 64), dtype=torch.bfloat16, device=device)
    labels = torch.zeros((n, 64, 64), dtype=torch.uint8, device=device)
    stats = dict(label_cells=0, grid_maxima=0, truth_tracks=0, truth_found=0)
    K = 1024
    a = 0
    for hits, offs, truth in generate("velo", RUN_SEED_TRAIN, n, chunk, workers):
        E = len(offs) - 1
        h = torch.from_numpy(hits).to(device)
        o = torch.from_numpy(offs).to(device)
        rt.slope_histogram(h, o, out=feats[a:a + E])
        srt, boxes = rt.prepare_hits(h, o, rt.VELO_SLOPES)
        g = rt.grid_scan(srt, o, rt.VELO_SLOPES, grid, wl.sigma_grid, wl.R0, K, boxes=boxes)
        nmax = np.minimum(g["n_max"].cpu().numpy(), K)
        th = g["max_theta"].cpu().numpy()
        lab = np.zeros((E, 64 * 64), np.uint8)
        for e in range(E):
            c = cells_of(th[e, :nmax[e]])
            lab[e, c[c >= 0]] = 1
            stats["grid_maxima"] += int(nmax[e])
            t = truth[e]
            stats["truth_tracks"] += len(t)
            if nmax[e] and len(t):
                d = np.abs(th[e, :nmax[e], None, :].astype(np.float64) - t[None]).max(-1)
                stats["truth_found"] += int((d <= 2 * wl.grid_step[0]).any(0).sum())
        stats["label_cells"] += int(lab.sum())
        labels[a:a + E].copy_(torch.from_numpy(lab.reshape(E, 64, 64)))
        a += E
    stats["grid_truth_efficiency"] = stats["truth_found"] / max(stats["truth_tracks"], 1)
    return feats, labels, stats


def train(feats, labels, epochs: int, batch: int, init_seed: int = 0, log_every: int = 100):
    from synth import seednet_init_params
    from .seednet import TrainState
    st = TrainState.fresh(seednet_init_params(init_seed), feats.device)
    n = feats.shape[0]
    curve: List[List[float]] = []
    for ep in range(epochs):
        for a in range(0, n - batch + 1, batch):
            rec = (st.n_steps % log_every) == 0
            st.step(feats[a:a + batch], labels[a:a + batch], record_loss=rec)
            if rec:
                curve.append([st.n_steps, st.losses[-1]])
    curve.append([st.n_steps, st.last_loss])
    return st, curve


def evaluate(params, n_events: int = 1024, workers: int = 8, k_learned=(512, 256), k_uniform=(4096, 512),
             device="cuda") -> Dict:
    """Held-out batch of ragged VELO-like events (tracks ~ Poisson(150) clipped
    to [20, 400], origin vertex, run seed 2000): MC-truth efficiency
    (|delta theta|_max <= 1e-3) and fakes of the batched search from uniform
    seeds and from learned seeds, and the fraction of the plain 4096-uniform
    method's tracks each learned variant recovers."""
    import torch
    from synth import WORKLOADS, uniform_seeds
    from . import retina as rt
    from .pipeline import BatchTracker, match_efficiency, recovered_fraction
    from .seednet import SeedProposer
    wl = WORKLOADS["velo_batch"]
    (hits, offs, truth), = list(generate("velo_batch", RUN_SEED_EVAL, n_events, n_events, 1))
    box = rt.Grid.of(wl)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    out = {"events": n_events, "hits": int(hits.shape[0])}
    found = {}
    for n in k_uniform:
        tr = BatchTracker(n_events, hits.shape[0], n, box, opts, wl.R0, device=device)
        S = np.stack([uniform_seeds(wl, n, RUN_SEED_EVAL, e) for e in range(n_events)])
        tr.load(hits, offs, S)
        tr.step()
        found["uniform_%d" % n] = tr.results()
    prop = SeedProposer(params, device=device)
    for k in k_learned:
        tr = BatchTracker(n_events, hits.shape[0], k, box, opts, wl.R0, proposer=prop, device=device)
        tr.load(hits, offs)
        tr.step()
        found["learned_%d" % k] = tr.results()
    torch.cuda.synchronize()
    plain = found["uniform_%d" % max(k_uniform)]
    for name, f in found.items():
        eff, fakes = match_efficiency(f, truth)
        out[name] = {"efficiency": eff, "fakes_per_event": fakes / n_events,
                     "recovers_plain": recovered_fraction(f, plain)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--events", type=int, default=100000)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--chunk", type=int, default=1024)
    ap.add_argument("--workers", type=int, default=max(1, min(16, (os.cpu_count() or 2) - 1)))
    ap.add_argument("--eval-events", type=int, default=1024)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    from .seednet import DEFAULT_WEIGHTS
    out = args.out or DEFAULT_WEIGHTS
    t0 = time.time()
    feats, labels, stats = build_dataset(args.events, args.chunk, args.workers)
    t1 = time.time()
    st, curve = train(feats, labels, args.epochs, args.batch)
    import torch
    torch.cuda.synchronize()
    t2 = time.time()
    ev = evaluate(st.params.cpu().numpy(), args.eval_events, args.workers)
    t3 = time.time()
    meta = {"recipe": {"events": args.events, "run_seed": RUN_SEED_TRAIN, "workload": "velo, origin vertex",
                       "labels": "64x64 cells of the 1024^2 grid-scan maxima above R0",
                       "epochs": args.epochs, "batch": args.batch, "init_seed": 0},
            "dataset": stats, "loss_curve": curve, "eval": ev,
            "seconds": {"data": t1 - t0, "train": t2 - t1, "eval": t3 - t2}}
    os.makedirs(os.path.dirname(os.path.abspath(out)), exist_ok=True)
    st.save(out, meta=meta)
    print(json.dumps({"checkpoint": out, "steps": st.n_steps, "final_loss": st.last_loss, "dataset": stats,
                      "eval": ev, "seconds": meta["seconds"]}))


if __name__ == "__main__":
    main()
