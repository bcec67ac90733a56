"""Readings of Section 3's search against its cost model and its sVELO result
(test infrastructure: runs the FP64 oracle only).

Section 3 names the update (truncated Newton), its cost (C0 ~ 30 response
evaluations per step), the bandwidth schedule and the seed budget
n = alpha n_grid / (C0 q), and reports an efficiency close to 1 at
alpha = 1/3 on sVELO events; it leaves open the prior P_theta of
Algorithm 1, the truncation of the Newton step and the step control.  This
script runs the oracle's search under several readings of those open points
on sVELO events with 50 to 350 reconstructible tracks and prints, per
reading, the response evaluations per update (a gradient/Hessian evaluation
counted as C = 3, the paper's ratio, plus the line-search trials) and the
efficiency (an estimate within 1e-3 rad of a track in the paper's angles).

  python -m oracle.study_search_readings [--events-per-multiplicity N]
"""
from __future__ import annotations

import argparse
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synth import WORKLOADS, make_event, slopes_to_angles, uniform_seeds  # noqa: E402
from synth.events import _rng  # noqa: E402

MULTIPLICITIES = (50, 100, 150, 200, 250, 300, 350)
RUN_SEED = 9100
N_GRID = (2 * 0.705 / 1e-3) ** 2  # cells of 1e-3 rad over the angular acceptance (eta >= 1)


def physics_prior_seeds(n: int, event_id: int) -> np.ndarray:
    """Seeds drawn from the tracks' own direction distribution (eta ~ U[1, 6],
    phi ~ U[0, 2 pi)), as slopes (u, v)."""
    rng = _rng(RUN_SEED, event_id, 7)
    eta = rng.uniform(1.0, 6.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    tp = np.tan(2.0 * np.arctan(np.exp(-eta)))
    return np.stack([tp * np.cos(phi), tp * np.sin(phi)], 1).astype(np.float32)


READINGS = [
    # name, prior, step cap (cells), halvings
    ("A8: uniform box prior, cap 4 cells, <= 8 halvings", "box", 4.0, 8),
    ("uniform box prior, no cap", "box", 1e9, 8),
    ("uniform box prior, cap 16 cells", "box", 16.0, 8),
    ("uniform box prior, cap 4 cells, <= 20 halvings", "box", 4.0, 20),
    ("track-direction prior, cap 4 cells", "physics", 4.0, 8),
    ("track-direction prior, no cap", "physics", 1e9, 8),
]


def run(events_per_mult: int, alphas=(1.0 / 3.0, 0.1), readings=READINGS, c0=None) -> list:
    """Each reading at the seed budget n = alpha n_grid / (C0 q): C0 = 30 (the
    paper's) by default, or, with c0 = {reading name: C0}, the cost that
    reading measured (the same compute as the grid fraction alpha)."""
    wl = WORKLOADS["svelo"]
    evs = []
    for k, m in enumerate(MULTIPLICITIES):
        for r in range(events_per_mult):
            evs.append(make_event(wl, RUN_SEED, k * 1000 + r, n_tracks=m))
    rows = []
    for alpha in alphas:
        for name, prior, cap, halvings in readings:
            n = int(round(alpha * N_GRID / ((30.0 if c0 is None else c0[name]) * 3)))
            t0 = time.time()
            found = truth = 0
            trials = []
            for e, ev in enumerate(evs):
                seeds = uniform_seeds(wl, n, RUN_SEED, e) if prior == "box" else physics_prior_seeds(n, e)
                th, R, st, tr = oracle.local_search(ev.hits, 1, seeds, wl.sigma_schedule, wl.grid_lo, wl.grid_step,
                                                    wl.grid_n, max_halvings=halvings, step_cap_cells=cap,
                                                    count_trials=True)
                trials.append(tr)
                keep = oracle.extract_tracks(th, R, st, wl.grid_lo, wl.grid_step, wl.grid_n, wl.R0, wl.merge_cells)
                a_t = slopes_to_angles(ev.truth[:, 0], ev.truth[:, 1])
                a_f = slopes_to_angles(th[keep, 0], th[keep, 1]) if len(keep) else np.zeros((0, 2))
                truth += len(a_t)
                if len(a_f):
                    d = np.max(np.abs(a_f[:, None, :] - a_t[None, :, :]), axis=2)
                    found += int((d.min(axis=0) <= 1e-3).sum())
            q = len(wl.sigma_schedule)
            per_update = 3.0 + float(np.concatenate(trials).mean()) / q
            rows.append(dict(alpha=alpha, seeds=n, reading=name, evals_per_update=per_update,
                             efficiency=found / truth, events=len(evs), seconds=time.time() - t0))
            print("alpha %.3f  %-48s  %6d seeds  %5.2f R-evals/update  efficiency %.3f  (%d events, %.0f s)"
                  % (alpha, name, n, per_update, found / truth, len(evs), time.time() - t0), flush=True)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--events-per-multiplicity", type=int, default=4)
    args = ap.parse_args()
    oracle.build()
    print("seed budgets with the paper's C0 = 30:")
    rows = run(args.events_per_multiplicity)
    # the same compute with each reading's own measured cost per update
    picks = [READINGS[0], READINGS[4]]
    c0 = {r["reading"]: r["evals_per_update"] for r in rows if r["alpha"] == rows[0]["alpha"]}
    print("seed budgets with each reading's measured C0:")
    run(args.events_per_multiplicity, readings=picks, c0=c0)


if __name__ == "__main__":
    main()
