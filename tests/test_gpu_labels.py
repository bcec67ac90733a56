"""Training labels of the learned proposer (reading A18) against the oracle.

The labels mark the 64 x 64 slope cells that hold a maximum of the plain grid
method (Eq. 2 on the 1024 x 1024 grid at the grid bandwidth, strict local
maxima above R0).  They are built with the parity-tested GPU grid scan over
100k events; here the oracle's own grid and maxima on the first training
events must give the same cells (all of them: these events hold no near-tie
maxima; the bound leaves 1 % for a tie).
"""
import numpy as np
import pytest

import oracle
from synth import WORKLOADS

pytestmark = pytest.mark.gpu


def test_training_labels_match_the_oracle_grid_maxima():
    from paper_1709_08610_gb300 import build as rbuild
    rbuild.build()
    from paper_1709_08610_gb300 import train_seednet as ts
    n = 3
    _, labels, stats = ts.build_dataset(n, n, 1)
    lab = labels.cpu().numpy().reshape(n, -1).astype(bool)
    wl = WORKLOADS["velo"]
    n0, n1 = wl.grid_n
    c0, c1 = oracle.cell_centres(wl.grid_lo, wl.grid_step, wl.grid_n)
    hits, offs, truth = next(ts.generate("velo", ts.RUN_SEED_TRAIN, n, n, 1))
    total = 0
    for e in range(n):
        h = hits[offs[e]:offs[e + 1]]
        R = oracle.grid_response(h, 1, wl.grid_lo, wl.grid_step, wl.grid_n, wl.sigma_grid)
        idx = oracle.grid_maxima(R, float(np.float32(wl.R0)))
        cells = ts.cells_of(np.stack([c0[idx % n0], c1[idx // n0]], 1))
        exp = np.zeros(64 * 64, bool)
        exp[cells[cells >= 0]] = True
        union, diff = int((exp | lab[e]).sum()), int((exp ^ lab[e]).sum())
        assert union > 50  # ~150 tracks per event, many sharing cells
        assert diff <= 0.01 * union, (e, diff, union)
        total += int(exp.sum())
    assert stats["label_cells"] == int(lab.sum())
    assert total > 0
