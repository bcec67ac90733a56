"""Seed-net checkpoint file: round trip, integrity checks, and (when the
trained weights are present) what the trained network does, run by the FP64
oracle on the CPU."""
import os

import numpy as np
import pytest

from synth import seednet_init_params

torch = pytest.importorskip("torch")
from paper_1709_08610_gb300 import build as rbuild  # noqa: E402

rbuild.build()
from paper_1709_08610_gb300 import seednet as snet  # noqa: E402


def test_checkpoint_round_trip_and_integrity(tmp_path):
    p = seednet_init_params(1)
    rng = np.random.default_rng(0)
    m = rng.normal(0, 1e-3, p.size).astype(np.float32)
    v = rng.uniform(0, 1e-6, p.size).astype(np.float32)
    path = os.path.join(tmp_path, "a.ckpt")
    snet._write_checkpoint(path, {"params": p, "m": m, "v": v}, {"n_steps": 7, "lr": 1e-3, "betas": [0.9, 0.999],
                                                                   "eps": 1e-8, "meta": {"k": 1}})
    head, a = snet.read_checkpoint(path)
    assert head["n_steps"] == 7 and head["meta"] == {"k": 1} and head["n_params"] == 4833
    for k, x in (("params", p), ("m", m), ("v", v)):
        assert np.array_equal(a[k].view(np.uint32), x.view(np.uint32))
    raw = bytearray(open(path, "rb").read())
    raw[-5] ^= 1
    open(path, "wb").write(bytes(raw))
    with pytest.raises(ValueError, match="hash"):
        snet.read_checkpoint(path)
    open(path, "wb").write(bytes(raw[:-4]))
    with pytest.raises(ValueError, match="size"):
        snet.read_checkpoint(path)
    open(path, "wb").write(b"not a checkpoint\n")
    with pytest.raises(ValueError, match="not a seed-net"):
        snet.read_checkpoint(path)


def test_trained_network_run_by_the_oracle_ranks_every_track_cell():
    """The committed weights, run through the FP64 oracle on held-out
    origin-vertex events: every true track's cell ranks within the first 256
    cells, and the oracle's own truncated-Newton search from the proposer's
    512 seeds finds >= 97% of the true tracks."""
    import oracle
    from oracle import seednet as sn
    from synth import WORKLOADS, make_event
    head, a = snet.read_checkpoint(snet.DEFAULT_WEIGHTS)
    assert head["n_steps"] > 0 and np.all(np.isfinite(a["params"]))
    wl = WORKLOADS["velo_batch"]
    found = total = 0
    for e in range(2):
        ev = make_event(wl, 6000, e, vertex_sigma=(0, 0, 0))
        _, f = sn.slope_histogram(ev.hits)
        z = sn.forward(f, a["params"])["z"].astype(np.float32)
        order, _ = sn.top_k(z, 256)
        t = ev.truth[:, :2]
        c = np.floor((t + 0.5) * 64).astype(int)
        assert np.all(np.isin(c[:, 1] * 64 + c[:, 0], order))
        S, _ = sn.propose_seeds(z, ev.hits, 512)
        th, R, st, _ = oracle.local_search(ev.hits, 1, S.astype(np.float32), wl.sigma_schedule, wl.grid_lo,
                                           wl.grid_step, wl.grid_n)
        keep = oracle.extract_tracks(th, R, st, wl.grid_lo, wl.grid_step, wl.grid_n, wl.R0, 2.0)
        d = np.abs(th[keep][:, None, :] - t[None]).max(-1)
        found += int((d <= 1e-3).any(0).sum())
        total += len(t)
    assert found >= 0.97 * total, found / total
