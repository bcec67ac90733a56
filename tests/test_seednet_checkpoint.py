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
