"""Learned seed proposer: training state, checkpoints and the proposal pipeline.

A small convolutional network (retina_seednet_* in include/retina.h) ranks the
64 x 64 cells of an event's hit-slope histogram; the K best cells' hit
centroids become the starting points of Algorithm 1's local searches in place
of a uniform draw from the prior P_theta.  Every step runs in the library's
CUDA kernels; this module only owns buffers, the Adam step counter and the
checkpoint file.

Checkpoint format (little-endian, self-describing, stable across machines):
    line 1  b"RETINA-SEEDNET 1\\n"
    line 2  one JSON object + "\\n": {"n_params", "n_steps", "arrays": [names],
            "sha256" (of the payload), "lr", "betas", "eps", "layout", "meta"}
    payload float32 params, then Adam's m and v (n_params values each).
Resuming from a checkpoint continues bit for bit: params, m, v and the step
counter are all the optimiser state there is, and every kernel of the
training step is deterministic.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Dict, List, Optional

import numpy as np
import torch

from . import retina as rt

MAGIC = b"RETINA-SEEDNET 1\n"
N_PARAMS = rt.SEEDNET_PARAMS
LAYOUT = {"W1": [0, 144], "b1": [144, 160], "W2": [160, 4768], "b2": [4768, 4800], "W3": [4800, 4832],
          "b3": [4832, 4833]}
DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "seednet_velo.ckpt")


def _write_checkpoint(path: str, arrays: Dict[str, np.ndarray], header: Dict):
    payload = b"".join(np.ascontiguousarray(arrays[k], dtype="<f4").tobytes() for k in ("params", "m", "v"))
    head = dict(header)
    head.update(n_params=N_PARAMS, arrays=["params", "m", "v"], layout=LAYOUT,
                sha256=hashlib.sha256(payload).hexdigest())
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "wb") as f:
        f.write(MAGIC)
        f.write((json.dumps(head, sort_keys=True) + "\n").encode())
        f.write(payload)
    os.replace(tmp, path)


def read_checkpoint(path: str):
    """(header dict, {"params", "m", "v"} float32 numpy arrays); checks magic, size and hash."""
    with open(path, "rb") as f:
        if f.readline() != MAGIC:
            raise ValueError("%s is not a seed-net checkpoint" % path)
        head = json.loads(f.readline().decode())
        payload = f.read()
    n = int(head["n_params"])
    if n != N_PARAMS or len(payload) != 3 * 4 * n:
        raise ValueError("%s: wrong size" % path)
    if hashlib.sha256(payload).hexdigest() != head["sha256"]:
        raise ValueError("%s: payload hash mismatch" % path)
    arr = np.frombuffer(payload, dtype="<f4").reshape(3, n)
    return head, {"params": arr[0].copy(), "m": arr[1].copy(), "v": arr[2].copy()}


class TrainState:
    """FP32 master weights plus Adam state on the device; one call = one step."""

    def __init__(self, params: torch.Tensor, m: torch.Tensor, v: torch.Tensor, n_steps: int = 0, lr: float = 1e-3,
                 betas=(0.9, 0.999), eps: float = 1e-8, meta: Optional[Dict] = None):
        self.params, self.m, self.v = params, m, v
        self.n_steps = int(n_steps)
        self.lr, self.betas, self.eps = float(lr), tuple(float(b) for b in betas), float(eps)
        self.meta = dict(meta or {})
        self.losses: List[float] = []
        dev = params.device
        self._loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self._ws = torch.empty(0, dtype=torch.uint8, device=dev)

    @staticmethod
    def fresh(params: np.ndarray, device="cuda", **kw) -> "TrainState":
        p = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).to(device)
        return TrainState(p, torch.zeros_like(p), torch.zeros_like(p), 0, **kw)

    def step(self, features: torch.Tensor, labels: torch.Tensor, record_loss: bool = True):
        E = features.numel() // 4096
        need = rt.seednet_train_workspace_size(E)
        if self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=features.device)
        rt.seednet_train_step(features, labels, self.params, self.m, self.v, self.n_steps + 1, lr=self.lr,
                              betas=self.betas, eps=self.eps, loss=self._loss, ws=self._ws)
        self.n_steps += 1
        if record_loss:
            self.losses.append(float(self._loss.item()))

    @property
    def last_loss(self) -> float:
        return float(self._loss.item())

    def save(self, path: str, meta: Optional[Dict] = None):
        m = dict(self.meta)
        m.update(meta or {})
        _write_checkpoint(path, {"params": self.params.cpu().numpy(), "m": self.m.cpu().numpy(),
                                 "v": self.v.cpu().numpy()},
                          {"n_steps": self.n_steps, "lr": self.lr, "betas": list(self.betas), "eps": self.eps,
                           "meta": m})

    @staticmethod
    def load(path: str, device="cuda") -> "TrainState":
        head, a = read_checkpoint(path)
        t = {k: torch.from_numpy(a[k]).to(device) for k in a}
        return TrainState(t["params"], t["m"], t["v"], head["n_steps"], head["lr"], head["betas"], head["eps"],
                          head.get("meta"))


class SeedProposer:
    """Histogram -> network -> ranked cells -> seeds at dense sub-cells, on the
    current stream.

    ``propose`` reuses its buffers while the event count stays the same, so it
    can be captured in a CUDA graph together with the search that follows.
    """

    def __init__(self, params, lo: float = -0.5, hi: float = 0.5, zmin: float = 50.0, min_sub_hits: int = 3,
                 device="cuda"):
        if isinstance(params, np.ndarray):
            params = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).to(device)
        if params.numel() != N_PARAMS:
            raise ValueError("expected %d parameters" % N_PARAMS)
        self.params = params
        self.lo, self.hi, self.zmin, self.min_sub_hits = float(lo), float(hi), float(zmin), int(min_sub_hits)
        self._E = -1

    @staticmethod
    def from_checkpoint(path: str = DEFAULT_WEIGHTS, device="cuda", **kw) -> "SeedProposer":
        _, a = read_checkpoint(path)
        return SeedProposer(a["params"], device=device, **kw)

    def _buffers(self, E: int, dev):
        if E != self._E:
            self.feat = torch.empty((E, 64, 64), dtype=torch.bfloat16, device=dev)
            self.logits = torch.empty((E, 64, 64), dtype=torch.float32, device=dev)
            self.h1 = torch.empty((E, 16, 64, 64), dtype=torch.bfloat16, device=dev)
            self._E = E

    def propose(self, hits: torch.Tensor, offsets: torch.Tensor, K: int, seeds: Optional[torch.Tensor] = None,
                stream=None) -> torch.Tensor:
        """float32 [E, K, 2] seeds for the events of (hits, offsets)."""
        E = offsets.numel() - 1
        self._buffers(E, hits.device)
        rt.slope_histogram(hits, offsets, self.lo, self.hi, self.zmin, out=self.feat, stream=stream)
        rt.seednet_forward(self.feat, self.params, logits=self.logits, h1=self.h1, stream=stream)
        return rt.topk_seeds(self.logits, K, self.lo, self.hi, hits=hits, offsets=offsets, zmin=self.zmin,
                             min_sub_hits=self.min_sub_hits, seeds=seeds, stream=stream)
