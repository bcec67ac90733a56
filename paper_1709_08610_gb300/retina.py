"""Thin Python binding of libretina (include/retina.h): argument marshalling only.

Every function takes and returns torch CUDA tensors, allocates its outputs
and workspace with torch (device memory and streams are torch's job here),
calls the C entry point of the same name on the current stream and raises
``RetinaError`` on a non-zero status.  There is no CPU path: if the compiled
library is missing the import of this module fails loudly.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

from . import build as _build

TOY2D = 0
VELO_SLOPES = 1
GRID_AUTO, GRID_DIRECT, GRID_SEPARABLE, GRID_TENSOR = 0, 1, 2, 3
MAX_Q = 8
MAX_EXTRACT_POINTS = 8192
OPT_LS_SEEDS_PER_WARP, OPT_LS_SMEM_HITS, OPT_GRID_SPLITS, OPT_LS_WARPS = 1, 2, 3, 4
OPT_BATCH_SEEDS_PER_WARP, OPT_BATCH_WARPS, OPT_BATCH_SMEM_HITS, OPT_BATCH_CTAS = 5, 6, 7, 8
UPDATE_TRUNCATED_NEWTON, UPDATE_STEEPEST_ASCENT, UPDATE_MODIFIED_NEWTON = 0, 1, 2
OPT_SEEDNET_TC = 9
OPT_GRID_TC = 10

HEADER = os.path.join(_build.INCLUDE, "retina.h")


class RetinaError(RuntimeError):
    def __init__(self, fn: str, code: int, text: str):
        super().__init__("%s failed: %s (status %d)" % (fn, text, code))
        self.code = code


class _CGrid(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 2), ("step", ctypes.c_float * 2), ("n", ctypes.c_int32 * 2)]


class _CLsOpts(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int32), ("sigma", ctypes.c_float * 8), ("c1", ctypes.c_float),
                ("max_halvings", ctypes.c_int32), ("step_cap_cells", ctypes.c_float), ("update", ctypes.c_int32)]


@dataclass(frozen=True)
class Grid:
    """Grid of units / search box: centres lo + (i + 1/2) step, i < n."""

    lo: Tuple[float, float]
    step: Tuple[float, float]
    n: Tuple[int, int]

    def c(self) -> _CGrid:
        g = _CGrid()
        for a in range(2):
            g.lo[a] = float(self.lo[a])
            g.step[a] = float(self.step[a])
            g.n[a] = int(self.n[a])
        return g

    @staticmethod
    def of(wl) -> "Grid":
        return Grid(tuple(wl.grid_lo), tuple(wl.grid_step), tuple(wl.grid_n))


@dataclass(frozen=True)
class LsOpts:
    """Local-search options (Algorithm 1, Section 3)."""

    sigma: Tuple[float, ...] = (0.3, 0.175, 0.05)
    c1: float = 1e-4
    max_halvings: int = 8
    step_cap_cells: float = 4.0
    update: int = 0  # UPDATE_TRUNCATED_NEWTON / UPDATE_STEEPEST_ASCENT / UPDATE_MODIFIED_NEWTON

    def c(self) -> _CLsOpts:
        o = _CLsOpts()
        o.q = len(self.sigma)
        for j, v in enumerate(self.sigma[:8]):
            o.sigma[j] = float(v)
        o.c1 = float(self.c1)
        o.max_halvings = int(self.max_halvings)
        o.step_cap_cells = float(self.step_cap_cells)
        o.update = int(self.update)
        return o


class _CLs4Opts(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int32), ("sigma", ctypes.c_float * 8), ("c1", ctypes.c_float),
                ("max_halvings", ctypes.c_int32), ("scale", ctypes.c_float * 4), ("step_cap", ctypes.c_float),
                ("zref", ctypes.c_float)]


@dataclass(frozen=True)
class LsOpts4:
    """Options of the four-parameter search (x0, y0, t_x, t_y) at the plane
    ``zref``; ``scale`` is each parameter's unit (about one peak width: CG
    scaling and step cap)."""

    sigma: Tuple[float, ...] = (0.3, 0.175, 0.05)
    scale: Tuple[float, float, float, float] = (0.25, 0.25, 2.0 ** -10, 2.0 ** -10)
    step_cap: float = 4.0
    zref: float = 0.0
    c1: float = 1e-4
    max_halvings: int = 8

    def c(self) -> _CLs4Opts:
        o = _CLs4Opts()
        o.q = len(self.sigma)
        for j, v in enumerate(self.sigma[:8]):
            o.sigma[j] = float(v)
        o.c1 = float(self.c1)
        o.max_halvings = int(self.max_halvings)
        for a in range(4):
            o.scale[a] = float(self.scale[a])
        o.step_cap = float(self.step_cap)
        o.zref = float(self.zref)
        return o


class _CPipelineConfig(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("grid", _CGrid), ("sigma_grid", ctypes.c_float), ("R0", ctypes.c_float),
                ("merge_cells", ctypes.c_float), ("opts", _CLsOpts), ("max_events", ctypes.c_int32),
                ("max_hits", ctypes.c_int64), ("seeds_per_event", ctypes.c_int32), ("max_maxima", ctypes.c_int32),
                ("max_tracks", ctypes.c_int32)]


class _CTrackerConfig(ctypes.Structure):
    _fields_ = [("box", _CGrid), ("opts", _CLsOpts), ("R0", ctypes.c_float), ("merge_cells", ctypes.c_float),
                ("max_events", ctypes.c_int32), ("max_hits", ctypes.c_int64), ("seeds_per_event", ctypes.c_int32),
                ("max_tracks", ctypes.c_int32), ("sort_seeds", ctypes.c_int32), ("seeds_per_warp", ctypes.c_int32),
                ("warps", ctypes.c_int32), ("smem_hits", ctypes.c_int32), ("ctas", ctypes.c_int32),
                ("use_graph", ctypes.c_int32)]


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError("libretina.so is not built (%s); run paper_1709_08610_gb300.build.build()" % path)
    L = ctypes.CDLL(path)
    P, I32, I64, F, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
    L.retina_pipeline_create.argtypes = [P, P]
    L.retina_pipeline_run.argtypes = [P, P, I64, P, I32, P, P, P, P, P, P, P, P]
    L.retina_pipeline_destroy.argtypes = [P]
    L.retina_pair_seeds4.argtypes = [P, I64, P, I32, P, I32, F, F, F, F, F, P, P, I32, P]
    L.retina_extract_tracks_workspace_size.argtypes = [I32, I32, P]
    L.retina_extract_tracks_ws.argtypes = [P, P, P, P, I32, I32, P, F, F, P, P, P, P, I32, P, SZ, P]
    L.retina_extract_tracks4.argtypes = [P, P, P, P, I32, I32, P, P, F, F, P, P, P, P, I32, P]
    L.retina_tracker_create.argtypes = [P, P, P]
    L.retina_tracker_buffers.argtypes = [P, P, P, P, P, P, P]
    L.retina_tracker_step.argtypes = [P, I32, P]
    L.retina_tracker_set_marks.argtypes = [P, P, I32]
    L.retina_tracker_run_host.argtypes = [P, P, I64, P, I32, P, P, P, P, P]
    L.retina_tracker_destroy.argtypes = [P]
    L.retina_strerror.argtypes = [ctypes.c_int]
    L.retina_strerror.restype = ctypes.c_char_p
    L.retina_abi_version.restype = ctypes.c_int
    L.retina_set_option.argtypes = [I32, I32]
    L.retina_get_option.argtypes = [I32, P]
    L.retina_grid_scan_workspace_size.argtypes = [I32, I32, P, I32, I32, P]
    L.retina_grid_scan.argtypes = [P, I64, P, P, I32, I32, P, F, F, I32, P, P, P, P, P, I32, P, SZ, P]
    L.retina_grid_maxima_workspace_size.argtypes = [I32, P, P]
    L.retina_grid_maxima.argtypes = [P, I32, P, F, P, P, P, P, I32, P, SZ, P]
    L.retina_response.argtypes = [P, I64, P, I32, I32, P, I32, F, I32, P, P]
    L.retina_local_search.argtypes = [P, I64, P, P, I32, I32, P, I32, P, P, P, P, P, P, P]
    L.retina_refine_maxima_workspace_size.argtypes = [I32, P]
    L.retina_local_search4.argtypes = [P, I64, P, I32, P, I32, P, P, P, P, P, P]
    L.retina_refine_maxima.argtypes = [P, I64, P, P, I32, I32, P, P, I32, P, P, P, P, P, P, SZ, P]
    L.retina_extract_tracks.argtypes = [P, P, P, P, I32, I32, P, F, F, P, P, P, P, I32, P]
    L.retina_grid_response_workspace_size.argtypes = [I32, I32, P, I32, P]
    L.retina_grid_response.argtypes = [P, I64, P, P, I32, I32, P, F, I32, P, P, SZ, P]
    L.retina_prepare_hits_box_count.argtypes = [I64, I32]
    L.retina_prepare_hits_box_count.restype = I64
    L.retina_prepare_hits.argtypes = [P, I64, P, I32, I32, P, P, P]
    L.retina_work_counters.argtypes = [I32, I32, P]
    L.retina_device_error.argtypes = [P, I32]
    L.retina_sort_seeds.argtypes = [P, I64, P, I32, P, P, P, P]
    L.retina_launch_count.restype = ctypes.c_uint64
    L.retina_alu_probe_sink_floats.restype = ctypes.c_int64
    L.retina_alu_probe.argtypes = [I32, I32, P, P, P]
    L.retina_grid_maxima_static.argtypes = [P, I32, P, F, P, P, P, P, I32, P]
    L.retina_batched_search_workspace_size.argtypes = [I32, P]
    L.retina_batched_search.argtypes = [P, I64, P, P, I32, I32, P, I64, P, P, P, P, P, P, P, P, P, SZ, P]
    L.retina_slope_histogram.argtypes = [P, I64, P, I32, F, F, F, P, P, P]
    L.retina_seednet_forward.argtypes = [P, I32, P, P, P, P, P]
    L.retina_seednet_train_workspace_size.argtypes = [I32, P]
    L.retina_seednet_train_step.argtypes = [P, P, I32, P, P, P, I32, F, F, F, F, P, P, P, SZ, P]
    L.retina_seednet_adam.argtypes = [P, P, P, P, I32, F, F, F, F, P]
    L.retina_topk_seeds.argtypes = [P, I32, I32, F, F, F, I32, P, I64, P, P, P, P]
    for name in ("retina_set_option", "retina_get_option", "retina_grid_scan_workspace_size", "retina_grid_scan",
                 "retina_grid_response_workspace_size", "retina_grid_response", "retina_alu_probe",
                 "retina_grid_maxima_static", "retina_batched_search_workspace_size", "retina_batched_search",
                 "retina_prepare_hits", "retina_work_counters",
                 "retina_grid_maxima_workspace_size", "retina_grid_maxima", "retina_response",
                 "retina_local_search", "retina_extract_tracks", "retina_slope_histogram",
                 "retina_seednet_forward", "retina_seednet_train_workspace_size", "retina_seednet_train_step",
                 "retina_seednet_adam", "retina_topk_seeds", "retina_device_error",
                 "retina_sort_seeds", "retina_pair_seeds4", "retina_extract_tracks4",
                 "retina_extract_tracks_workspace_size", "retina_extract_tracks_ws"):
        getattr(L, name).restype = ctypes.c_int
    return L


lib = _load()


def header_functions() -> list:
    """Names of the functions include/retina.h declares."""
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(retina_\w+)\s*\(", src, flags=re.M)))


def _check(fn: str, code: int):
    if code != 0:
        raise RetinaError(fn, code, lib.retina_strerror(code).decode())


def _p(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, dtype, name: str, last: Optional[int] = None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if last is not None and (t.dim() < 1 or t.shape[-1] != last):
        raise ValueError("%s must have last dimension %d" % (name, last))
    return t


def set_option(option: int, value: int):
    _check("retina_set_option", lib.retina_set_option(option, value))


def get_option(option: int) -> int:
    v = ctypes.c_int32()
    _check("retina_get_option", lib.retina_get_option(option, ctypes.byref(v)))
    return v.value


def grid_scan_workspace_size(n_events: int, model: int, grid: Grid, flags: int = 0, store_R: bool = False) -> int:
    b = ctypes.c_size_t()
    g = grid.c()
    _check("retina_grid_scan_workspace_size",
           lib.retina_grid_scan_workspace_size(n_events, model, ctypes.byref(g), flags, int(store_R), ctypes.byref(b)))
    return b.value


def grid_scan(hits: torch.Tensor, offsets: torch.Tensor, model: int, grid: Grid, sigma: float, R0: float, K: int,
              flags: int = GRID_AUTO, store_R: bool = False, ws: Optional[torch.Tensor] = None, out=None,
              boxes: Optional[torch.Tensor] = None, stream=None) -> dict:
    """Eq. 2 on the grid plus strict local maxima >= R0 (grid algorithm steps 2-4)."""
    _dev(hits, torch.float32, "hits", 4)
    _dev(offsets, torch.int64, "offsets")
    E = offsets.numel() - 1
    dev = hits.device
    n0, n1 = grid.n
    if out is None:
        out = dict(max_idx=torch.empty((E, K), dtype=torch.int32, device=dev),
                   max_theta=torch.empty((E, K, 2), dtype=torch.float32, device=dev),
                   max_R=torch.empty((E, K), dtype=torch.float32, device=dev),
                   n_max=torch.empty((E,), dtype=torch.int32, device=dev),
                   R=torch.empty((E, n1, n0), dtype=torch.float32, device=dev) if store_R else None)
    need = grid_scan_workspace_size(E, model, grid, flags, store_R)
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    g = grid.c()
    _check("retina_grid_scan", lib.retina_grid_scan(
        _p(hits), hits.shape[0], _p(offsets), _p(boxes), E, model, ctypes.byref(g), float(sigma), float(R0), flags,
        _p(out["R"]), _p(out["max_idx"]), _p(out["max_theta"]), _p(out["max_R"]), _p(out["n_max"]), K,
        _p(ws), ws.numel(), _stream(stream)))
    return out


def grid_response(hits: torch.Tensor, offsets: torch.Tensor, model: int, grid: Grid, sigma: float,
                  flags: int = GRID_AUTO, R_out: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None,
                  boxes: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Eq. 2 alone: R [E, n1, n0]."""
    _dev(hits, torch.float32, "hits", 4)
    _dev(offsets, torch.int64, "offsets")
    E = offsets.numel() - 1
    n0, n1 = grid.n
    if R_out is None:
        R_out = torch.empty((E, n1, n0), dtype=torch.float32, device=hits.device)
    g = grid.c()
    b = ctypes.c_size_t()
    _check("retina_grid_response_workspace_size",
           lib.retina_grid_response_workspace_size(E, model, ctypes.byref(g), flags, ctypes.byref(b)))
    if ws is None or ws.numel() < b.value:
        ws = torch.empty(max(b.value, 1), dtype=torch.uint8, device=hits.device)
    _check("retina_grid_response", lib.retina_grid_response(
        _p(hits), hits.shape[0], _p(offsets), _p(boxes), E, model, ctypes.byref(g), float(sigma), flags, _p(R_out), _p(ws),
        ws.numel(), _stream(stream)))
    return R_out


def grid_response_workspace_size(n_events: int, model: int, grid: Grid, flags: int = 0) -> int:
    g = grid.c()
    b = ctypes.c_size_t()
    _check("retina_grid_response_workspace_size",
           lib.retina_grid_response_workspace_size(n_events, model, ctypes.byref(g), flags, ctypes.byref(b)))
    return b.value


WORK_GRID, WORK_RGH, WORK_R = 0, 1, 2


def work_counters(enable: Optional[bool] = None, reset: bool = False) -> list:
    """Read (and optionally reset / switch) the device work counters."""
    out = (ctypes.c_uint64 * 4)()
    _check("retina_work_counters", lib.retina_work_counters(-1 if enable is None else int(enable), int(reset), out))
    return list(out)


def device_error(reset: bool = False) -> int:
    """The library's device-side error flag (1 after a kernel's bounded wait expired)."""
    v = ctypes.c_int32()
    _check("retina_device_error", lib.retina_device_error(ctypes.byref(v), int(reset)))
    return v.value


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib.retina_launch_count())


def alu_probe(kind: int, iters: int, sink: torch.Tensor, stream=None) -> float:
    """Launch the FP32 (0), MUFU ex2 (1) or packed FP32x2 (2) throughput probe; returns its op count."""
    ops = ctypes.c_double()
    _check("retina_alu_probe", lib.retina_alu_probe(kind, iters, _p(sink), ctypes.byref(ops), _stream(stream)))
    return ops.value


def alu_probe_sink_floats() -> int:
    return int(lib.retina_alu_probe_sink_floats())


def prepare_hits(hits: torch.Tensor, offsets: torch.Tensor, model: int, out=None,
                 stream=None) -> Tuple[torch.Tensor, torch.Tensor]:
    """Spatially ordered hits and per-32-hit boxes for exact block skipping."""
    _dev(hits, torch.float32, "hits", 4)
    _dev(offsets, torch.int64, "offsets")
    E = offsets.numel() - 1
    nb = int(lib.retina_prepare_hits_box_count(hits.shape[0], E))
    if out is None:
        out = (torch.empty_like(hits), torch.empty((nb, 8), dtype=torch.float32, device=hits.device))
    _check("retina_prepare_hits", lib.retina_prepare_hits(_p(hits), hits.shape[0], _p(offsets), E, model, _p(out[0]),
                                                          _p(out[1]), _stream(stream)))
    return out


def grid_maxima(R: torch.Tensor, grid: Grid, R0: float, K: int, out=None, ws=None, stream=None) -> dict:
    """Strict 3x3 local maxima >= R0 of a response grid [E, n1, n0]."""
    _dev(R, torch.float32, "R")
    E = R.shape[0]
    dev = R.device
    b = ctypes.c_size_t()
    g = grid.c()
    _check("retina_grid_maxima_workspace_size", lib.retina_grid_maxima_workspace_size(E, ctypes.byref(g),
                                                                                        ctypes.byref(b)))
    if ws is None or ws.numel() < b.value:
        ws = torch.empty(max(b.value, 1), dtype=torch.uint8, device=dev)
    if out is None:
        out = dict(max_idx=torch.empty((E, K), dtype=torch.int32, device=dev),
               max_theta=torch.empty((E, K, 2), dtype=torch.float32, device=dev),
               max_R=torch.empty((E, K), dtype=torch.float32, device=dev),
               n_max=torch.empty((E,), dtype=torch.int32, device=dev))
    _check("retina_grid_maxima", lib.retina_grid_maxima(
        _p(R), E, ctypes.byref(g), float(R0), _p(out["max_idx"]), _p(out["max_theta"]), _p(out["max_R"]),
        _p(out["n_max"]), K, _p(ws), ws.numel(), _stream(stream)))
    return out


def response(hits: torch.Tensor, offsets: torch.Tensor, model: int, theta: torch.Tensor, sigma: float,
             want_derivs: bool = True, stream=None) -> torch.Tensor:
    """[E, P, 6] = (R, g0, g1, H00, H01, H11) at theta [E, P, 2] (Eq. 1 + derivatives)."""
    _dev(hits, torch.float32, "hits", 4)
    _dev(offsets, torch.int64, "offsets")
    _dev(theta, torch.float32, "theta", 2)
    E = offsets.numel() - 1
    P = theta.shape[-2] if theta.dim() == 3 else theta.shape[0]
    out = torch.zeros((E, P, 6), dtype=torch.float32, device=hits.device)
    _check("retina_response", lib.retina_response(_p(hits), hits.shape[0], _p(offsets), E, model, _p(theta), P,
                                                  float(sigma), int(want_derivs), _p(out), _stream(stream)))
    return out


def refine_opts(sigma_grid: float, iters: int = 4, step_cap_cells: float = 1.0) -> LsOpts:
    """Options of the grid-maximum refinement: ``iters`` updates at the grid's
    own bandwidth, each step capped to ``step_cap_cells`` cells."""
    return LsOpts(sigma=(float(sigma_grid),) * int(iters), step_cap_cells=float(step_cap_cells))


def refine_maxima_workspace_size(n_events: int) -> int:
    b = ctypes.c_size_t(0)
    _check("retina_refine_maxima_workspace_size", lib.retina_refine_maxima_workspace_size(n_events, ctypes.byref(b)))
    return b.value


def refine_maxima(hits: torch.Tensor, offsets: torch.Tensor, model: int, theta_c: torch.Tensor,
                  n_max: torch.Tensor, opts: LsOpts, box: Grid, out=None, ws: Optional[torch.Tensor] = None,
                  boxes: Optional[torch.Tensor] = None, stream=None) -> Tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
    """Step 4 of the grid algorithm: the first min(n_max[e], K) points of
    theta_c [E, K, 2] refined by opts' truncated-Newton updates; returns
    (theta [E, K, 2], R [E, K], status [E, K] uint8), rows past the count
    untouched."""
    _dev(hits, torch.float32, "hits", 4)
    _dev(offsets, torch.int64, "offsets")
    _dev(theta_c, torch.float32, "theta_c", 2)
    _dev(n_max, torch.int32, "n_max")
    E = offsets.numel() - 1
    K = theta_c.shape[-2]
    if theta_c.numel() != E * K * 2 or n_max.numel() != E:
        raise ValueError("theta_c must be [E, K, 2] and n_max [E]")
    dev = hits.device
    if out is None:
        out = (torch.empty((E, K, 2), dtype=torch.float32, device=dev),
               torch.empty((E, K), dtype=torch.float32, device=dev),
               torch.empty((E, K), dtype=torch.uint8, device=dev))
    need = refine_maxima_workspace_size(E)
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    o = opts.c()
    g = box.c()
    _check("retina_refine_maxima", lib.retina_refine_maxima(
        _p(hits), hits.shape[0], _p(offsets), _p(boxes), E, model, _p(theta_c), _p(n_max), K, ctypes.byref(o),
        ctypes.byref(g), _p(out[0]), _p(out[1]), _p(out[2]), _p(ws), ws.numel(), _stream(stream)))
    return out


def local_search4(hits: torch.Tensor, offsets: torch.Tensor, seeds: torch.Tensor, opts: LsOpts4, out=None,
                  stream=None, seed_count: Optional[torch.Tensor] = None) -> Tuple[torch.Tensor, torch.Tensor,
                                                                                   torch.Tensor]:
    """Algorithm 1 for four-parameter tracks: seeds [E, n, 4] ->
    (theta [E, n, 4], R [E, n], status [E, n] uint8); with seed_count [E]
    int32 only each event's first seed_count[e] seeds are searched."""
    _dev(hits, torch.float32, "hits", 4)
    _dev(offsets, torch.int64, "offsets")
    _dev(seeds, torch.float32, "seeds", 4)
    E = offsets.numel() - 1
    n = seeds.shape[-2]
    if seeds.numel() != E * n * 4:
        raise ValueError("seeds must be [E, n_seeds, 4]")
    dev = hits.device
    if out is None:
        out = (torch.empty((E, n, 4), dtype=torch.float32, device=dev),
               torch.empty((E, n), dtype=torch.float32, device=dev),
               torch.empty((E, n), dtype=torch.uint8, device=dev))
    o = opts.c()
    _check("retina_local_search4", lib.retina_local_search4(
        _p(hits), hits.shape[0], _p(offsets), E, _p(seeds), n, _p(seed_count), ctypes.byref(o), _p(out[0]),
        _p(out[1]), _p(out[2]), _stream(stream)))
    return out


def pair_seeds4(hits: torch.Tensor, offsets: torch.Tensor, layer_pairs, dz_tol: float, d_max: float, zc_range,
                zref: float, K: int, out=None, stream=None):
    """Starting points of the four-parameter search from hit pairs on the
    layer pairs [(z_a, z_b), ...] (retina_pair_seeds4); returns (seeds
    [E, K, 4], n_seeds [E] int32: pairs kept, may exceed K; -1 when a layer
    overflowed)."""
    _dev(hits, torch.float32, "hits", 4)
    _dev(offsets, torch.int64, "offsets")
    E = offsets.numel() - 1
    lz = np.ascontiguousarray(np.asarray(layer_pairs, dtype=np.float32).reshape(-1, 2))
    if out is None:
        out = (torch.empty((E, K, 4), dtype=torch.float32, device=hits.device),
               torch.empty((E,), dtype=torch.int32, device=hits.device))
    _check("retina_pair_seeds4", lib.retina_pair_seeds4(
        _p(hits), hits.shape[0], _p(offsets), E, lz.ctypes.data_as(ctypes.c_void_p), lz.shape[0], float(dz_tol),
        float(d_max), float(zc_range[0]), float(zc_range[1]), float(zref), _p(out[0]), _p(out[1]), int(K),
        _stream(stream)))
    return out


def extract_tracks4(theta: torch.Tensor, R: torch.Tensor, status: Optional[torch.Tensor], slope_box: Grid, unit,
                    R0: float, merge_units: float, K: int, n_valid: Optional[torch.Tensor] = None, out=None,
                    stream=None) -> dict:
    """Cluster / select of four-parameter points [E, n, 4] (retina_extract_tracks4)."""
    _dev(theta, torch.float32, "theta", 4)
    E, n = theta.shape[0], theta.shape[1]
    dev = theta.device
    if out is None:
        out = dict(tracks=torch.empty((E, K, 4), dtype=torch.float32, device=dev),
                   track_R=torch.empty((E, K), dtype=torch.float32, device=dev),
                   track_src=torch.empty((E, K), dtype=torch.int32, device=dev),
                   n_tracks=torch.empty((E,), dtype=torch.int32, device=dev))
    u = np.ascontiguousarray(np.asarray(unit, dtype=np.float32).reshape(4))
    g = slope_box.c()
    _check("retina_extract_tracks4", lib.retina_extract_tracks4(
        _p(theta), _p(R), _p(status), _p(n_valid), E, n, ctypes.byref(g), u.ctypes.data_as(ctypes.c_void_p), float(R0),
        float(merge_units), _p(out["tracks"]), _p(out["track_R"]), _p(out["track_src"]), _p(out["n_tracks"]), int(K),
        _stream(stream)))
    return out


def local_search(hits: torch.Tensor, offsets: torch.Tensor, model: int, seeds: torch.Tensor, opts: LsOpts,
                 box: Grid, out=None, n_evals: Optional[torch.Tensor] = None, boxes: Optional[torch.Tensor] = None,
                 stream=None) -> Tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
    """Algorithm 1's q truncated-Newton updates: (theta [E,n,2], R [E,n], status [E,n] uint8).

    n_evals (optional uint8 [E, n]) receives each seed's number of R-only passes.
    """
    _dev(hits, torch.float32, "hits", 4)
    _dev(offsets, torch.int64, "offsets")
    _dev(seeds, torch.float32, "seeds", 2)
    E = offsets.numel() - 1
    n = seeds.shape[-2]
    if seeds.numel() != E * n * 2:
        raise ValueError("seeds must be [E, n_seeds, 2]")
    dev = hits.device
    if out is None:
        out = (torch.empty((E, n, 2), dtype=torch.float32, device=dev),
               torch.empty((E, n), dtype=torch.float32, device=dev),
               torch.empty((E, n), dtype=torch.uint8, device=dev))
    o = opts.c()
    g = box.c()
    _check("retina_local_search", lib.retina_local_search(
        _p(hits), hits.shape[0], _p(offsets), _p(boxes), E, model, _p(seeds), n, ctypes.byref(o), ctypes.byref(g),
        _p(out[0]), _p(out[1]), _p(out[2]), _p(n_evals), _stream(stream)))
    return out


def batched_search_workspace_size(n_events: int) -> int:
    b = ctypes.c_size_t()
    _check("retina_batched_search_workspace_size", lib.retina_batched_search_workspace_size(n_events, ctypes.byref(b)))
    return b.value


def batched_search(hits: torch.Tensor, offsets: torch.Tensor, model: int, seeds: torch.Tensor,
                   seed_offsets: torch.Tensor, opts: LsOpts, box: Grid, order: Optional[torch.Tensor] = None,
                   out=None, n_evals: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None,
                   boxes: Optional[torch.Tensor] = None, stream=None) -> Tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
    """Algorithm 1 over a ragged batch in one persistent launch.

    seeds [S, 2] float32 with seed_offsets int64 [E + 1]; returns per seed
    (theta [S, 2], R [S], status [S] uint8).
    """
    _dev(hits, torch.float32, "hits", 4)
    _dev(offsets, torch.int64, "offsets")
    _dev(seeds, torch.float32, "seeds", 2)
    _dev(seed_offsets, torch.int64, "seed_offsets")
    if order is not None:
        _dev(order, torch.int32, "order")
    E = offsets.numel() - 1
    if seed_offsets.numel() != E + 1:
        raise ValueError("seed_offsets must have n_events + 1 entries")
    S = seeds.numel() // 2
    dev = hits.device
    if out is None:
        out = (torch.empty((S, 2), dtype=torch.float32, device=dev),
               torch.empty((S,), dtype=torch.float32, device=dev),
               torch.empty((S,), dtype=torch.uint8, device=dev))
    need = batched_search_workspace_size(E)
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    o = opts.c()
    g = box.c()
    _check("retina_batched_search", lib.retina_batched_search(
        _p(hits), hits.shape[0], _p(offsets), _p(boxes), E, model, _p(seeds), S, _p(seed_offsets), _p(order), ctypes.byref(o),
        ctypes.byref(g), _p(out[0]), _p(out[1]), _p(out[2]), _p(n_evals), _p(ws), ws.numel(), _stream(stream)))
    return out


def sort_seeds(seeds: torch.Tensor, seed_offsets: torch.Tensor, box: Grid, out: Optional[torch.Tensor] = None,
               perm: Optional[torch.Tensor] = None, want_perm: bool = False, stream=None):
    """Seeds [S, 2] in spatial order per event (and the int32 map to the original rows if asked)."""
    _dev(seeds, torch.float32, "seeds", 2)
    _dev(seed_offsets, torch.int64, "seed_offsets")
    E = seed_offsets.numel() - 1
    S = seeds.numel() // 2
    out = out if out is not None else torch.empty_like(seeds)
    if want_perm and perm is None:
        perm = torch.empty((S,), dtype=torch.int32, device=seeds.device)
    g = box.c()
    _check("retina_sort_seeds", lib.retina_sort_seeds(_p(seeds), S, _p(seed_offsets), E, ctypes.byref(g), _p(out),
                                                      _p(perm), _stream(stream)))
    return (out, perm) if (want_perm or perm is not None) else out


def extract_tracks_workspace_size(n_events: int, n_points: int) -> int:
    b = ctypes.c_size_t()
    _check("retina_extract_tracks_workspace_size", lib.retina_extract_tracks_workspace_size(n_events, n_points,
                                                                                           ctypes.byref(b)))
    return b.value


def extract_tracks(theta: torch.Tensor, R: torch.Tensor, status: Optional[torch.Tensor], box: Grid, R0: float,
                   merge_cells: float, K: int, n_valid: Optional[torch.Tensor] = None, out=None,
                   stream=None, ws: Optional[torch.Tensor] = None) -> dict:
    """Cluster + select best above R0 (Algorithm 1): kept points in visiting
    order.  Beyond RETINA_MAX_EXTRACT_POINTS points per event the candidates
    go to a workspace (retina_extract_tracks_ws; allocated here unless ws is
    given)."""
    _dev(theta, torch.float32, "theta", 2)
    _dev(R, torch.float32, "R")
    if status is not None:
        _dev(status, torch.uint8, "status")
    if n_valid is not None:
        _dev(n_valid, torch.int32, "n_valid")
    E = theta.shape[0] if theta.dim() == 3 else 1
    n = theta.shape[-2]
    dev = theta.device
    if out is None:
        out = dict(tracks=torch.empty((E, K, 2), dtype=torch.float32, device=dev),
                   track_R=torch.empty((E, K), dtype=torch.float32, device=dev),
                   track_src=torch.empty((E, K), dtype=torch.int32, device=dev),
                   n_tracks=torch.empty((E,), dtype=torch.int32, device=dev))
    g = box.c()
    need = extract_tracks_workspace_size(E, n)
    if need > 0 and (ws is None or ws.numel() < need):
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    _check("retina_extract_tracks_ws", lib.retina_extract_tracks_ws(
        _p(theta), _p(R), _p(status), _p(n_valid), E, n, ctypes.byref(g), float(R0), float(merge_cells),
        _p(out["tracks"]), _p(out["track_R"]), _p(out["track_src"]), _p(out["n_tracks"]), K,
        _p(ws) if need > 0 else None, ws.numel() if (need > 0 and ws is not None) else 0, _stream(stream)))
    return out


# ---------------------------------------------------------------------------
# learned seed proposer
# ---------------------------------------------------------------------------
SEEDNET_BINS = 64
SEEDNET_PARAMS = 4833


def slope_histogram(hits: torch.Tensor, offsets: torch.Tensor, lo: float = -0.5, hi: float = 0.5,
                    zmin: float = 50.0, out: Optional[torch.Tensor] = None, counts: bool = False,
                    counts_out: Optional[torch.Tensor] = None, stream=None):
    """bfloat16 [E, 64, 64] log1p of the slope histogram (and the int32 counts if asked)."""
    _dev(hits, torch.float32, "hits", 4)
    _dev(offsets, torch.int64, "offsets")
    E = offsets.numel() - 1
    dev = hits.device
    feat = out if out is not None else torch.empty((E, 64, 64), dtype=torch.bfloat16, device=dev)
    _dev(feat, torch.bfloat16, "out")
    counts = counts or counts_out is not None
    cnt = counts_out if counts_out is not None else (
        torch.empty((E, 64, 64), dtype=torch.int32, device=dev) if counts else None)
    if cnt is not None:
        _dev(cnt, torch.int32, "counts_out")
    _check("retina_slope_histogram", lib.retina_slope_histogram(
        _p(hits), hits.shape[0], _p(offsets), E, lo, hi, zmin, _p(feat), _p(cnt), _stream(stream)))
    return (feat, cnt) if counts else feat


def seednet_forward(features: torch.Tensor, params: torch.Tensor, logits: Optional[torch.Tensor] = None,
                    h1: Optional[torch.Tensor] = None, want_h2: bool = False, stream=None):
    """Logits float32 [E, 64, 64]; with want_h2 also (h1, h2) bfloat16 activations."""
    _dev(features, torch.bfloat16, "features")
    _dev(params, torch.float32, "params")
    if params.numel() != SEEDNET_PARAMS:
        raise ValueError("params must hold %d values" % SEEDNET_PARAMS)
    E = features.numel() // 4096
    dev = features.device
    logits = logits if logits is not None else torch.empty((E, 64, 64), dtype=torch.float32, device=dev)
    h1 = h1 if h1 is not None else torch.empty((E, 16, 64, 64), dtype=torch.bfloat16, device=dev)
    h2 = torch.empty((E, 32, 64, 64), dtype=torch.bfloat16, device=dev) if want_h2 else None
    _check("retina_seednet_forward", lib.retina_seednet_forward(
        _p(features), E, _p(params), _p(logits), _p(h1), _p(h2), _stream(stream)))
    return (logits, h1, h2) if want_h2 else logits


def seednet_train_workspace_size(n_events: int) -> int:
    b = ctypes.c_size_t()
    _check("retina_seednet_train_workspace_size", lib.retina_seednet_train_workspace_size(n_events, ctypes.byref(b)))
    return b.value


def seednet_train_step(features: torch.Tensor, labels: torch.Tensor, params: torch.Tensor, m: torch.Tensor,
                       v: torch.Tensor, step: int, lr: float = 1e-3, betas=(0.9, 0.999), eps: float = 1e-8,
                       loss: Optional[torch.Tensor] = None, grad: Optional[torch.Tensor] = None,
                       ws: Optional[torch.Tensor] = None, stream=None):
    """One Adam step on the weighted BCE; params, m, v updated in place."""
    _dev(features, torch.bfloat16, "features")
    _dev(labels, torch.uint8, "labels")
    for t, n in ((params, "params"), (m, "m"), (v, "v")):
        _dev(t, torch.float32, n)
    E = features.numel() // 4096
    if labels.numel() != E * 4096:
        raise ValueError("labels must match features")
    need = seednet_train_workspace_size(E)
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=features.device)
    _check("retina_seednet_train_step", lib.retina_seednet_train_step(
        _p(features), _p(labels), E, _p(params), _p(m), _p(v), int(step), lr, betas[0], betas[1], eps, _p(loss),
        _p(grad), _p(ws), ws.numel(), _stream(stream)))


def seednet_adam(params: torch.Tensor, m: torch.Tensor, v: torch.Tensor, grad: torch.Tensor, step: int,
                 lr: float = 1e-3, betas=(0.9, 0.999), eps: float = 1e-8, stream=None):
    for t, n in ((params, "params"), (m, "m"), (v, "v"), (grad, "grad")):
        _dev(t, torch.float32, n)
    _check("retina_seednet_adam", lib.retina_seednet_adam(_p(params), _p(m), _p(v), _p(grad), int(step), lr,
                                                          betas[0], betas[1], eps, _stream(stream)))


def topk_seeds(logits: torch.Tensor, K: int, lo: float = -0.5, hi: float = 0.5, hits=None, offsets=None,
               zmin: float = 50.0, min_sub_hits: int = 3, seeds: Optional[torch.Tensor] = None,
               want_idx: bool = False, stream=None):
    """float32 [E, K, 2] seeds from the ranked cells - cell centres, or with the
    events' hits the sub-cell hit means - and, if asked, int32 [E, K] cells."""
    _dev(logits, torch.float32, "logits")
    n_hits = 0
    if hits is not None:
        _dev(hits, torch.float32, "hits", 4)
        _dev(offsets, torch.int64, "offsets")
        n_hits = hits.shape[0]
    E = logits.numel() // 4096
    dev = logits.device
    seeds = seeds if seeds is not None else torch.empty((E, K, 2), dtype=torch.float32, device=dev)
    idx = torch.empty((E, K), dtype=torch.int32, device=dev) if want_idx else None
    _check("retina_topk_seeds", lib.retina_topk_seeds(_p(logits), E, K, lo, hi, zmin, int(min_sub_hits), _p(hits),
                                                      n_hits, _p(offsets), _p(seeds), _p(idx), _stream(stream)))
    return (seeds, idx) if want_idx else seeds


class Pipeline:
    """The whole path for a batch of events in one native call
    (retina_pipeline_*): hit ordering, then the grid method and Algorithm 1
    from the given starting points on two concurrent streams.  Owns its
    device workspace (allocated here, for the given capacities)."""

    def __init__(self, model: int, grid: Grid, sigma_grid: float, R0: float, opts: LsOpts, merge_cells: float,
                 max_events: int, max_hits: int, seeds_per_event: int, max_maxima: int = 4096,
                 max_tracks: int = 1024):
        c = _CPipelineConfig()
        c.model, c.grid, c.sigma_grid, c.R0, c.merge_cells = model, grid.c(), sigma_grid, R0, merge_cells
        c.opts = opts.c()
        c.max_events, c.max_hits, c.seeds_per_event = max_events, max_hits, seeds_per_event
        c.max_maxima, c.max_tracks = max_maxima, max_tracks
        self.S, self.K, self.max_events = int(seeds_per_event), int(max_tracks), int(max_events)
        h = ctypes.c_void_p()
        _check("retina_pipeline_create", lib.retina_pipeline_create(ctypes.byref(c), ctypes.byref(h)))
        self._h = h

    def run(self, hits: torch.Tensor, offsets: torch.Tensor, seeds: torch.Tensor, out=None, stream=None) -> dict:
        """seeds [n_events * S, 2]; returns {"grid": {...}, "search": {...}} with
        tracks [E, K, 2], track_R [E, K], n_tracks [E] per method."""
        if not self._h:
            raise RuntimeError("pipeline closed")
        _dev(hits, torch.float32, "hits", 4)
        _dev(offsets, torch.int64, "offsets")
        _dev(seeds, torch.float32, "seeds", 2)
        E = offsets.numel() - 1
        if seeds.numel() != 2 * E * self.S:
            raise ValueError("seeds must hold n_events * seeds_per_event points")
        dev = hits.device
        if out is None:
            out = {m: dict(tracks=torch.empty((E, self.K, 2), dtype=torch.float32, device=dev),
                           track_R=torch.empty((E, self.K), dtype=torch.float32, device=dev),
                           n_tracks=torch.empty((E,), dtype=torch.int32, device=dev)) for m in ("grid", "search")}
        g, s = out["grid"], out["search"]
        _check("retina_pipeline_run", lib.retina_pipeline_run(
            self._h, _p(hits), hits.shape[0], _p(offsets), E, _p(seeds), _p(g["tracks"]), _p(g["track_R"]),
            _p(g["n_tracks"]), _p(s["tracks"]), _p(s["track_R"]), _p(s["n_tracks"]), _stream(stream)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib.retina_pipeline_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceArray:
    """A view of library-owned device memory for torch.as_tensor (CUDA array interface)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2, "strides": None}


class Tracker:
    """Algorithm 1 over a batch of events in one native call
    (retina_tracker_*): hit ordering, the learned proposer's starting points
    (when ``params`` are given) or the caller's, their spatial order, the
    persistent batched search and cluster / select, replayed as one CUDA
    graph.  The tracker owns its input / output buffers (``hits``,
    ``offsets``, ``seeds``, ``tracks``, ``track_R``, ``n_tracks`` are torch
    views of them)."""

    def __init__(self, box: Grid, opts: LsOpts, R0: float, merge_cells: float, max_events: int, max_hits: int,
                 seeds_per_event: int, max_tracks: int = 1024, params=None, sort_seeds: bool = True,
                 seeds_per_warp: int = 0, warps: int = 0, smem_hits: int = 0, ctas: int = 0, use_graph: bool = True):
        c = _CTrackerConfig()
        c.box, c.opts, c.R0, c.merge_cells = box.c(), opts.c(), float(R0), float(merge_cells)
        c.max_events, c.max_hits, c.seeds_per_event, c.max_tracks = max_events, max_hits, seeds_per_event, max_tracks
        c.sort_seeds, c.seeds_per_warp, c.warps, c.smem_hits, c.ctas = int(sort_seeds), seeds_per_warp, warps, \
            smem_hits, ctas
        c.use_graph = int(use_graph)
        self.E, self.H, self.S, self.K = int(max_events), int(max_hits), int(seeds_per_event), int(max_tracks)
        self.learned = params is not None
        keep = None
        if params is not None:
            keep = torch.as_tensor(np.ascontiguousarray(params, dtype=np.float32)) if isinstance(params, np.ndarray) \
                else params.to(torch.float32).contiguous()
            if keep.numel() != 4833:
                raise ValueError("expected 4833 network parameters")
        h = ctypes.c_void_p()
        _check("retina_tracker_create", lib.retina_tracker_create(ctypes.byref(c), _p(keep), ctypes.byref(h)))
        self._h = h
        ptrs = [ctypes.c_void_p() for _ in range(6)]
        _check("retina_tracker_buffers", lib.retina_tracker_buffers(self._h, *[ctypes.byref(x) for x in ptrs]))
        dev = torch.device("cuda", torch.cuda.current_device())
        E, H, S, K = self.E, self.H, self.S, self.K
        view = lambda p, shape, t: torch.as_tensor(_DeviceArray(p.value, shape, t), device=dev)
        self.hits = view(ptrs[0], (H, 4), "<f4")
        self.offsets = view(ptrs[1], (E + 1,), "<i8")
        self.seeds = view(ptrs[2], (E, S, 2), "<f4")
        self.tracks = view(ptrs[3], (E, K, 2), "<f4")
        self.track_R = view(ptrs[4], (E, K), "<f4")
        self.n_tracks = view(ptrs[5], (E,), "<i4")

    def load(self, hits, offsets, seeds=None):
        """Copy a batch (host arrays or tensors) into the owned input buffers;
        returns the number of events."""
        hits = torch.as_tensor(np.ascontiguousarray(hits, dtype=np.float32)) if isinstance(hits, np.ndarray) else hits
        offsets = torch.as_tensor(np.ascontiguousarray(offsets, dtype=np.int64)) \
            if isinstance(offsets, np.ndarray) else offsets
        E = offsets.numel() - 1
        if hits.shape[0] > self.H or not 0 <= E <= self.E:
            raise ValueError("batch does not fit the tracker's capacity")
        self.hits[:hits.shape[0]].copy_(hits)
        self.offsets[:E + 1].copy_(offsets)
        if seeds is not None:
            seeds = torch.as_tensor(np.ascontiguousarray(seeds, dtype=np.float32)) \
                if isinstance(seeds, np.ndarray) else seeds
            self.seeds[:E].copy_(seeds.reshape(E, self.S, 2))
        return E

    def set_marks(self, events):
        """Stage marks recorded by every later step (6 torch.cuda.Event: before
        the hit ordering, after it, after the starting points, after their
        ordering, after the search, after cluster / select), or None."""
        if events is None:
            _check("retina_tracker_set_marks", lib.retina_tracker_set_marks(self._h, None, 0))
            self._marks = None
            return
        if len(events) != 6:
            raise ValueError("6 events")
        for e in events:  # the handles exist once recorded
            e.record()
        arr = (ctypes.c_void_p * 6)(*[e.cuda_event for e in events])
        _check("retina_tracker_set_marks", lib.retina_tracker_set_marks(self._h, arr, 6))
        self._marks = list(events)

    def step(self, n_events: int, stream=None):
        _check("retina_tracker_step", lib.retina_tracker_step(self._h, int(n_events), _stream(stream)))

    def run_host(self, hits: torch.Tensor, offsets: torch.Tensor, out: dict, seeds: Optional[torch.Tensor] = None,
                 stream=None):
        """One step from host tensors (page-locked for asynchronous copies):
        hits [n_hits, 4] float32, offsets [E + 1] int64, seeds [E, S, 2]
        (caller seeds only); out holds host tensors tracks [>= E, K, 2],
        track_R [>= E, K], n_tracks [>= E].  Enqueued on the stream: synchronise
        before reading ``out``."""
        for t, dt, name in ((hits, torch.float32, "hits"), (offsets, torch.int64, "offsets")):
            if t.is_cuda or t.dtype != dt or not t.is_contiguous():
                raise ValueError("%s must be a contiguous host %s tensor" % (name, dt))
        E = offsets.numel() - 1
        _check("retina_tracker_run_host", lib.retina_tracker_run_host(
            self._h, _p(hits), hits.shape[0], _p(offsets), E, _p(seeds), _p(out["tracks"]), _p(out["track_R"]),
            _p(out["n_tracks"]), _stream(stream)))

    def results(self, n_events: int):
        """Per event: float64 [n_tracks, 2] track parameters (host)."""
        n = self.n_tracks[:n_events].cpu().numpy()
        tr = self.tracks[:n_events].cpu().numpy()
        return [tr[e, :min(int(n[e]), self.K)].astype(np.float64) for e in range(n_events)]

    def close(self):
        if getattr(self, "_h", None):
            lib.retina_tracker_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
