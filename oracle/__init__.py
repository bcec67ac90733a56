"""FP64 CPU oracle of the modified Artificial Retina - TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA path never calls it and it
never calls the CUDA path; the two share no code.  The arithmetic lives in
``retina_oracle.c`` (plain C, double precision, libm ``exp``) plus, for the
learned-seed rows, ``seednet.py`` (numpy, double precision).  This module only
compiles that C file with gcc, loads it with ctypes and marshals numpy arrays.

Functions and the passages they follow (arXiv:1709.08610):

* :func:`rgh`, :func:`response` - Eq. 1 and its gradient / Hessian
  (Section 2, the remark on the small overhead of derivatives).
* :func:`grid_response` - Eq. 2, step 2 of the grid algorithm (Section 2).
* :func:`grid_maxima` - steps 3-4 of the grid algorithm: strict 8-neighbour
  local maxima at or above R0.
* :func:`local_search` - Algorithm 1 with the truncated Newton update and the
  annealed sigma schedule of Section 3.
* :func:`refine_maxima` - step 4 of the grid algorithm (estimate the track
  parameters of each selected cluster), read as Section 3's truncated-Newton
  updates at the grid's bandwidth started from each maximum's cell centre.
* :func:`extract_tracks` - the last two lines of Algorithm 1: cluster the
  converged points and keep the best of each cluster above R0.
* :func:`rgh4`, :func:`response4`, :func:`local_search4` - Eq. 1, its
  derivatives and Algorithm 1's truncated-Newton updates for a four-parameter
  straight track (x0, y0, t_x, t_y) that need not pass through the origin.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "retina_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libretina_oracle.so")
_LOCK = threading.Lock()
_LIB = None

TOY2D = 0
VELO_SLOPES = 1


class _Grid(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 2), ("step", ctypes.c_double * 2), ("n", ctypes.c_int64 * 2)]


class _LsOpts(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int32), ("sigma", ctypes.c_double * 8), ("c1", ctypes.c_double),
                ("max_halvings", ctypes.c_int32), ("step_cap_cells", ctypes.c_double), ("update", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, IEEE semantics, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            D = ctypes.c_double
            L.or_rgh.argtypes = [P, I64, ctypes.c_int, P, D, P]
            L.or_response.argtypes = [P, I64, ctypes.c_int, P, D]
            L.or_response.restype = D
            L.or_response_points.argtypes = [P, I64, ctypes.c_int, P, I64, D, P]
            L.or_grid_response.argtypes = [P, I64, ctypes.c_int, P, D, P]
            L.or_grid_maxima.argtypes = [P, I64, I64, D, P, I64, P]
            L.or_grid_maxima.restype = I64
            L.or_local_search.argtypes = [P, I64, ctypes.c_int, P, I64, P, P, P, P, P, P]
            L.or_extract_tracks.argtypes = [P, P, P, I64, P, D, D, P, I64]
            L.or_extract_tracks.restype = I64
            L.or_rgh4.argtypes = [P, I64, P, D, D, P]
            L.or_response4.argtypes = [P, I64, P, D, D]
            L.or_response4.restype = D
            L.or_local_search4.argtypes = [P, I64, P, I64, P, P, P, P, P]
            U64 = ctypes.c_uint64
            L.or_local_search_perturbed.argtypes = [P, I64, ctypes.c_int, P, I64, P, P, D, U64, I64, P, P, P, P]
            L.or_local_search4_perturbed.argtypes = [P, I64, P, I64, P, D, U64, I64, P, P, P, P]
            L.or_local_search_counted.argtypes = [P, I64, ctypes.c_int, P, I64, P, P, P, P, P, P]
            L.or_pair_seeds4.argtypes = [P, I64, P, ctypes.c_int32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                         ctypes.c_float, ctypes.c_float, P, I64]
            L.or_pair_seeds4.restype = I64
            L.or_extract_tracks4.argtypes = [P, P, P, I64, P, P, D, D, P, I64]
            L.or_extract_tracks4.restype = I64
            L.or_splitmix64.argtypes = [P]
            L.or_splitmix64.restype = U64
            L.or_perturb_u.argtypes = [U64, I64, ctypes.c_int, ctypes.c_int]
            L.or_perturb_u.restype = D
            _LIB = L
    return _LIB


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _hits(h) -> np.ndarray:
    h = np.ascontiguousarray(h, dtype=np.float32)
    if h.ndim != 2 or h.shape[1] != 4:
        raise ValueError("hits must be float32 [H, 4]")
    return h


def make_grid(lo: Sequence[float], step: Sequence[float], n: Sequence[int]) -> _Grid:
    g = _Grid()
    for a in range(2):
        g.lo[a] = float(lo[a])
        g.step[a] = float(step[a])
        g.n[a] = int(n[a])
    return g


def grid_of(wl) -> _Grid:
    return make_grid(wl.grid_lo, wl.grid_step, wl.grid_n)


def cell_centres(lo, step, n) -> Tuple[np.ndarray, np.ndarray]:
    """Cell centres lo + (i + 1/2) step per axis (exact binary for step = 2^-k)."""
    c0 = lo[0] + (np.arange(n[0], dtype=np.float64) + 0.5) * step[0]
    c1 = lo[1] + (np.arange(n[1], dtype=np.float64) + 0.5) * step[1]
    return c0, c1


def rgh(hits, model: int, theta, sigma: float) -> dict:
    """R, grad R, Hess R at one theta (Eq. 1 and its derivatives)."""
    h = _hits(hits)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(2)
    out = np.zeros(12)
    lib().or_rgh(_ptr(h), h.shape[0], model, _ptr(th), float(sigma), _ptr(out))
    return dict(R=out[0], grad=out[1:3].copy(), hess=np.array([[out[3], out[4]], [out[4], out[5]]]),
                grad_abs=out[7:9].copy(), hess_abs=np.array([[out[9], out[10]], [out[10], out[11]]]))


def response(hits, model: int, theta, sigma: float) -> np.ndarray:
    """R(theta_p) for points theta [P, 2] (Eq. 1)."""
    h = _hits(hits)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, 2)
    R = np.zeros(th.shape[0])
    lib().or_response_points(_ptr(h), h.shape[0], model, _ptr(th), th.shape[0], float(sigma), _ptr(R))
    return R


def grid_response(hits, model: int, lo, step, n, sigma: float) -> np.ndarray:
    """R[i1, i0] over the grid of units (Eq. 2)."""
    h = _hits(hits)
    g = make_grid(lo, step, n)
    R = np.zeros((int(n[1]), int(n[0])))
    lib().or_grid_response(_ptr(h), h.shape[0], model, ctypes.byref(g), float(sigma), _ptr(R))
    return R


def grid_maxima(R: np.ndarray, R0: float, cap: Optional[int] = None, with_margin: bool = False):
    """Linear indices of strict 3x3 local maxima with R >= R0 (ties -> lower index)."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    n1, n0 = R.shape
    cap = R.size if cap is None else cap
    idx = np.zeros(max(cap, 1), dtype=np.int64)
    margin = np.zeros(R.shape) if with_margin else None
    cnt = lib().or_grid_maxima(_ptr(R), n0, n1, float(R0), _ptr(idx), cap, _ptr(margin))
    out = idx[:min(cnt, cap)].copy()
    return (out, cnt, margin) if with_margin else out


UPDATE_TRUNCATED_NEWTON, UPDATE_STEEPEST_ASCENT, UPDATE_MODIFIED_NEWTON = 0, 1, 2


def local_search(hits, model: int, seeds, sigma_schedule: Sequence[float], lo, step, n,
                 c1: float = 1e-4, max_halvings: int = 8, step_cap_cells: float = 4.0, update: int = 0,
                 perturb: Optional[Tuple[float, int]] = None, count_trials: bool = False):
    """Algorithm 1's q updates for every seed.

    update picks the direction of each update: 0 the truncated Newton
    direction of Section 3 (the paper's choice), or one of the other methods
    Section 3 says were examined, read as 1 steepest ascent (p = grad R) and
    2 Newton with a modified Hessian (-Hess R shifted to be positive
    definite); the step cap and Armijo backtracking are common to all.

    perturb = (level, key) runs a perturbed replica: R, the gradient and the
    Hessian at each update and R at each trial are displaced by level * u
    times their parity tolerance, u in [-1, 1) drawn per (key, seed, update,
    quantity) (see :func:`path_conditioning`).

    Returns (theta [n, 2] float64, R_final [n], status [n] uint8, margin [n]);
    with count_trials, (theta, R_final, status, trials [n]): the responses
    each seed's line searches evaluated.
    """
    if update not in (0, 1, 2):
        raise ValueError("update must be 0, 1 or 2")
    h = _hits(hits)
    s = np.ascontiguousarray(seeds, dtype=np.float32).reshape(-1, 2)
    o = _LsOpts()
    o.q = len(sigma_schedule)
    if not 1 <= o.q <= 8:
        raise ValueError("1 <= q <= 8")
    for j, v in enumerate(sigma_schedule):
        o.sigma[j] = float(v)
    o.c1 = float(c1)
    o.max_halvings = int(max_halvings)
    o.step_cap_cells = float(step_cap_cells)
    o.update = int(update)
    g = make_grid(lo, step, n)
    ns = s.shape[0]
    th = np.zeros((ns, 2))
    R = np.zeros(ns)
    st = np.zeros(ns, dtype=np.uint8)
    m = np.zeros(ns)
    if count_trials:
        tr = np.zeros(ns, dtype=np.int32)
        lib().or_local_search_counted(_ptr(h), h.shape[0], model, _ptr(s), ns, ctypes.byref(o), ctypes.byref(g),
                                      _ptr(th), _ptr(R), _ptr(st), _ptr(tr))
        return th, R, st, tr
    if perturb is None:
        lib().or_local_search(_ptr(h), h.shape[0], model, _ptr(s), ns, ctypes.byref(o), ctypes.byref(g),
                              _ptr(th), _ptr(R), _ptr(st), _ptr(m))
    else:
        lib().or_local_search_perturbed(_ptr(h), h.shape[0], model, _ptr(s), ns, ctypes.byref(o), ctypes.byref(g),
                                        float(perturb[0]), int(perturb[1]) & (2 ** 64 - 1), 0,
                                        _ptr(th), _ptr(R), _ptr(st), _ptr(m))
    return th, R, st, m


# replica keys: a path near a decision boundary is crossed by about half of
# the replicas, so 16 leave a chance of 2^-16 of missing one
PERTURB_KEYS = tuple(0x5EED0001 + i for i in range(16))


def splitmix64(state: int, n: int):
    """The first n outputs of the oracle's SplitMix64 from ``state``."""
    st = ctypes.c_uint64(state & (2 ** 64 - 1))
    return [lib().or_splitmix64(ctypes.byref(st)) for _ in range(n)]


def perturb_u(key: int, seed_index: int, update: int, quantity: int) -> float:
    return lib().or_perturb_u(key & (2 ** 64 - 1), seed_index, update, quantity)


def path_conditioning(run, base, tol, keys: Sequence[int] = PERTURB_KEYS, level: float = 1.0):
    """Which search paths float32 arithmetic is expected to reproduce.

    ``run(perturb)`` runs the oracle search (perturb None or (level, key)) and
    returns (theta, R, status, margin); ``base`` is its unperturbed result.
    A path is well conditioned when every perturbed replica - every quantity
    the CUDA path sums in float32 displaced by up to ``level`` times its
    parity tolerance - ends with the same status and within ``tol`` (absolute,
    per parameter; an array broadcastable to theta's shape, e.g. the
    comparison tolerance of each seed) of the unperturbed end point.
    Returns (stable [n] bool, replica end points [reps, n, d], replica
    statuses [reps, n]).
    """
    th0, _, st0, _ = base
    tol = np.broadcast_to(np.asarray(tol, dtype=np.float64), th0.shape)
    stable = np.ones(len(st0), dtype=bool)
    ends, sts = [], []
    for k in keys:
        th, _, st, _ = run((level, k))
        ends.append(th)
        sts.append(st)
        stable &= (st == st0) & np.all(np.abs(th - th0) <= tol, axis=1)
    return stable, np.stack(ends), np.stack(sts)


class _Ls4Opts(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int32), ("sigma", ctypes.c_double * 8), ("c1", ctypes.c_double),
                ("max_halvings", ctypes.c_int32), ("scale", ctypes.c_double * 4), ("step_cap", ctypes.c_double),
                ("zref", ctypes.c_double)]


_TRI4 = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]


def _sym4(v) -> np.ndarray:
    H = np.zeros((4, 4))
    for i, (a, b) in enumerate(_TRI4):
        H[a, b] = H[b, a] = v[i]
    return H


def rgh4(hits, theta, sigma: float, zref: float = 0.0) -> dict:
    """R, grad R [4], Hess R [4, 4] of the four-parameter track (x0, y0, t_x,
    t_y) at the reference plane zref, crossing the layer z at
    (x0 + t_x (z - zref), y0 + t_y (z - zref)) (Eq. 1)."""
    h = _hits(hits)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(4)
    out = np.zeros(29)
    lib().or_rgh4(_ptr(h), h.shape[0], _ptr(th), float(zref), float(sigma), _ptr(out))
    return dict(R=out[0], grad=out[1:5].copy(), hess=_sym4(out[5:15]), grad_abs=out[15:19].copy(),
                hess_abs=_sym4(out[19:29]))


def response4(hits, theta, sigma: float, zref: float = 0.0) -> float:
    h = _hits(hits)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(4)
    return lib().or_response4(_ptr(h), h.shape[0], _ptr(th), float(zref), float(sigma))


def local_search4(hits, seeds, sigma_schedule: Sequence[float], scale: Sequence[float], step_cap: float = 4.0,
                  c1: float = 1e-4, max_halvings: int = 8, zref: float = 0.0,
                  perturb: Optional[Tuple[float, int]] = None):
    """Algorithm 1's q truncated-Newton updates (Newton-CG in four dimensions,
    at most four CG iterations) for four-parameter seeds [n, 4]; the step is
    capped to max_a |p_a| / scale_a <= step_cap.

    Returns (theta [n, 4] float64, R_final [n], status [n] uint8, margin [n]).
    """
    h = _hits(hits)
    s = np.ascontiguousarray(seeds, dtype=np.float32).reshape(-1, 4)
    o = _Ls4Opts()
    o.q = len(sigma_schedule)
    if not 1 <= o.q <= 8:
        raise ValueError("1 <= q <= 8")
    for j, v in enumerate(sigma_schedule):
        o.sigma[j] = float(v)
    o.c1 = float(c1)
    o.max_halvings = int(max_halvings)
    for a in range(4):
        o.scale[a] = float(scale[a])
    o.step_cap = float(step_cap)
    o.zref = float(zref)
    ns = s.shape[0]
    th = np.zeros((ns, 4))
    R = np.zeros(ns)
    st = np.zeros(ns, dtype=np.uint8)
    m = np.zeros(ns)
    if perturb is None:
        lib().or_local_search4(_ptr(h), h.shape[0], _ptr(s), ns, ctypes.byref(o), _ptr(th), _ptr(R), _ptr(st),
                               _ptr(m))
    else:
        lib().or_local_search4_perturbed(_ptr(h), h.shape[0], _ptr(s), ns, ctypes.byref(o), float(perturb[0]),
                                         int(perturb[1]) & (2 ** 64 - 1), 0, _ptr(th), _ptr(R), _ptr(st), _ptr(m))
    return th, R, st, m


def pair_seeds4(hits, layer_pairs, dz_tol: float, d_max: float, zc_range, zref: float,
                cap: Optional[int] = None):
    """Starting points of the four-parameter search from hit pairs on the
    given layer pairs [(z_a, z_b), ...] (see or_pair_seeds4): lines through
    two hits passing within d_max of the z axis at zc_range[0] <= z_c <=
    zc_range[1], as (x0, y0, t_x, t_y) at zref, in pair order; float32
    decisions.  Returns (seeds float32 [m, 4], number kept (>= m))."""
    h = _hits(hits)
    lz = np.ascontiguousarray(np.asarray(layer_pairs, dtype=np.float32).reshape(-1, 2))
    n = int(cap) if cap is not None else 1 << 20
    out = np.zeros((max(n, 1), 4), dtype=np.float32)
    cnt = lib().or_pair_seeds4(_ptr(h), h.shape[0], _ptr(lz), lz.shape[0], float(dz_tol), float(d_max),
                               float(zc_range[0]), float(zc_range[1]), float(zref), _ptr(out), n)
    return out[:min(cnt, n)].copy(), int(cnt)


def extract_tracks4(theta, R, status, lo, step, n, units, R0: float, merge_units: float = 2.0) -> np.ndarray:
    """Indices of the kept four-parameter points, in decreasing-R order
    (cluster + select with max_a |dtheta_a| / units_a < merge_units as the
    conflict; slopes inside the slope box lo / step / n)."""
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, 4)
    Rr = np.ascontiguousarray(R, dtype=np.float64).reshape(-1)
    st = None if status is None else np.ascontiguousarray(status, dtype=np.uint8).reshape(-1)
    u = np.ascontiguousarray(units, dtype=np.float64).reshape(4)
    g = make_grid(lo, step, n)
    keep = np.zeros(max(len(Rr), 1), dtype=np.int64)
    cnt = lib().or_extract_tracks4(_ptr(th), _ptr(Rr), _ptr(st), len(Rr), ctypes.byref(g), _ptr(u), float(R0),
                                   float(merge_units), _ptr(keep), len(keep))
    return keep[:cnt].copy()


def maxima_centres(idx, lo, step, n) -> np.ndarray:
    """Cell centres [m, 2] of grid maxima given as linear indices i1 * n0 + i0."""
    idx = np.asarray(idx, dtype=np.int64).reshape(-1)
    c0, c1 = cell_centres(lo, step, n)
    return np.stack([c0[idx % int(n[0])], c1[idx // int(n[0])]], 1)


def refine_maxima(hits, model: int, theta_c, sigma: float, lo, step, n, iters: int = 4,
                  step_cap_cells: float = 1.0, c1: float = 1e-4, max_halvings: int = 8):
    """Step 4 of the grid algorithm (Section 2): the track parameters of each
    selected cluster, estimated from its maximum's cell centre theta_c [m, 2]
    by ``iters`` truncated-Newton updates of Section 3 (Newton-CG direction,
    step capped to step_cap_cells, Armijo backtracking) at the grid's own
    bandwidth ``sigma``.  The updates are Algorithm 1's, so this is
    :func:`local_search` with the constant schedule (sigma,) * iters started
    from the centres; lo / step / n are the grid the maxima come from.

    Returns (theta [m, 2] float64, R [m] at sigma, status [m] uint8, margin [m]).
    """
    if not 1 <= iters <= 8:
        raise ValueError("1 <= iters <= 8")
    return local_search(hits, model, np.asarray(theta_c, dtype=np.float32).reshape(-1, 2), [float(sigma)] * iters,
                        lo, step, n, c1=c1, max_halvings=max_halvings, step_cap_cells=step_cap_cells)


def extract_tracks(theta, R, status, lo, step, n, R0: float, merge_cells: float = 2.0) -> np.ndarray:
    """Indices of the kept points, in decreasing-R order (cluster + select)."""
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, 2)
    Rv = np.ascontiguousarray(R, dtype=np.float64).reshape(-1)
    st = None if status is None else np.ascontiguousarray(status, dtype=np.uint8).reshape(-1)
    g = make_grid(lo, step, n)
    npt = th.shape[0]
    keep = np.zeros(max(npt, 1), dtype=np.int64)
    cnt = lib().or_extract_tracks(_ptr(th), _ptr(Rv), _ptr(st), npt, ctypes.byref(g), float(R0),
                                  float(merge_cells), _ptr(keep), npt)
    return keep[:cnt].copy()


# ---------------------------------------------------------------------------
# Track-finding evaluation (Section 3: a track is reconstructed when an
# estimate lies within epsilon of its true parameters).
# ---------------------------------------------------------------------------

def match_tracks(found: np.ndarray, truth: np.ndarray, tol: Sequence[float]) -> Tuple[int, int]:
    """Greedy one-to-one matching by ascending inf-norm distance (scaled by tol).

    Returns (matched, n_found).  truth: [T, 2] parameters of reconstructible
    tracks; found: [F, 2].
    """
    found = np.asarray(found, dtype=np.float64).reshape(-1, 2)
    truth = np.asarray(truth, dtype=np.float64).reshape(-1, 2)
    if found.size == 0 or truth.size == 0:
        return 0, found.shape[0]
    tol = np.asarray(tol, dtype=np.float64)
    d = np.max(np.abs(found[:, None, :] - truth[None, :, :]) / tol[None, None, :], axis=2)
    pairs = np.argwhere(d <= 1.0)
    order = np.argsort(d[pairs[:, 0], pairs[:, 1]], kind="stable")
    used_f = np.zeros(found.shape[0], bool)
    used_t = np.zeros(truth.shape[0], bool)
    m = 0
    for k in order:
        f, t = pairs[k]
        if not used_f[f] and not used_t[t]:
            used_f[f] = used_t[t] = True
            m += 1
    return m, found.shape[0]
