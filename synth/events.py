"""Seeded synthetic events of the shapes the paper's experiments use.

Every draw goes through numpy's PCG64 keyed by ``SeedSequence([run_seed,
event_id, stream])`` so that the oracle, the CUDA path, the tests and the
bench all see bit-identical float32 inputs.  Streams: 0 = the event itself,
1 = uniform multistart seeds.

Two track models, matching the two distance functions the paper uses:

* ``MODEL_TOY2D`` - straight lines ``y = alpha*x + beta`` crossing detector
  planes at ``x = const`` (Section 2, Figure 1 and Eq. 1); a hit is
  ``(x, y, 0, 0)``.
* ``MODEL_VELO_SLOPES`` - straight 3D tracks through the origin with slopes
  ``(t_x, t_y)`` crossing layers at ``z = const`` (Section 3, the simplified
  VELO model); a hit is ``(x, y, z, 0)``.

Workload recipes (sizes, smearing, noise, grids, bandwidths) are the ones the
design notes list for the five configurations; the noise placement, the plane
positions and the unit conventions follow the readings recorded there.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

MODEL_TOY2D = 0
MODEL_VELO_SLOPES = 1

STREAM_EVENT = 0
STREAM_SEEDS = 1

# 26 equally spaced layers covering z in [-300, 750] mm inclusive (42 mm pitch).
VELO_PLANES_Z = np.array([-300.0 + 42.0 * p for p in range(26)], dtype=np.float64)
# The paper's sVELO: 20 disk layers equally spaced within 700 mm (read as z = 35, 70, ..., 700 mm,
# none at the vertex), each an annulus 8 mm <= r <= 42 mm.
SVELO_PLANES_Z = np.array([35.0 * (p + 1) for p in range(20)], dtype=np.float64)
SVELO_R_INNER, SVELO_R_OUTER = 8.0, 42.0
TOY_PLANES_X = np.arange(1, 11, dtype=np.float64)


def _rng(run_seed: int, event_id: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(run_seed), int(event_id), int(stream)])))


@dataclass
class Event:
    """One event: float32 hits [H, 4], per-hit truth label, truth tracks."""

    model: int
    hits: np.ndarray  # float32 [H, 4]
    labels: np.ndarray  # int32 [H]: track index or -1 for noise
    truth: np.ndarray  # float64 [T, 6]: (theta0, theta1, vx, vy, vz, n_hits)

    @property
    def n_hits(self) -> int:
        return int(self.hits.shape[0])


@dataclass
class Batch:
    """Events concatenated in CSR form: hits [sum H, 4] and offsets [E + 1]."""

    model: int
    hits: np.ndarray  # float32 [sum H, 4]
    offsets: np.ndarray  # int64 [E + 1]
    events: List[Event]

    @property
    def n_events(self) -> int:
        return len(self.events)


@dataclass
class Workload:
    """A named workload: generator recipe plus the method's parameters."""

    name: str
    model: int
    grid_lo: Tuple[float, float]
    grid_step: Tuple[float, float]
    grid_n: Tuple[int, int]
    sigma_grid: float
    sigma_schedule: Tuple[float, ...]
    R0: float
    n_seeds: int
    n_events: int = 1
    merge_cells: float = 2.0
    match_tol: Tuple[float, float] = (1e-3, 1e-3)
    gen: Dict = field(default_factory=dict)

    @property
    def grid_hi(self) -> Tuple[float, float]:
        return tuple(self.grid_lo[a] + self.grid_n[a] * self.grid_step[a] for a in range(2))

    def cell_centre(self, i0: int, i1: int) -> Tuple[float, float]:
        return (self.grid_lo[0] + (i0 + 0.5) * self.grid_step[0], self.grid_lo[1] + (i1 + 0.5) * self.grid_step[1])


# --------------------------------------------------------------------------
# generators
# --------------------------------------------------------------------------

def make_toy2d_event(run_seed: int, event_id: int, n_tracks: int = 10, smear: float = 0.005,
                     noise_frac: float = 0.2, noise_halfwidth: float = 3.5,
                     planes_x: Sequence[float] = TOY_PLANES_X,
                     alpha_range: float = 0.3, beta_sigma: float = 0.1) -> Event:
    """2D straight-line toy: lines y = alpha x + beta seen by planes x = const.

    alpha ~ U(-0.3, 0.3), beta ~ N(0, 0.1), every plane hit, hit y smeared by
    N(0, smear); round(noise_frac * track hits) noise hits on uniformly chosen
    planes with y ~ U(-3.5, 3.5).
    """
    rng = _rng(run_seed, event_id, STREAM_EVENT)
    px = np.asarray(planes_x, dtype=np.float64)
    alpha = rng.uniform(-alpha_range, alpha_range, n_tracks)
    beta = rng.normal(0.0, beta_sigma, n_tracks)
    y = alpha[:, None] * px[None, :] + beta[:, None] + rng.normal(0.0, smear, (n_tracks, px.size))
    tx = np.broadcast_to(px[None, :], y.shape)
    n_sig = n_tracks * px.size
    n_noise = int(round(noise_frac * n_sig))
    nx = px[rng.integers(0, px.size, n_noise)]
    ny = rng.uniform(-noise_halfwidth, noise_halfwidth, n_noise)
    xs = np.concatenate([tx.reshape(-1), nx])
    ys = np.concatenate([y.reshape(-1), ny])
    labels = np.concatenate([np.repeat(np.arange(n_tracks), px.size), -np.ones(n_noise, dtype=np.int64)])
    perm = rng.permutation(xs.size)
    hits = np.zeros((xs.size, 4), dtype=np.float32)
    hits[:, 0] = xs[perm]
    hits[:, 1] = ys[perm]
    truth = np.zeros((n_tracks, 6))
    truth[:, 0] = alpha
    truth[:, 1] = beta
    truth[:, 5] = px.size
    return Event(MODEL_TOY2D, hits, labels[perm].astype(np.int32), truth)


def make_velo_event(run_seed: int, event_id: int, n_tracks=150, plane_eff: float = 0.9,
                    hit_sigma: float = 0.01, slope_sigma: float = 0.1,
                    vertex_sigma: Tuple[float, float, float] = (0.05, 0.05, 50.0),
                    noise_frac: float = 0.1,
                    planes_z: Sequence[float] = VELO_PLANES_Z) -> Event:
    """VELO-like event: straight tracks from a smeared origin through 26 layers.

    ``n_tracks`` is an int or a (mean, lo, hi) triple for a clipped Poisson
    draw.  Vertex v ~ N(0, vertex_sigma) per axis, slopes ~ N(0, 0.1), each
    layer hit with probability ``plane_eff``, hit x, y smeared by
    N(0, hit_sigma) mm.  Noise: round(noise_frac * track hits) hits on
    uniformly chosen layers, x, y ~ U(+-(0.5 |z| + 1)) mm.
    """
    rng = _rng(run_seed, event_id, STREAM_EVENT)
    pz = np.asarray(planes_z, dtype=np.float64)
    if isinstance(n_tracks, (tuple, list)):
        mean, lo, hi = n_tracks
        nt = int(np.clip(rng.poisson(mean), lo, hi))
    else:
        nt = int(n_tracks)
    v = rng.normal(0.0, 1.0, (nt, 3)) * np.asarray(vertex_sigma, dtype=np.float64)[None, :]
    t = rng.normal(0.0, slope_sigma, (nt, 2))
    hit_mask = rng.uniform(0.0, 1.0, (nt, pz.size)) < plane_eff
    smear = rng.normal(0.0, hit_sigma, (nt, pz.size, 2))
    dz = pz[None, :] - v[:, 2:3]
    x = v[:, 0:1] + t[:, 0:1] * dz + smear[:, :, 0]
    y = v[:, 1:2] + t[:, 1:2] * dz + smear[:, :, 1]
    z = np.broadcast_to(pz[None, :], x.shape)
    lab = np.broadcast_to(np.arange(nt)[:, None], x.shape)
    xs, ys, zs, ls = x[hit_mask], y[hit_mask], z[hit_mask], lab[hit_mask]
    n_noise = int(round(noise_frac * xs.size))
    nz = pz[rng.integers(0, pz.size, n_noise)]
    w = 0.5 * np.abs(nz) + 1.0
    nx = rng.uniform(-1.0, 1.0, n_noise) * w
    ny = rng.uniform(-1.0, 1.0, n_noise) * w
    xs = np.concatenate([xs, nx])
    ys = np.concatenate([ys, ny])
    zs = np.concatenate([zs, nz])
    labels = np.concatenate([ls, -np.ones(n_noise, dtype=np.int64)])
    perm = rng.permutation(xs.size)
    hits = np.zeros((xs.size, 4), dtype=np.float32)
    hits[:, 0] = xs[perm]
    hits[:, 1] = ys[perm]
    hits[:, 2] = zs[perm]
    truth = np.zeros((nt, 6))
    truth[:, 0:2] = t
    truth[:, 2:5] = v
    truth[:, 5] = hit_mask.sum(axis=1)
    return Event(MODEL_VELO_SLOPES, hits, labels[perm].astype(np.int32), truth)


def close_tracks_event(run_seed: int = 0, smear: float = 1e-2, n_planes: int = 20,
                       lines=((0.20, 0.00), (0.26, 0.00))) -> Event:
    """Two close 2D lines with 20 hits each and N(0, 1e-2) measurement noise.

    The workload of Figure 2 (merging and splitting of close tracks as sigma
    varies).  Planes at x = 0.1, 0.2, ..., 2.0; no noise hits.
    """
    rng = _rng(run_seed, 0, STREAM_EVENT)
    px = 0.1 * np.arange(1, n_planes + 1, dtype=np.float64)
    xs, ys, ls = [], [], []
    for ti, (a, b) in enumerate(lines):
        xs.append(px)
        ys.append(a * px + b + rng.normal(0.0, smear, px.size))
        ls.append(np.full(px.size, ti))
    hits = np.zeros((n_planes * len(lines), 4), dtype=np.float32)
    hits[:, 0] = np.concatenate(xs)
    hits[:, 1] = np.concatenate(ys)
    truth = np.zeros((len(lines), 6))
    truth[:, 0:2] = np.asarray(lines)
    truth[:, 5] = n_planes
    return Event(MODEL_TOY2D, hits, np.concatenate(ls).astype(np.int32), truth)


def slopes_to_angles(u, v) -> np.ndarray:
    """The paper's two angles (x = t sin(theta), y = t cos(theta) sin(phi),
    z = t cos(theta) cos(phi)) of the lines through the origin with slopes
    (u, v) = (x / z, y / z), z > 0; returns [..., 2] = (theta, phi)."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    n = np.sqrt(1.0 + u * u + v * v)
    return np.stack([np.arcsin(u / n), np.arctan2(v, np.ones_like(v))], -1)


def make_svelo_event(run_seed: int, event_id: int, n_tracks: int = 200, p_hit: float = 0.5,
                     hit_sigma: float = 0.01, eta_range: Tuple[float, float] = (1.0, 6.0),
                     noise_mean: float = 250.0, n_min: int = 2,
                     planes_z: Sequence[float] = SVELO_PLANES_Z) -> Event:
    """The paper's sVELO event (Section 4): straight tracks from the origin
    with pseudo-rapidity eta ~ U[1, 6] and azimuth phi ~ U[0, 2 pi); each
    disk layer (8 <= r <= 42 mm) a track crosses records a hit with
    probability p_hit, x and y measured with N(0, hit_sigma) errors; a track
    with fewer than n_min hits is undetectable and its hits count as noise;
    Poisson(noise_mean) noise hits, each on a uniformly chosen layer and
    uniform over the annulus.  Tracks are drawn until ``n_tracks`` of them are
    reconstructible (>= n_min hits); only those are truth tracks, as slopes
    (u, v) = (x / z, y / z) in columns 0-1 (use slopes_to_angles for the
    paper's angles) and their hit count in column 5."""
    rng = _rng(run_seed, event_id, STREAM_EVENT)
    pz = np.asarray(planes_z, dtype=np.float64)
    r2_in, r2_out = SVELO_R_INNER ** 2, SVELO_R_OUTER ** 2
    xs, ys, zs, ls, truth = [], [], [], [], []
    n_rec = 0
    for _ in range(100 * max(int(n_tracks), 1) + 1000):
        if n_rec >= n_tracks:
            break
        eta = rng.uniform(eta_range[0], eta_range[1])
        phi = rng.uniform(0.0, 2.0 * math.pi)
        tan_p = math.tan(2.0 * math.atan(math.exp(-eta)))
        u, v = tan_p * math.cos(phi), tan_p * math.sin(phi)
        r = tan_p * pz
        inside = (r * r >= r2_in) & (r * r <= r2_out)
        fired = inside & (rng.uniform(0.0, 1.0, pz.size) < p_hit)
        err = rng.normal(0.0, hit_sigma, (pz.size, 2))
        k = np.flatnonzero(fired)
        rec = k.size >= n_min
        xs.append(u * pz[k] + err[k, 0])
        ys.append(v * pz[k] + err[k, 1])
        zs.append(pz[k])
        ls.append(np.full(k.size, n_rec if rec else -1, dtype=np.int64))
        if rec:
            truth.append((u, v, 0.0, 0.0, 0.0, float(k.size)))
            n_rec += 1
    n_noise = int(rng.poisson(noise_mean))
    nz = pz[rng.integers(0, pz.size, n_noise)]
    nr = np.sqrt(rng.uniform(r2_in, r2_out, n_noise))
    na = rng.uniform(0.0, 2.0 * math.pi, n_noise)
    xs.append(nr * np.cos(na))
    ys.append(nr * np.sin(na))
    zs.append(nz)
    ls.append(-np.ones(n_noise, dtype=np.int64))
    xs, ys, zs, labels = (np.concatenate(a) for a in (xs, ys, zs, ls))
    perm = rng.permutation(xs.size)
    hits = np.zeros((xs.size, 4), dtype=np.float32)
    hits[:, 0] = xs[perm]
    hits[:, 1] = ys[perm]
    hits[:, 2] = zs[perm]
    tr = np.array(truth, dtype=np.float64).reshape(-1, 6)
    return Event(MODEL_VELO_SLOPES, hits, labels[perm].astype(np.int32), tr)


def make_event(wl: Workload, run_seed: int, event_id: int, **over) -> Event:
    kw = dict(wl.gen)
    kw.update(over)
    if kw.pop("generator", None) == "svelo":
        return make_svelo_event(run_seed, event_id, **kw)
    if wl.model == MODEL_TOY2D:
        return make_toy2d_event(run_seed, event_id, **kw)
    return make_velo_event(run_seed, event_id, **kw)


def make_batch(wl: Workload, run_seed: int, event_ids: Sequence[int], **over) -> Batch:
    evs = [make_event(wl, run_seed, e, **over) for e in event_ids]
    return batch_of(evs)


def batch_of(evs: Sequence[Event]) -> Batch:
    counts = np.array([e.n_hits for e in evs], dtype=np.int64)
    offsets = np.zeros(len(evs) + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    hits = np.concatenate([e.hits for e in evs]) if evs else np.zeros((0, 4), np.float32)
    return Batch(evs[0].model if evs else MODEL_VELO_SLOPES, np.ascontiguousarray(hits, dtype=np.float32),
                 offsets, list(evs))


def seednet_init_params(seed: int = 0) -> np.ndarray:
    """Initial float32 parameter vector (4833 values) of the seed-proposal
    network: He-style normal weights (PCG64 keyed by ``seed``), zero biases
    except the head's, set to the prior log-odds -3.  Layout: W1 [16,1,3,3],
    b1 [16], W2 [32,16,3,3], b2 [32], W3 [32], b3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.normal(0, math.sqrt(2.0 / 9), 16 * 9)
    W2 = rng.normal(0, math.sqrt(2.0 / (9 * 16)), 32 * 16 * 9)
    W3 = rng.normal(0, math.sqrt(1.0 / 32), 32)
    return np.concatenate([W1, np.zeros(16), W2, np.zeros(32), W3, [-3.0]]).astype(np.float32)


def uniform_seeds(wl: Workload, n: int, run_seed: int, event_id: int) -> np.ndarray:
    """Uniform multistart seeds over the grid box (the prior of Algorithm 1)."""
    rng = _rng(run_seed, event_id, STREAM_SEEDS)
    u = rng.uniform(0.0, 1.0, (n, 2))
    lo = np.asarray(wl.grid_lo, dtype=np.float64)
    ext = np.asarray(wl.grid_n, dtype=np.float64) * np.asarray(wl.grid_step, dtype=np.float64)
    return (lo[None, :] + u * ext[None, :]).astype(np.float32)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def _z_rms() -> float:
    return float(math.sqrt(np.mean(VELO_PLANES_Z ** 2)))


def _x_rms() -> float:
    return float(math.sqrt(np.mean(TOY_PLANES_X ** 2)))


_TOY_STEP = 2.0 ** -8
_TOY_SIGMA = max(_TOY_STEP * _x_rms(), _TOY_STEP)
_VELO_SCHEDULE = (0.3, 0.175, 0.05)

WORKLOADS: Dict[str, Workload] = {
    # 2D toy: 10 lines, 200 x 200 (alpha, beta) grid, 256-seed search.
    "toy2d": Workload(
        name="toy2d", model=MODEL_TOY2D,
        grid_lo=(-100 * _TOY_STEP, -100 * _TOY_STEP), grid_step=(_TOY_STEP, _TOY_STEP), grid_n=(200, 200),
        sigma_grid=_TOY_SIGMA,
        sigma_schedule=tuple(max(_TOY_SIGMA * s / _VELO_SCHEDULE[0], 2 * 0.005) for s in _VELO_SCHEDULE),
        R0=5.0, n_seeds=256, match_tol=(_TOY_STEP, _TOY_STEP),
        gen=dict(n_tracks=10)),
    # VELO-like single event: 150 tracks, 1024^2 slope grid vs 8192 seeds.
    "velo": Workload(
        name="velo", model=MODEL_VELO_SLOPES,
        grid_lo=(-0.5, -0.5), grid_step=(2.0 ** -10, 2.0 ** -10), grid_n=(1024, 1024),
        sigma_grid=2.0 ** -10 * _z_rms(), sigma_schedule=_VELO_SCHEDULE,
        R0=0.5 * 26 * 0.9, n_seeds=8192,
        gen=dict(n_tracks=150)),
    # 1024 ragged VELO-like events, 4096 seeds each.
    "velo_batch": Workload(
        name="velo_batch", model=MODEL_VELO_SLOPES,
        grid_lo=(-0.5, -0.5), grid_step=(2.0 ** -10, 2.0 ** -10), grid_n=(1024, 1024),
        sigma_grid=2.0 ** -10 * _z_rms(), sigma_schedule=_VELO_SCHEDULE,
        R0=0.5 * 26 * 0.9, n_seeds=4096, n_events=1024,
        gen=dict(n_tracks=(150, 20, 400))),
    # The paper's sVELO (20 disks, eta ~ U[1, 6], p_hit 0.5, Poisson(250) noise), slopes up to
    # tan(2 atan(e^-1)) = 0.85; 2048^2 grid over [-1, 1]^2; R0 keeps lines through >= 2 hits.
    "svelo": Workload(
        name="svelo", model=MODEL_VELO_SLOPES,
        grid_lo=(-1.0, -1.0), grid_step=(2.0 ** -10, 2.0 ** -10), grid_n=(2048, 2048),
        sigma_grid=2.0 ** -10 * float(math.sqrt(np.mean(SVELO_PLANES_Z ** 2))), sigma_schedule=_VELO_SCHEDULE,
        R0=1.5, n_seeds=4096, n_events=1024,
        gen=dict(generator="svelo", n_tracks=200)),
    # High multiplicity: ~600 tracks/event, 15 % noise, 2048^2 grid.
    "velo_stress": Workload(
        name="velo_stress", model=MODEL_VELO_SLOPES,
        grid_lo=(-0.5, -0.5), grid_step=(2.0 ** -11, 2.0 ** -11), grid_n=(2048, 2048),
        sigma_grid=2.0 ** -11 * _z_rms(), sigma_schedule=_VELO_SCHEDULE,
        R0=0.5 * 26 * 0.9, n_seeds=4096, n_events=1024,
        gen=dict(n_tracks=(600, 200, 1200), noise_frac=0.15 / 0.85)),
}
