"""The native batch executor (retina_tracker_*) against the separate entry
points it enqueues: the learned-seed path and the caller-seed path give the
same tracks bit for bit as BatchTracker (the same launches made one by one
from Python), graph replays equal eager steps, and a step from host buffers
(copies in, step, copies out) equals a step on device-resident inputs."""
import numpy as np
import pytest
import torch

from synth import WORKLOADS, batch_of, make_event, uniform_seeds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    from paper_1709_08610_gb300 import build as rbuild
    rbuild.build()
    from paper_1709_08610_gb300 import retina
    return retina


def _batch(wl, E, seed):
    evs = [make_event(wl, seed, e, vertex_sigma=(0, 0, 0)) for e in range(E)]
    return evs, batch_of(evs)


def _same(a_tracks, a_R, a_n, b_tracks, b_R, b_n, K):
    a_n, b_n = np.asarray(a_n), np.asarray(b_n)
    assert np.array_equal(a_n, b_n)
    for e, n in enumerate(a_n):
        k = min(int(n), K)
        assert np.array_equal(np.asarray(a_tracks[e, :k]), np.asarray(b_tracks[e, :k]))
        assert np.array_equal(np.asarray(a_R[e, :k]), np.asarray(b_R[e, :k]))


@pytest.mark.parametrize("learned", [True, False])
def test_tracker_equals_the_separate_launches(rt, learned):
    from paper_1709_08610_gb300.pipeline import BatchTracker
    from paper_1709_08610_gb300.seednet import DEFAULT_WEIGHTS, SeedProposer, read_checkpoint
    wl = WORKLOADS["velo_batch"]
    E, S, K = 24, 512, 512
    evs, b = _batch(wl, E, 77)
    box = rt.Grid.of(wl)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    params = read_checkpoint(DEFAULT_WEIGHTS)[1]["params"] if learned else None
    seeds = None if learned else np.stack([uniform_seeds(wl, S, 77, e) for e in range(E)])
    shape = dict(seeds_per_warp=2, warps=32, smem_hits=12288)
    ref = BatchTracker(E, b.hits.shape[0], S, box, opts, wl.R0, max_tracks=K, sort_seeds=True,
                       proposer=SeedProposer(params) if learned else None, **shape)
    ref.load(b.hits, b.offsets, seeds)
    ref.step()
    outs = []
    for use_graph in (True, False):
        tr = rt.Tracker(box, opts, wl.R0, 2.0, E, b.hits.shape[0], S, max_tracks=K, params=params,
                        use_graph=use_graph, **shape)
        n = tr.load(b.hits, b.offsets, seeds)
        for _ in range(2):  # the second step replays the recorded graph
            tr.step(n)
        torch.cuda.synchronize()
        _same(ref.tracks["tracks"].cpu(), ref.tracks["track_R"].cpu(), ref.tracks["n_tracks"].cpu(),
              tr.tracks.cpu(), tr.track_R.cpu(), tr.n_tracks.cpu(), K)
        outs.append(tr)
    assert int(ref.tracks["n_tracks"].sum()) > 20 * E if learned else True
    # a different batch size records another graph
    tr = outs[0]
    n = tr.load(b.hits[:b.offsets[E // 2]], b.offsets[:E // 2 + 1],
                None if seeds is None else seeds[:E // 2])
    tr.step(n)
    ref2 = BatchTracker(E // 2, b.hits.shape[0], S, box, opts, wl.R0, max_tracks=K, sort_seeds=True,
                        proposer=SeedProposer(params) if learned else None, **shape)
    ref2.load(b.hits[:b.offsets[E // 2]], b.offsets[:E // 2 + 1], None if seeds is None else seeds[:E // 2])
    ref2.step()
    torch.cuda.synchronize()
    _same(ref2.tracks["tracks"].cpu(), ref2.tracks["track_R"].cpu(), ref2.tracks["n_tracks"].cpu(),
          tr.tracks[:E // 2].cpu(), tr.track_R[:E // 2].cpu(), tr.n_tracks[:E // 2].cpu(), K)
    for t in outs:
        t.close()


def test_tracker_from_host_buffers_equals_device_step(rt):
    from paper_1709_08610_gb300.seednet import DEFAULT_WEIGHTS, read_checkpoint
    wl = WORKLOADS["velo_stress"]
    E, S, K = 6, 2048, 2048
    evs, b = _batch(wl, E, 78)
    box = rt.Grid.of(wl)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    params = read_checkpoint(DEFAULT_WEIGHTS)[1]["params"]
    tr = rt.Tracker(box, opts, wl.R0, 2.0, E, b.hits.shape[0], S, max_tracks=K, params=params)
    n = tr.load(b.hits, b.offsets)
    tr.step(n)
    torch.cuda.synchronize()
    ref = (tr.tracks.cpu().clone(), tr.track_R.cpu().clone(), tr.n_tracks.cpu().clone())
    # scribble over the device inputs and outputs, then run from host memory twice
    tr.hits.fill_(7.0)
    tr.offsets.zero_()
    tr.n_tracks.fill_(-1)
    hits_h = torch.from_numpy(b.hits).pin_memory()
    offs_h = torch.from_numpy(b.offsets).pin_memory()
    out = dict(tracks=torch.full((E, K, 2), -5.0).pin_memory(), track_R=torch.full((E, K), -5.0).pin_memory(),
               n_tracks=torch.full((E,), -5, dtype=torch.int32).pin_memory())
    s = torch.cuda.Stream()
    for _ in range(2):
        tr.run_host(hits_h, offs_h, out, stream=s)
        s.synchronize()
        _same(ref[0], ref[1], ref[2], out["tracks"], out["track_R"], out["n_tracks"], K)
    assert int(ref[2].min()) > 200  # high-multiplicity events: hundreds of tracks each
    # malformed offsets are refused before anything is enqueued
    bad = offs_h.clone()
    bad[2] = bad[1] - 1
    with pytest.raises(rt.RetinaError):
        tr.run_host(hits_h, bad, out, stream=s)
    tr.close()


def test_back_to_back_host_runs_overlap_safely(rt):
    # consecutive run_host calls without a synchronisation in between: each
    # step's hit copy overlaps the previous step's search (it waits only for
    # that step's hit ordering), and every step still returns exactly its own
    # batch's tracks
    from paper_1709_08610_gb300.seednet import DEFAULT_WEIGHTS, read_checkpoint
    wl = WORKLOADS["velo_stress"]
    E, S, K = 6, 2048, 2048
    batches = [_batch(wl, E, 79)[1], _batch(wl, E, 80)[1]]
    H = max(bb.hits.shape[0] for bb in batches)
    box = rt.Grid.of(wl)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    params = read_checkpoint(DEFAULT_WEIGHTS)[1]["params"]
    tr = rt.Tracker(box, opts, wl.R0, 2.0, E, H, S, max_tracks=K, params=params)
    refs = []
    for bb in batches:
        tr.step(tr.load(bb.hits, bb.offsets))
        torch.cuda.synchronize()
        refs.append((tr.tracks.cpu().clone(), tr.track_R.cpu().clone(), tr.n_tracks.cpu().clone()))
    ins = [(torch.from_numpy(bb.hits).pin_memory(), torch.from_numpy(bb.offsets).pin_memory()) for bb in batches]
    outs = [dict(tracks=torch.full((E, K, 2), -5.0).pin_memory(), track_R=torch.full((E, K), -5.0).pin_memory(),
                 n_tracks=torch.full((E,), -5, dtype=torch.int32).pin_memory()) for _ in range(4)]
    s = torch.cuda.Stream()
    for i in range(4):
        tr.run_host(ins[i % 2][0], ins[i % 2][1], outs[i], stream=s)
    s.synchronize()
    for i in range(4):
        r = refs[i % 2]
        _same(r[0], r[1], r[2], outs[i]["tracks"], outs[i]["track_R"], outs[i]["n_tracks"], K)
    tr.close()
