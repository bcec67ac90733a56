"""What the trained seed network gains over the method without it (GPU).

On held-out VELO-like events (ragged track counts, origin vertex, a run seed
the training never saw) the batched search is run from the committed
network's top-512 hit-centroid seeds and from uniform seeds (the prior of
Algorithm 1).  The plain method - 4096 uniform seeds per event - judges the
learned one's missed-track rate: the learned seeds must recover almost every
track it finds while using 8x fewer starting points, and must beat uniform
seeding at the same seed count by a wide margin.  The whole learned step is
also replayed as one CUDA graph and must give the eager result bitwise.
"""
import numpy as np
import pytest
import torch

from synth import WORKLOADS, batch_of, make_event, uniform_seeds

pytestmark = pytest.mark.gpu

RUN_SEED = 3000
N_EVENTS = 128


@pytest.fixture(scope="module")
def env():
    from paper_1709_08610_gb300 import build as rbuild
    rbuild.build()
    from paper_1709_08610_gb300 import retina as rt
    from paper_1709_08610_gb300.pipeline import BatchTracker, match_efficiency, recovered_fraction
    from paper_1709_08610_gb300.seednet import DEFAULT_WEIGHTS, SeedProposer
    wl = WORKLOADS["velo_batch"]
    evs = [make_event(wl, RUN_SEED, e, vertex_sigma=(0, 0, 0)) for e in range(N_EVENTS)]
    b = batch_of(evs)
    box = rt.Grid.of(wl)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))

    def run(n, learned):
        prop = SeedProposer.from_checkpoint(DEFAULT_WEIGHTS) if learned else None
        tr = BatchTracker(N_EVENTS, b.hits.shape[0], n, box, opts, wl.R0, proposer=prop)
        S = None if learned else np.stack([uniform_seeds(wl, n, RUN_SEED, e) for e in range(N_EVENTS)])
        tr.load(b.hits, b.offsets, S)
        tr.step()
        return tr

    truth = [ev.truth[:, :2] for ev in evs]
    return dict(rt=rt, run=run, truth=truth, eff=match_efficiency, rec=recovered_fraction)


def test_learned_512_seeds_match_4096_uniform_seeds(env):
    plain = env["run"](4096, False).results()
    learned = env["run"](512, True).results()
    uni512 = env["run"](512, False).results()
    e_plain, _ = env["eff"](plain, env["truth"])
    e_learn, fake_learn = env["eff"](learned, env["truth"])
    e_u512, _ = env["eff"](uni512, env["truth"])
    rec = env["rec"](learned, plain)
    print("efficiency: uniform-4096 %.3f  learned-512 %.3f  uniform-512 %.3f  recovered %.3f  fakes/event %.2f"
          % (e_plain, e_learn, e_u512, rec, fake_learn / N_EVENTS))
    assert rec >= 0.95                 # the plain method's tracks, found from 8x fewer seeds
    assert e_learn >= 0.95 * e_plain   # at least equal efficiency
    assert e_learn >= e_u512 + 0.3     # and far above uniform seeding at the same count


def test_learned_step_replays_as_one_cuda_graph(env):
    tr = env["run"](512, True)
    eager = {k: v.clone() for k, v in tr.tracks.items()}
    seeds = tr.seeds.clone()
    tr.capture()
    for k in tr.tracks:
        tr.tracks[k].zero_()
    tr.seeds.zero_()
    tr.replay()
    torch.cuda.synchronize()
    assert torch.equal(tr.seeds, seeds)
    assert torch.equal(tr.tracks["n_tracks"], eager["n_tracks"])
    n = eager["n_tracks"].clamp(max=tr.K).cpu().numpy()
    for e in range(N_EVENTS):  # entries past n_tracks are not written
        for k in ("tracks", "track_R", "track_src"):
            assert torch.equal(tr.tracks[k][e, :n[e]], eager[k][e, :n[e]]), (e, k)
