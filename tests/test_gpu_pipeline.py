"""The native executor (retina_pipeline_*) against the separate entry points.

A run enqueues the same launchers with the same launch options as the
separate calls, so both methods' track lists must agree bit for bit, on one
full-size event and on a ragged batch, and repeated runs must not change a bit.
"""
import numpy as np
import pytest
import torch

from synth import WORKLOADS, make_event, batch_of, uniform_seeds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    from paper_1709_08610_gb300 import build as rbuild
    rbuild.build()
    from paper_1709_08610_gb300 import retina
    return retina


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _separate(rt, wl, hits, offs, seeds, S, K, Km):
    E = offs.numel() - 1
    grid = rt.Grid.of(wl)
    opts = rt.LsOpts(sigma=tuple(wl.sigma_schedule))
    srt, boxes = rt.prepare_hits(hits, offs, wl.model)
    so = _dev(np.arange(E + 1, dtype=np.int64) * S)
    th, R, st = rt.batched_search(srt, offs, wl.model, seeds, so, opts, grid, boxes=boxes)
    search = rt.extract_tracks(th.view(E, S, 2), R.view(E, S), st.view(E, S), grid, wl.R0, wl.merge_cells, K)
    Rg = rt.grid_response(srt, offs, wl.model, grid, wl.sigma_grid, boxes=boxes)
    mx = rt.grid_maxima(Rg, grid, wl.R0, Km)
    gridt = rt.extract_tracks(mx["max_theta"], mx["max_R"], None, grid, wl.R0, wl.merge_cells, K, n_valid=mx["n_max"])
    return {"grid": gridt, "search": search}


@pytest.mark.parametrize("case", ["one_event", "ragged_batch"])
def test_pipeline_equals_the_separate_calls(rt, case):
    wl = WORKLOADS["velo"]
    if case == "one_event":
        evs, S = [make_event(wl, 3, 0, vertex_sigma=(0, 0, 0))], 8192
    else:
        evs = [make_event(wl, 3, e, n_tracks=nt, vertex_sigma=(0, 0, 0)) for e, nt in enumerate((150, 0, 40, 300, 90))]
        S = 512
    b = batch_of(evs)
    E = len(evs)
    hits, offs = _dev(b.hits), _dev(b.offsets)
    seeds = _dev(np.concatenate([uniform_seeds(wl, S, 3, e) for e in range(E)]).astype(np.float32))
    K, Km = 1024, 4096
    ref = _separate(rt, wl, hits, offs, seeds, S, K, Km)
    p = rt.Pipeline(wl.model, rt.Grid.of(wl), wl.sigma_grid, wl.R0, rt.LsOpts(sigma=tuple(wl.sigma_schedule)),
                    wl.merge_cells, max_events=E, max_hits=len(b.hits), seeds_per_event=S, max_maxima=Km,
                    max_tracks=K)
    try:
        for rep in range(2):
            got = p.run(hits, offs, seeds)
            torch.cuda.synchronize()
            for m in ("grid", "search"):
                n_ref = ref[m]["n_tracks"].cpu().numpy()
                np.testing.assert_array_equal(got[m]["n_tracks"].cpu().numpy(), n_ref)
                for e in range(E):
                    k = min(K, int(n_ref[e]))
                    for key in ("tracks", "track_R"):
                        np.testing.assert_array_equal(got[m][key].cpu().numpy()[e, :k],
                                                      ref[m][key].cpu().numpy()[e, :k])
        assert int(ref["grid"]["n_tracks"].sum()) > 0 and int(ref["search"]["n_tracks"].sum()) > 0
    finally:
        p.close()
