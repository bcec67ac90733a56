"""The tie-aware track-set comparison of the GPU tests, checked on the CPU:
the oracle against one of its own perturbed replicas (a stand-in for a
float32 run of the same search) must pass, and planted differences - a
dropped track, a displaced track, an extra track - must fail."""
import numpy as np
import pytest

import oracle
from parity_rules import R_ABS, R_REL, candidates, compare_track_sets, search_tolerance
from synth import WORKLOADS, make_event, uniform_seeds


def _converged(ev, wl):
    step = np.asarray(wl.grid_step)

    def at(th):
        o = oracle.rgh(ev.hits, wl.model, th, wl.sigma_schedule[-1])
        H, g = o["hess"], o["grad"]
        if not np.all(np.linalg.eigvalsh(H) < 0):
            return None
        if np.max(np.abs(np.linalg.solve(H, g)) / step) > 0.05:
            return None
        return g, H, o["grad_abs"]
    return at


@pytest.fixture(scope="module")
def case():
    wl = WORKLOADS["velo"]
    ev = make_event(wl, 0, 1, vertex_sigma=(0, 0, 0))
    seeds = uniform_seeds(wl, 2048, 0, 1)
    box = (wl.grid_lo, wl.grid_step, wl.grid_n)
    sig = tuple(wl.sigma_schedule)

    def run(pt):
        return oracle.local_search(ev.hits, 1, seeds, sig, *box, perturb=pt)

    base = run(None)
    other = run((0.5, 0xABCDEF))  # the stand-in for the other side
    R0 = wl.R0
    th_o, R_o, st_o, m_o = base
    th_g, R_g, st_g, _ = other
    cand_o = candidates(th_o, R_o, st_o, *box, R0)
    cand_g = candidates(th_g, R_g, st_g, *box, R0)
    tol = search_tolerance(_converged(ev, wl), th_o, cand_o | cand_g, wl.grid_step)
    stable, _, _ = oracle.path_conditioning(run, base, tol)
    tie = (m_o < 1.0) | ~stable
    keep_o = oracle.extract_tracks(th_o, R_o, st_o, *box, R0, wl.merge_cells)
    keep_g = oracle.extract_tracks(th_g, R_g, st_g, *box, R0, wl.merge_cells)
    return dict(wl=wl, th_o=th_o, R_o=R_o, cand_o=cand_o, th_g=th_g, R_g=R_g, cand_g=cand_g, tie=tie,
                keep_o=keep_o, keep_g=keep_g, tol=tol)


def _cmp(c, **over):
    d = dict(c)
    d.update(over)
    wl = d["wl"]
    return compare_track_sets(d["th_o"], d["R_o"], d["cand_o"], d["th_g"], d["R_g"], d["cand_g"], d["tie"],
                              d["keep_o"], d["keep_g"], d["tol"], wl.grid_step, wl.merge_cells, R0=wl.R0)


def test_oracle_against_its_own_replica_passes(case):
    comps, tied, compared = _cmp(case)
    assert compared >= 10 and tied < comps, (comps, tied, compared)


def test_a_dropped_track_fails(case):
    _, _, compared = _cmp(case)
    # drop the best-ranked kept track whose component is untied from the other side
    for k in range(len(case["keep_g"])):
        kg = np.delete(case["keep_g"], k)
        try:
            _cmp(case, keep_g=kg)
        except AssertionError:
            return
    pytest.fail("no dropped track was detected")


def test_a_displaced_track_fails(case):
    th = case["th_g"].copy()
    for i in case["keep_g"]:
        th2 = th.copy()
        th2[i] = th2[i] + 0.01 * np.asarray(case["wl"].grid_step)  # 10x the converged tolerance
        try:
            _cmp(case, th_g=th2)
        except AssertionError:
            return
    pytest.fail("no displaced track was detected")


def test_an_extra_track_fails(case):
    # a far-away extra candidate kept by the other side only
    th = case["th_g"].copy()
    cand = case["cand_g"].copy()
    R = case["R_g"].copy()
    i = int(np.flatnonzero(~case["cand_o"] & ~case["cand_g"] & ~case["tie"])[0])
    th[i] = [0.45, 0.45]
    R[i] = 50.0
    cand[i] = True
    with pytest.raises(AssertionError):
        _cmp(case, th_g=th, R_g=R, cand_g=cand, keep_g=np.append(case["keep_g"], i))
