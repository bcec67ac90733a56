"""Four-parameter search (x0, y0, t_x, t_y) on the GPU vs the FP64 oracle,
through the C ABI, on a VELO-like event with the smeared vertex that the
two-parameter slope model cannot fit."""
import numpy as np
import pytest
import torch

import oracle
from parity_rules import check_conditioned
from synth import WORKLOADS, make_event

pytestmark = pytest.mark.gpu

R_REL, R_ABS = 1e-5, 1e-6
GH_REL = 1e-4
TH_UNITS = 1e-3
SCALE = (0.25, 0.25, 2.0 ** -10, 2.0 ** -10)
SIGMA = (0.3, 0.175, 0.05, 0.05, 0.05)
ZREF = 225.0  # the mean z of the 26 layers
CONV_MIN = 80  # the oracle ends 103 robust, well-conditioned seeds of 400 at converged maxima


@pytest.fixture(scope="module")
def rt():
    from paper_1709_08610_gb300 import build as rbuild
    rbuild.build()
    from paper_1709_08610_gb300 import retina
    return retina


def _event_and_seeds():
    ev = make_event(WORKLOADS["velo"], 31, 0)  # vertex smeared by (0.05, 0.05, 50) mm
    t, v = ev.truth[:, :2], ev.truth[:, 2:5]
    truth4 = np.stack([v[:, 0] + t[:, 0] * (ZREF - v[:, 2]), v[:, 1] + t[:, 1] * (ZREF - v[:, 2]), t[:, 0], t[:, 1]],
                      1)
    rng = np.random.default_rng(11)
    pick = rng.integers(0, len(truth4), 400)
    seeds = truth4[pick] + rng.normal(0, 1, (400, 4)) * np.array([0.2, 0.2, 5e-4, 5e-4])
    return ev, truth4, seeds.astype(np.float32)


def _converged_at(ev):
    def at(th):
        o = oracle.rgh4(ev.hits, th, SIGMA[-1], zref=ZREF)
        H, g = o["hess"], o["grad"]
        if not np.all(np.linalg.eigvalsh(H) < 0):
            return None
        try:
            if np.max(np.abs(np.linalg.solve(H, g)) / np.asarray(SCALE)) > 0.05:
                return None
        except np.linalg.LinAlgError:
            return None
        return g, H, o["grad_abs"]
    return at


def _response_with_bound(ev):
    """R(theta; sigma_q) in FP64 and the error float32 adds to it at theta:
    each residual is one rounding of x - t_x w (about x0 + r, so at most
    2^-24 (|x0| + |r|)) followed by an exact subtraction, and a residual error
    dr moves a term by at most e 2 |r| dr / sigma^2 (plus R's own 1e-5)."""
    h = ev.hits.astype(np.float64)
    sig = SIGMA[-1]

    def at(th):
        w = h[:, 2] - ZREF
        r0 = h[:, 0] - th[0] - th[2] * w
        r1 = h[:, 1] - th[1] - th[3] * w
        e = np.exp(-(r0 * r0 + r1 * r1) / sig ** 2)
        u = 2.0 ** -24
        dr0 = u * (abs(th[0]) + np.abs(r0))
        dr1 = u * (abs(th[1]) + np.abs(r1))
        bound = float(np.sum(e * 2.0 * (np.abs(r0) * dr0 + np.abs(r1) * dr1) / sig ** 2))
        return oracle.response4(ev.hits, th, sig, zref=ZREF), bound
    return at


def test_search4_matches_oracle_on_a_smeared_vertex_event(rt):
    # point-wise parity on every robust seed whose path the oracle's perturbed
    # replicas show to be well conditioned; ill-conditioned paths must end in
    # the region the replicas reach (check_conditioned, shared with the
    # modified-Newton parity test)
    ev, truth4, seeds = _event_and_seeds()
    off = torch.tensor([0, ev.n_hits], dtype=torch.int64, device="cuda")
    th_g, R_g, st_g = rt.local_search4(torch.from_numpy(ev.hits).cuda(), off, torch.from_numpy(seeds).cuda()[None],
                                       rt.LsOpts4(sigma=SIGMA, scale=SCALE, zref=ZREF))
    th_g, R_g, st_g = th_g.cpu().numpy()[0].astype(float), R_g.cpu().numpy()[0].astype(float), st_g.cpu().numpy()[0]

    def run(pt):
        return oracle.local_search4(ev.hits, seeds, SIGMA, SCALE, zref=ZREF, perturb=pt)

    check_conditioned(th_g, R_g, st_g, run(None), run, SCALE, _converged_at(ev), _response_with_bound(ev),
                      min_firm_conv=CONV_MIN)


def test_search4_edge_cases(rt):
    # an event without hits (R = 0, g = 0: p = 0, the unit trial passes, theta
    # stays) and an event with one hit; malformed offsets are clamped
    hits = np.array([[1.0, -2.0, 100.0, 0.0]], np.float32)
    seeds = np.array([[[0.0, 0.0, 0.01, -0.02], [0.5, -0.5, 0.0, 0.0]]] * 2, np.float32)
    off = torch.tensor([0, 0, 1], dtype=torch.int64, device="cuda")
    th, R, st = rt.local_search4(torch.from_numpy(hits).cuda(), off, torch.from_numpy(seeds).cuda(),
                                 rt.LsOpts4(sigma=SIGMA, scale=SCALE))
    th, R, st = th.cpu().numpy(), R.cpu().numpy(), st.cpu().numpy()
    assert np.all(R[0] == 0) and np.all(th[0] == seeds[0]) and np.all(st[0] == 0)
    th_o, R_o, st_o, m_o = oracle.local_search4(hits, seeds[1], SIGMA, SCALE)
    ok = m_o >= 1
    assert np.all(st[1][ok] == st_o[ok])
    assert np.all(np.abs(R[1][ok] - R_o[ok]) <= R_REL * R_o[ok] + R_ABS)
    bad = torch.tensor([0, 5, -3], dtype=torch.int64, device="cuda")
    th, R, st = rt.local_search4(torch.from_numpy(hits).cuda(), bad, torch.from_numpy(seeds).cuda(),
                                 rt.LsOpts4(sigma=SIGMA, scale=SCALE))
    torch.cuda.synchronize()
    assert np.all(np.isfinite(R.cpu().numpy()))

