"""The paper's sVELO generator (Section 4): geometry, acceptance, hit counts,
noise and the angle parametrisation, checked against their definitions."""
import math

import numpy as np
import pytest

from synth import SVELO_PLANES_Z, WORKLOADS, make_event, make_svelo_event, slopes_to_angles
from synth.events import SVELO_R_INNER, SVELO_R_OUTER


def test_layers_are_twenty_equally_spaced_within_700mm():
    assert SVELO_PLANES_Z.size == 20
    assert np.allclose(np.diff(SVELO_PLANES_Z), 35.0) and SVELO_PLANES_Z[-1] == 700.0


@pytest.mark.parametrize("n", [50, 200, 350])
def test_reconstructible_tracks_and_their_hits(n):
    ev = make_svelo_event(4, n, n_tracks=n)
    assert ev.truth.shape == (n, 6)
    h = ev.hits.astype(np.float64)
    assert set(np.unique(h[:, 2])) <= set(SVELO_PLANES_Z)
    for t in range(n):
        k = ev.labels == t
        assert k.sum() == ev.truth[t, 5] >= 2
        u, v = ev.truth[t, :2]
        # on the track within 6 sigma of the 1e-2 mm measurement error, inside the annulus up to it
        assert np.all(np.abs(h[k, 0] - u * h[k, 2]) < 0.06) and np.all(np.abs(h[k, 1] - v * h[k, 2]) < 0.06)
        r = np.hypot(u * h[k, 2], v * h[k, 2])
        assert np.all((r >= SVELO_R_INNER) & (r <= SVELO_R_OUTER))
        # pseudo-rapidity of the track within [1, 6]
        eta = -math.log(math.tan(0.5 * math.atan(math.hypot(u, v))))
        assert 1.0 <= eta <= 6.0


def test_noise_is_on_the_annuli_and_poisson_250():
    counts = []
    for e in range(40):
        ev = make_svelo_event(5, e, n_tracks=20)
        h = ev.hits[ev.labels < 0].astype(np.float64)
        r = np.hypot(h[:, 0], h[:, 1])
        # noise, plus the hits of undetectable tracks (fewer than 2 hits, all in the annulus)
        assert np.all((r >= SVELO_R_INNER - 0.1) & (r <= SVELO_R_OUTER + 0.1))
        counts.append(len(h))
    # Poisson(250) noise plus a few single-hit tracks: the mean sits a little above 250
    assert 245 < np.mean(counts) < 290


def test_seeded_and_reproducible():
    a = make_event(WORKLOADS["svelo"], 9, 3)
    b = make_event(WORKLOADS["svelo"], 9, 3)
    c = make_event(WORKLOADS["svelo"], 9, 4)
    assert np.array_equal(a.hits, b.hits) and np.array_equal(a.truth, b.truth)
    assert not np.array_equal(a.hits[:10], c.hits[:10])


def test_slopes_to_angles_inverts_the_paper_parametrisation():
    # x = t sin(theta), y = t cos(theta) sin(phi), z = t cos(theta) cos(phi)
    rng = np.random.default_rng(1)
    th = rng.uniform(-0.7, 0.7, 100)
    ph = rng.uniform(-0.7, 0.7, 100)
    d = np.stack([np.sin(th), np.cos(th) * np.sin(ph), np.cos(th) * np.cos(ph)], 1)
    a = slopes_to_angles(d[:, 0] / d[:, 2], d[:, 1] / d[:, 2])
    np.testing.assert_allclose(a[:, 0], th, atol=1e-14)
    np.testing.assert_allclose(a[:, 1], ph, atol=1e-14)
