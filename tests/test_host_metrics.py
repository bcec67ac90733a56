"""Host-side evaluation helpers of the batch pipeline (no GPU): MC matching,
residuals, efficiency by multiplicity, recovered fraction."""
import numpy as np

from paper_1709_08610_gb300.pipeline import (efficiency_by_multiplicity, match_efficiency, match_residuals,
                                             recovered_fraction)


def test_match_efficiency_counts_matches_and_fakes():
    truth = [np.array([[0.0, 0.0], [0.1, 0.1]]), np.array([[0.2, -0.2]])]
    found = [np.array([[0.0005, -0.0009], [0.5, 0.5]]), np.zeros((0, 2))]
    eff, fakes = match_efficiency(found, truth, eps=1e-3)
    assert eff == 1 / 3 and fakes == 1
    # max norm: 1.1e-3 in one coordinate misses
    eff, _ = match_efficiency([np.array([[0.0011, 0.0]])], [np.array([[0.0, 0.0]])], eps=1e-3)
    assert eff == 0.0


def test_residuals_are_the_nearest_found_track_per_matched_truth_track():
    truth = [np.array([[0.0, 0.0], [0.1, 0.1], [0.3, 0.3]])]
    found = [np.array([[0.0002, -0.0001], [0.0009, 0.0], [0.1, 0.1004]])]
    r = match_residuals(found, truth, eps=1e-3)
    np.testing.assert_allclose(r, [[0.0002, 0.0001], [0.0, 0.0004]], atol=1e-15)


def test_efficiency_by_multiplicity_bins_events_by_truth_count():
    truth = [np.zeros((10, 2)), np.ones((25, 2)), np.zeros((10, 2))]
    found = [np.zeros((1, 2)), np.zeros((0, 2)), np.zeros((0, 2))]
    out = efficiency_by_multiplicity(found, truth, [10, 25, 50])
    assert out == {"10-25": {"events": 2, "efficiency": 0.5}, "25-50": {"events": 1, "efficiency": 0.0}}


def test_recovered_fraction_is_matching_against_the_reference_method():
    ref = [np.array([[0.0, 0.0], [0.5, 0.5]])]
    got = [np.array([[0.0, 0.0004]])]
    assert recovered_fraction(got, ref) == 0.5
