"""The host restatement of the prepared-hit order, pinned on the CPU: its
Hilbert index against the curve's defining properties, and its order against
what the documentation fixes (a permutation, grouped by band, each chunk in
code order)."""
import numpy as np

import pytest

from hit_order import bands_codes, documented_order, hilbert


@pytest.mark.parametrize("order", [1, 2, 8, 9])
def test_host_hilbert_is_a_hilbert_curve(order):
    # the restatement against the curve's defining properties: a bijection of
    # the 2^order x 2^order cells onto 0 .. 4^order - 1 whose consecutive
    # cells share an edge, from (0, 0) to (2^order - 1, 0), each quarter of the
    # index range filling one quadrant, the quadrants in the cup order (0,0),
    # (0,1), (1,1), (1,0); at order 2 the curve is the textbook one
    n = 1 << order
    X, Y = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    d = hilbert(X.ravel(), Y.ravel(), order)
    assert np.array_equal(np.sort(d), np.arange(n * n))
    inv = np.empty((n * n, 2), np.int64)
    inv[d] = np.stack([X.ravel(), Y.ravel()], 1)
    assert np.all(np.abs(np.diff(inv, axis=0)).sum(1) == 1)
    assert tuple(inv[0]) == (0, 0) and tuple(inv[-1]) == (n - 1, 0)
    h = n // 2
    quad = (inv[:, 0] // h) * 2 + (inv[:, 1] // h)
    q4 = n * n // 4
    assert [set(quad[q * q4:(q + 1) * q4]) for q in range(4)] == [{0}, {1}, {3}, {2}]
    if order == 2:
        path = [tuple(c) for c in inv]
        assert path == [(0, 0), (1, 0), (1, 1), (0, 1), (0, 2), (0, 3), (1, 3), (1, 2),
                        (2, 2), (2, 3), (3, 3), (3, 2), (3, 1), (2, 1), (2, 0), (3, 0)]


def test_documented_order_sorts_each_super_chunk():
    rng = np.random.default_rng(3)
    n = 40000  # two super-chunks
    h = np.zeros((n, 4), np.float32)
    h[:, 2] = rng.choice([-300.0, -20.0, 40.0, 100.0, 200.0, 300.0, 700.0], n) * rng.uniform(0.9, 1.0, n)
    h[:, :2] = rng.uniform(-0.3, 0.3, (n, 2)) * np.abs(h[:, 2:3])
    h[::97, :2] = 0.0  # repeated codes: ties keep index order
    p = documented_order(h, 1)
    assert np.array_equal(np.sort(p), np.arange(n))
    band, _ = bands_codes(h, 1)
    for s0, s1 in ((0, 32768), (32768, n)):
        q = p[s0:s1]
        assert q.min() == s0 and q.max() == s1 - 1  # a super-chunk stays in place
        _, c = bands_codes(h[s0:s1], 1)
        c = c[q - s0]
        assert np.all(np.diff(c) >= 0)  # codes ascend
        tie = np.diff(c) == 0
        assert tie.any() and np.all(np.diff(q)[tie] > 0)  # equal codes in index order
        assert np.all(np.diff(band[q]) >= 0)  # so the bands come grouped
