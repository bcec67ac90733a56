"""Host restatement of retina_prepare_hits' documented hit order (test
infrastructure): each super-chunk of 32768 consecutive hits of an event is
sorted by (spatial code, index).  Slope model: code = octave band of |z| from
16 mm (7 bands, NaN in the last) above the Hilbert index (order 8) of the
slopes quantised on [-1, 1]; 2D toy: code = a band of x above the quantised y.
"""
import numpy as np


def hilbert(x, y, order=8):
    """Hilbert index of cells (x, y) in [0, 2^order)^2, quadrant by quadrant from
    the top level: quadrants taken in the order (0,0), (0,1), (1,1), (1,0),
    the first one's frame transposed and the last one's reflected through the
    anti-diagonal."""
    x = x.astype(np.int64).copy()
    y = y.astype(np.int64).copy()
    d = np.zeros_like(x)
    for lev in range(order - 1, -1, -1):
        s = 1 << lev
        rx, ry = (x >> lev) & 1, (y >> lev) & 1
        d += s * s * ((3 * rx) ^ ry)
        x, y = x & (s - 1), y & (s - 1)
        flip = (ry == 0) & (rx == 1)
        x, y = np.where(flip, s - 1 - x, x), np.where(flip, s - 1 - y, y)
        x, y = np.where(ry == 0, y, x), np.where(ry == 0, x, y)
    return d


def _quant(v, lo, inv_range, levels):
    with np.errstate(invalid="ignore", over="ignore"):
        t = ((v - np.float32(lo)) * np.float32(inv_range)).astype(np.float32)
        t = np.where(np.isfinite(t), np.clip(t, 0, 1), np.where(t > 0, 1, 0)).astype(np.float32)
        return (t * np.float32(levels)).astype(np.int64)


def bands_codes(h, model):
    h = h.astype(np.float32)
    if model != 1:
        u = h[:, 0].view(np.uint32).astype(np.int64)
        key = np.where(u & 0x80000000, ~u & 0xffffffff, u | 0x80000000)
        return np.zeros(len(h), np.int64), ((key >> 25) << 7) | _quant(h[:, 1], -8, 1 / 16, 127)
    az = np.abs(h[:, 2])
    band = np.zeros(len(h), np.int64)
    for k in range(6):
        band += ~(az < np.float32(16 * 2 ** k))  # NaN lands in the last band
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        rz = (np.float32(1) / h[:, 2]).astype(np.float32)
        u, v = (h[:, 0] * rz).astype(np.float32), (h[:, 1] * rz).astype(np.float32)
    return band, (band << 16) | hilbert(_quant(u, -1, 0.5, 255), _quant(v, -1, 0.5, 255))


def documented_order(h, model):
    perm = []
    for s0 in range(0, len(h), 32768):
        _, code = bands_codes(h[s0:s0 + 32768], model)
        perm.append(s0 + np.lexsort((np.arange(len(code)), code)))
    return np.concatenate(perm) if perm else np.zeros(0, np.int64)
