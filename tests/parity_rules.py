"""Parity rules shared by the GPU tests (CUDA path vs the FP64 oracle).

Tolerances, from the FP32 arithmetic of the kernels:
  R                 |dR| <= 1e-5 R + 1e-6
  gradient, Hessian |d|  <= 1e-4 * sum of |terms|
  end points        |dtheta| <= 1e-3 of a grid step (or parameter unit) at
                    converged maxima
"""
import numpy as np

import oracle

R_REL, R_ABS = 1e-5, 1e-6
GH_REL = 1e-4
TH_CELLS = 1e-3


def check_conditioned(th_g, R_g, st_g, base, run, units, converged_at, response_at, min_firm_conv):
    """Point-wise parity for searches whose paths may amplify float32
    rounding (the shifted modified-Newton step, the four-parameter search).

    Per seed, the comparison tolerance is 1e-3 of a unit per parameter where
    the oracle's end point is a converged maximum (``converged_at(theta)``
    returns the oracle's (gradient, Hessian, |gradient terms|) there, or None:
    negative-definite Hessian and Newton distance <= 0.05 unit) - widened to
    |H^-1| (1e-4 sum |gradient terms|), the displacement the gradient
    tolerance allows, on an ill-conditioned peak - and 0.05 unit elsewhere.
    Seeds with an oracle decision within tolerance of its threshold (margin
    < 1) are ties (either outcome is correct) and are counted, not compared.
    The other seeds' paths are rerun by the oracle with every float32
    quantity displaced within its tolerance (oracle.path_conditioning):
    * well conditioned (every replica ends with the same status within the
      seed's tolerance): same status, end point within the tolerance, R within
      its tolerance plus |g| dtheta + |H| dtheta^2;
    * ill conditioned: several end points are correct, so what is checked
      is what the CUDA path reports about its own: a status one of the
      oracle's runs (unperturbed or replica) ended with, and R at its end
      point equal, within R's tolerance, to the oracle's R at that same point
      (``response_at(theta)``: R(theta; sigma_q) in FP64, or (R, extra) with
      an absolute term the kernel's own rounding adds to the tolerance).
    Returns the counts (firm, firm converged, ill conditioned, ties)."""
    th_o, R_o, st_o, m_o = base
    units = np.asarray(units, dtype=np.float64)
    n, d = th_o.shape
    tol = np.tile(0.05 * units, (n, 1))
    conv = np.zeros(n, dtype=bool)
    info = {}
    for i in np.flatnonzero(st_o <= 1):
        c = converged_at(th_o[i])
        if c is None:
            continue
        g, H, gabs = c
        conv[i] = True
        info[i] = (g, H)
        tol[i] = np.maximum(TH_CELLS * units, np.abs(np.linalg.inv(H)) @ (GH_REL * gabs))
    robust = m_o >= 1.0
    stable, _, sts = oracle.path_conditioning(run, base, tol)
    firm = robust & stable
    for i in np.flatnonzero(firm):
        assert st_g[i] == st_o[i], (i, st_g[i], st_o[i])
        if st_o[i] > 2:
            continue
        dth = np.abs(th_g[i] - th_o[i])
        assert np.all(dth <= tol[i]), (i, conv[i], dth / units)
        if i in info:
            g, H = info[i]
            r_tol = R_REL * R_o[i] + R_ABS + np.abs(g) @ tol[i] + np.abs(H).max() * (tol[i] @ tol[i])
            assert abs(R_g[i] - R_o[i]) <= r_tol, (i, R_g[i], R_o[i], r_tol)
    ill = robust & ~stable
    for i in np.flatnonzero(ill):
        assert st_g[i] == st_o[i] or st_g[i] in sts[:, i], (i, st_g[i], st_o[i], sts[:, i])
        if st_g[i] > 2:
            continue
        r_at = response_at(th_g[i])
        r_at, extra = r_at if isinstance(r_at, tuple) else (r_at, 0.0)
        assert abs(R_g[i] - r_at) <= R_REL * r_at + R_ABS + extra, (i, R_g[i], r_at, extra)
    n_firm_conv = int((firm & conv).sum())
    assert n_firm_conv >= min_firm_conv, (n_firm_conv, int(conv.sum()), int(firm.sum()), int(ill.sum()))
    return int(firm.sum()), n_firm_conv, int(ill.sum()), int((~robust).sum())


def compare_track_sets(pos_o, R_o, cand_o, pos_g, R_g, cand_g, tie, kept_o, kept_g, tol, step, merge_cells,
                       R0=None):
    """Found-track sets of the CUDA path and the oracle, equal up to near-ties.

    Items are the starting points of the extraction (search seeds, or grid
    cells), indexed alike on both sides: end points pos_* [n, D] (NaN where a
    side has none), responses R_* [n], candidate masks cand_* [n] (what each
    side's cluster/select step considered), ``tie`` [n] the items whose own
    outcome is a near-tie (an oracle decision within tolerance of its
    threshold), kept_* the indices each side kept, ``tol`` [n, 2] the
    position tolerance of each item.

    The greedy selection decides each cluster from its own candidates only, so
    the candidates are split into components (linked when closer than the
    merge distance plus the position tolerance, on either side's positions).
    A component is tied when it holds a tie item, an item that only one side
    counts as a candidate, an item at R0 within R's tolerance, two items at
    distinct positions (farther apart than their tolerance) but within the
    merge distance whose responses are equal within R's tolerance (their order
    decides which is kept), or two items within their tolerance of the merge
    distance.  An item that is not a tie and not at R0 must be a candidate on
    both sides or on neither.  In every other component the kept positions
    must be the same on both sides within the tolerance.  Returns
    (components, tied components, oracle tracks compared)."""
    n = len(R_o)
    dim = pos_o.shape[1]
    step = np.asarray(step, dtype=np.float64)
    tol = np.broadcast_to(np.asarray(tol, dtype=np.float64), (n, dim))
    tolR = lambda r: R_REL * np.abs(r) + R_ABS
    items = np.flatnonzero(cand_o | cand_g)
    if len(items) == 0:
        assert len(kept_o) == 0 and len(kept_g) == 0
        return 0, 0, 0
    # positions in cells; an item present on one side only uses that side's
    P_o = np.where(np.isfinite(pos_o[items]), pos_o[items], pos_g[items]) / step
    P_g = np.where(np.isfinite(pos_g[items]), pos_g[items], pos_o[items]) / step
    T = tol[items] / step
    Rm = np.where(np.isfinite(R_o[items]), R_o[items], R_g[items])
    m = len(items)
    parent = np.arange(m)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    from scipy.spatial import cKDTree
    tmax = np.max(T, axis=1)
    r = merge_cells + 2 * float(tmax.max())
    pairs = set()
    for P in (P_o, P_g):
        pairs |= cKDTree(P).query_pairs(r, p=np.inf)
    pairs = np.array(sorted(pairs), dtype=np.int64).reshape(-1, 2)
    a, b = pairs[:, 0], pairs[:, 1]
    d_o = np.max(np.abs(P_o[a] - P_o[b]), axis=1)
    d_g = np.max(np.abs(P_g[a] - P_g[b]), axis=1)
    slack = tmax[a] + tmax[b]
    link = np.minimum(d_o, d_g) < merge_cells + slack
    for x, y in zip(a[link], b[link]):
        rx, ry = find(x), find(y)
        if rx != ry:
            parent[rx] = ry
    root = np.array([find(k) for k in range(m)])
    at_R0 = (np.abs(Rm - R0) <= tolR(Rm)) if R0 is not None else np.zeros(m, dtype=bool)
    one_sided = cand_o[items] != cand_g[items]
    # an item whose own outcome is firm is a candidate on both sides or on neither
    assert not np.any(one_sided & ~tie[items] & ~at_R0), \
        ("firm items counted as candidates by one side only", items[one_sided & ~tie[items] & ~at_R0])
    bad = tie[items] | one_sided | at_R0
    near = np.abs(Rm[a] - Rm[b]) <= tolR(Rm[a]) + tolR(Rm[b])
    order_tie = near & (d_o > slack) & (d_o < merge_cells + slack)
    boundary_tie = np.abs(d_o - merge_cells) <= slack
    for mask in (order_tie, boundary_tie):
        bad[a[mask]] = True
        bad[b[mask]] = True
    tied_roots = set(root[bad].tolist())
    where = {int(it): k for k, it in enumerate(items)}
    ko = [i for i in kept_o if where.get(int(i)) is not None and root[where[int(i)]] not in tied_roots]
    kg = [i for i in kept_g if where.get(int(i)) is not None and root[where[int(i)]] not in tied_roots]
    # kept items outside every candidate set cannot happen
    assert all(int(i) in where for i in kept_o) and all(int(i) in where for i in kept_g)
    # each side's kept positions in untied components have a partner on the other side
    A = pos_o[np.asarray(ko, dtype=np.int64)].reshape(-1, dim)
    B = pos_g[np.asarray(kg, dtype=np.int64)].reshape(-1, dim)
    ta = tol[np.asarray(ko, dtype=np.int64)].reshape(-1, dim)
    tb = tol[np.asarray(kg, dtype=np.int64)].reshape(-1, dim)
    assert len(A) == len(B), ("kept counts differ in untied components", len(A), len(B))
    if len(A):
        dA = np.abs(A[:, None] - B[None])
        okA = np.all(dA <= ta[:, None] + tb[None], axis=2)
        assert np.all(okA.any(axis=1)), ("oracle tracks without a CUDA partner", A[~okA.any(axis=1)] / step)
        assert np.all(okA.any(axis=0)), ("CUDA tracks without an oracle partner", B[~okA.any(axis=0)] / step)
    return len(set(root.tolist())), len(tied_roots), len(A)


def search_tolerance(converged_at, th_o, items, units):
    """Position tolerance [n, 2] of search end points: 1e-3 of a unit (or the
    displacement the gradient tolerance allows on an ill-conditioned peak)
    where the oracle's end point is a converged maximum, 0.05 unit
    elsewhere; only ``items`` are evaluated (others get 0.05 unit)."""
    units = np.asarray(units, dtype=np.float64)
    tol = np.tile(0.05 * units, (len(th_o), 1))
    for i in np.flatnonzero(items):
        c = converged_at(th_o[i])
        if c is not None:
            g, H, gabs = c
            tol[i] = np.maximum(TH_CELLS * units, np.abs(np.linalg.inv(H)) @ (GH_REL * gabs))
    return tol


def candidates(theta, R, status, lo, step, n, R0):
    """The extraction's candidate rule: status 0/1, finite, inside the box, R >= R0."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = lo + np.asarray(n, dtype=np.float64) * np.asarray(step, dtype=np.float64)
    ok = np.isfinite(R) & np.all(np.isfinite(theta), axis=1) & (R >= R0)
    ok &= np.all((theta >= lo) & (theta < hi), axis=1)
    if status is not None:
        ok &= status <= 1
    return ok
