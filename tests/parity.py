"""Comparison rules between the CUDA path and the FP64 oracle.

* Indices: bit-exact at every rank whose oracle distance is separated from
  its neighbours by more than GAP (relative); inside a near-tie group any
  member is accepted, provided its exact distance lies in the group's range.
  The returned set equals the oracle's whenever the k-th / (k+1)-th gap
  exceeds GAP.
* Distances: every returned distance within DIST_RTOL of the exact FP64
  distance of the returned row.
* Locations: within XY_ATOL metres.
"""
import numpy as np

from oracle import retrieval as oret

GAP = 1e-4
DIST_RTOL = 1e-5
XY_ATOL = 1e-3


def _sep(d, r):
    """True when oracle distance d[r] is more than GAP away from both neighbours."""
    scale = max(abs(d[r]), 1e-12)
    left = r == 0 or (d[r] - d[r - 1]) > GAP * scale
    right = r + 1 >= len(d) or (d[r + 1] - d[r]) > GAP * scale
    return left and right


def check_list(q, X, g_idx, g_dist, o_idx, o_dist, k, rows=None, where="", w=None):
    """One query's GPU list (k entries) against the oracle's top-(k+1) list.

    ``rows`` restricts the candidate rows (a subspace); ``o_idx``/``o_dist``
    must hold at least k entries (k+1 when available) in oracle order; ``w``
    are per-dimension distance weights (None = 1).
    Returns the number of positions compared bit-exactly.
    """
    g_idx = np.asarray(g_idx)
    g_dist = np.asarray(g_dist, dtype=np.float64)
    valid = g_idx >= 0
    n_avail = int(np.sum(np.asarray(o_idx[:k]) >= 0))
    assert valid.sum() == n_avail, f"{where}: {valid.sum()} rows returned, oracle has {n_avail}"
    assert np.all(valid[:n_avail]) and not np.any(valid[n_avail:]), f"{where}: padding not at the tail"
    assert np.all(np.isinf(g_dist[n_avail:])), f"{where}: padding distance must be +inf"
    if n_avail == 0:
        return 0
    gi = g_idx[:n_avail]
    assert len(set(gi.tolist())) == n_avail, f"{where}: duplicate rows"
    if rows is not None:
        assert np.isin(gi, rows).all(), f"{where}: row outside the subspace"
    exact = oret.sq_dist(q, X[gi], w)
    err = np.abs(g_dist[:n_avail] - exact)
    assert np.all(err <= DIST_RTOL * exact + 1e-7), \
        f"{where}: distance error {np.max(err / np.maximum(exact, 1e-12)):.3g} rel"
    assert np.all(np.diff(g_dist[:n_avail]) >= 0), f"{where}: list not ascending"
    od = np.asarray(o_dist, dtype=np.float64)
    oi = np.asarray(o_idx)
    exact_cmp = 0
    for r in range(n_avail):
        if _sep(od[:min(len(od), n_avail + 1)], r):
            assert gi[r] == oi[r], f"{where}: rank {r}: row {gi[r]} != oracle {oi[r]} (d {exact[r]} vs {od[r]})"
            exact_cmp += 1
        else:
            lo = od[r] * (1 - 2 * GAP) - 1e-7
            hi = od[r] * (1 + 2 * GAP) + 1e-7
            assert lo <= exact[r] <= hi, f"{where}: rank {r}: near-tie member out of range"
    if len(od) > n_avail and n_avail == k:
        if od[k] - od[k - 1] > GAP * max(od[k - 1], 1e-12):
            assert set(gi.tolist()) == set(oi[:k].tolist()), f"{where}: top-k set differs"
    return exact_cmp


def check_hier_ambiguous(q, X, dc, S, g_idx, g_dist, k, where=""):
    """Coarse-to-fine list of a frame whose S-th / (S+1)-th coarse distances nearly
    tie, so that which boundary rows enter the shortlist is decided by rounding.
    The list must be the exact top k of SOME valid shortlist: every returned row's
    coarse distance is at most the S-th one (+ 2 GAP), distances are exact and
    ascending, and every row whose coarse distance is surely below the boundary
    (- 2 GAP) and whose full distance is below the list's k-th (- 2 GAP) is in it."""
    g_idx = np.asarray(g_idx)
    g_dist = np.asarray(g_dist, dtype=np.float64)
    dcoarse = oret.sq_dist(q[:dc], X[:, :dc])
    cS = np.sort(dcoarse)[S - 1]
    lo, hi = cS * (1 - 2 * GAP), cS * (1 + 2 * GAP) + 1e-12
    n_ret = min(k, X.shape[0])
    gi = g_idx[:n_ret]
    assert np.all(gi >= 0) and len(set(gi.tolist())) == n_ret, f"{where}: padding or duplicate rows"
    assert np.all(dcoarse[gi] <= hi), f"{where}: a returned row cannot be in any valid shortlist"
    exact = oret.sq_dist(q, X[gi])
    assert np.all(np.abs(g_dist[:n_ret] - exact) <= DIST_RTOL * exact + 1e-7), f"{where}: distance error"
    assert np.all(np.diff(g_dist[:n_ret]) >= 0), f"{where}: list not ascending"
    sure = np.nonzero(dcoarse < lo)[0]
    full = oret.sq_dist(q, X[sure])
    must = set(sure[full < g_dist[n_ret - 1] * (1 - 2 * GAP) - 1e-7].tolist())
    assert must <= set(gi.tolist()), f"{where}: rows {sorted(must - set(gi.tolist()))[:5]} missing"
