"""Oracle for the retrieval steps (distance, top-N, coarse-to-fine, windows).

TEST INFRASTRUCTURE ONLY -- imported by tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the library.

All arithmetic is IEEE double. Readings of the paper taken here:

* The distance is Euclidean (§4, "smallest Euclidean distance"); candidates
  are ranked by, and reported as, the squared distance, which orders the same.
* Top-N is taken per query frame and per database subspace (§3.1: each frame
  is compared with all frames of every subspace; §4: N x M x P candidates).
* Ties are broken by the lower database row index; a subspace with fewer than
  N rows pads its list with row -1 and distance +inf.
* The coarse-to-fine level (not in the paper; it is this build's hierarchical
  form) scores the first ``coarse_dim`` feature dimensions over all rows,
  keeps the ``shortlist`` best, and ranks those by the full-vector distance.
"""
from __future__ import annotations

import numpy as np

_ROW_CHUNK = 1 << 15


def sq_dist(q, X, w=None) -> np.ndarray:
    """Squared Euclidean distance of query ``q`` (D,) to every row of ``X`` (n, D).

    §3.1 ``calculateDistance(q_m, f_i)`` and §4 (Euclidean). With per-dimension
    weights ``w`` (D,) each squared difference is multiplied by w_j.
    """
    q = np.asarray(q, dtype=np.float64)
    X = np.asarray(X)
    out = np.empty(X.shape[0], dtype=np.float64)
    wv = None if w is None else np.asarray(w, dtype=np.float64)
    for s in range(0, X.shape[0], _ROW_CHUNK):
        diff = X[s:s + _ROW_CHUNK].astype(np.float64) - q
        sq = diff * diff
        if wv is not None:
            sq = sq * wv
        out[s:s + _ROW_CHUNK] = sq.sum(axis=1)
    return out


def top_n(d: np.ndarray, rows: np.ndarray, n: int):
    """The ``n`` smallest (distance, row) pairs in ascending (distance, row) order.

    §3.1 ``selectTopCandidates()``: a stable ascending sort, first n entries;
    positions beyond the available rows hold row -1 and distance +inf.
    """
    d = np.asarray(d, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    order = np.lexsort((rows, d))[:n]
    idx = np.full(n, -1, dtype=np.int64)
    dist = np.full(n, np.inf, dtype=np.float64)
    idx[:order.size] = rows[order]
    dist[:order.size] = d[order]
    return idx, dist


def exhaustive_topk(Q, X, k: int, subspace=None, n_subspaces: int | None = None, w=None):
    """Exhaustive per-frame, per-subspace top-k (§3.1, Algorithm 1).

    Returns ``idx`` int64 (nq, n_s, k) and ``dist`` float64 (nq, n_s, k).
    ``subspace`` (n,) gives each row's subspace id in [0, n_s); None means one
    subspace holding every row.
    """
    Q = np.atleast_2d(np.asarray(Q))
    X = np.asarray(X)
    n = X.shape[0]
    if subspace is None:
        groups = [np.arange(n, dtype=np.int64)]
    else:
        subspace = np.asarray(subspace)
        ns = int(subspace.max()) + 1 if n_subspaces is None else int(n_subspaces)
        groups = [np.nonzero(subspace == s)[0].astype(np.int64) for s in range(ns)]
    idx = np.empty((Q.shape[0], len(groups), k), dtype=np.int64)
    dist = np.empty((Q.shape[0], len(groups), k), dtype=np.float64)
    for qi in range(Q.shape[0]):
        d = sq_dist(Q[qi], X, w)
        for s, rows in enumerate(groups):
            idx[qi, s], dist[qi, s] = top_n(d[rows], rows, k)
    return idx, dist


def hierarchical_topk(Q, X, coarse_dim: int, shortlist: int, k: int):
    """Coarse-to-fine top-k: prefix distance over all rows, then full distance.

    Step 1: d_c = squared distance over dimensions [0, coarse_dim) for every
    row; keep the ``shortlist`` smallest by (d_c, row). Step 2: full squared
    distance on those rows; keep the ``k`` smallest by (d, row).
    Returns ``idx`` int64 (nq, k), ``dist`` float64 (nq, k) and the shortlist
    rows int64 (nq, shortlist) in coarse order.
    """
    Q = np.atleast_2d(np.asarray(Q))
    X = np.asarray(X)
    n = X.shape[0]
    all_rows = np.arange(n, dtype=np.int64)
    idx = np.empty((Q.shape[0], k), dtype=np.int64)
    dist = np.empty((Q.shape[0], k), dtype=np.float64)
    short = np.empty((Q.shape[0], shortlist), dtype=np.int64)
    for qi in range(Q.shape[0]):
        dc = sq_dist(Q[qi, :coarse_dim], X[:, :coarse_dim])
        s_rows, _ = top_n(dc, all_rows, shortlist)
        short[qi] = s_rows
        valid = s_rows[s_rows >= 0]
        d = sq_dist(Q[qi], X[valid])
        idx[qi], dist[qi] = top_n(d, valid, k)
    return idx, dist, short


def hierarchical_topk_subspaces(Q, X, coarse_dim: int, shortlist: int, k: int, subspace, n_subspaces=None):
    """Coarse-to-fine top-k of every frame in every subspace (§3.1: each
    subspace is searched on its own): ``hierarchical_topk`` over the rows of
    subspace s alone, its rows reported in the database's numbering.
    Returns ``idx`` int64 (nq, n_s, k) and ``dist`` float64 (nq, n_s, k).
    """
    Q = np.atleast_2d(np.asarray(Q))
    X = np.asarray(X)
    subspace = np.asarray(subspace)
    ns = int(subspace.max()) + 1 if n_subspaces is None else int(n_subspaces)
    idx = np.empty((Q.shape[0], ns, k), dtype=np.int64)
    dist = np.empty((Q.shape[0], ns, k), dtype=np.float64)
    for s in range(ns):
        rows = np.nonzero(subspace == s)[0].astype(np.int64)
        i_s, d_s, _ = hierarchical_topk(Q, X[rows], coarse_dim, shortlist, k)
        idx[:, s] = np.where(i_s >= 0, rows[np.maximum(i_s, 0)], -1)
        dist[:, s] = d_s
    return idx, dist


def window_candidates(frame_idx: np.ndarray, offsets: np.ndarray):
    """Candidates of each window: the per-frame lists of its frames, concatenated.

    §3.1: a request for frame q_m carries its neighbouring frames and every
    frame is queried; §4: all returned candidates, duplicates included, go to
    aggregation (N x M x P of them). ``frame_idx`` is (W, ...) per frame.
    """
    frame_idx = np.asarray(frame_idx)
    offsets = np.asarray(offsets, dtype=np.int64)
    out = []
    for w in range(offsets.size - 1):
        out.append(frame_idx[offsets[w]:offsets[w + 1]].reshape(-1))
    return out
