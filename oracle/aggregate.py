"""Oracle for Algorithm 2: 2-D multi-frame localization candidate aggregation.

TEST INFRASTRUCTURE ONLY -- imported by tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the library.

Algorithm 2 with the text after it (§3.2): candidate rows are mapped to
floor-plan coordinates through the geo-referenced table, the plan is cut into
square tiles (30 cm, the ground-tile width), candidates are counted per tile,
the tiles are ranked by count, and the first TopC (10) tiles are visited in
rank order; the first whose tolerance circle (radius 3 m) holds more than
tolerPer (20 %) of all candidates is the final position.

Readings taken where the paper is silent or loose:

* Tiles are half-open [i t, (i+1) t) from the plan origin: tx = floor(x / t),
  ty = floor(y / t) in IEEE double (a correctly rounded divide).
* Equal counts are ranked by ty, then tx, ascending.
* The tolerance circle is taken over tiles (Algorithm 2 works on the tile
  count array): a tile belongs to the circle of tile r when its centre lies
  within the radius of r's centre, i.e. the integer test
  (tx - tx_r)^2 + (ty - ty_r)^2 <= floor((radius / t)^2), where radius / t and
  its square are snapped to the nearest integer when within 1e-9 relative
  (3 m / 0.3 m gives exactly 10, so the limit is 100).
* "Greater than tolerPer of all candidates" is strict and evaluated in
  integers: 100 * circle > toler_pct * C, C counting duplicates (§4: a star
  may stand for several candidates). Rows -1 (padding) are not candidates.
* If no TopC tile passes, the top-ranked tile is returned with status 1
  (low confidence); the paper's loop simply ends there.
* The final position is the winning tile's centre ((tx + 1/2) t, (ty + 1/2) t)
  (mode "tile"). Mode "centroid" returns instead the multiplicity-weighted mean
  of the exact coordinates of the candidates whose tiles lie in the winning
  tile's circle (the "weighted 2-D centroid" variant). Mode "softmax" returns
  sum_i p_i xy_i with p = softmax(-d_i / tau) over the window's candidates.
"""
from __future__ import annotations

import math

import numpy as np

STATUS_OK = 0
STATUS_LOW_CONFIDENCE = 1


def _snap(v: float) -> float:
    r = float(round(v))
    return r if abs(v - r) <= 1e-9 * max(1.0, abs(v)) else v


def circle_r2_limit(radius_m: float, tile_m: float) -> int:
    """Largest integer squared tile offset inside the tolerance circle."""
    rt = _snap(radius_m / tile_m)
    return int(math.floor(_snap(rt * rt)))


def tile_of(x: float, y: float, tile_m: float):
    return int(math.floor(x / tile_m)), int(math.floor(y / tile_m))


def aggregate_details(cand_idx, xy, dist=None, tile_m=0.30, top_c=10, radius_m=3.0,
                      toler_pct=20, mode="tile", tau=None) -> dict:
    """Algorithm 2 on one window's candidates; returns every intermediate."""
    cand = [int(c) for c in np.asarray(cand_idx).reshape(-1)]
    dvals = None if dist is None else [float(v) for v in np.asarray(dist).reshape(-1)]
    keep = [i for i, c in enumerate(cand) if c >= 0]
    if not keep:
        raise ValueError("window has no candidates")
    C = len(keep)
    # Initialization: row -> floor-plan coordinates -> tile (geo-referenced table).
    pts = [(float(xy[cand[i]][0]), float(xy[cand[i]][1])) for i in keep]
    tiles = [tile_of(x, y, tile_m) for x, y in pts]
    # Step 2: 2-D binning into locationDistriArray.
    counts: dict = {}
    for t in tiles:
        counts[t] = counts.get(t, 0) + 1
    # Steps 5-6: rank tiles by count (descending), ties by (ty, tx); take TopC.
    ranked = sorted(counts.keys(), key=lambda t: (-counts[t], t[1], t[0]))
    n_top = min(int(top_c), len(ranked))
    r2max = circle_r2_limit(radius_m, tile_m)

    def circle(t0):
        return sum(c for t, c in counts.items()
                   if (t[0] - t0[0]) ** 2 + (t[1] - t0[1]) ** 2 <= r2max)

    # Step 7: first TopC tile whose tolerance circle holds > tolerPer of C.
    circles = []
    win = None
    for r in range(n_top):
        cs = circle(ranked[r])
        circles.append(cs)
        if 100 * cs > int(toler_pct) * C:
            win = r
            break
    status = STATUS_OK if win is not None else STATUS_LOW_CONFIDENCE
    best = ranked[win if win is not None else 0]
    if mode == "tile":
        pos = ((best[0] + 0.5) * tile_m, (best[1] + 0.5) * tile_m)
    elif mode == "centroid":
        sel = [p for p, t in zip(pts, tiles)
               if (t[0] - best[0]) ** 2 + (t[1] - best[1]) ** 2 <= r2max]
        pos = (math.fsum(p[0] for p in sel) / len(sel), math.fsum(p[1] for p in sel) / len(sel))
    elif mode == "softmax":
        if dvals is None or tau is None:
            raise ValueError("softmax mode needs distances and tau")
        logits = [-dvals[i] / tau for i in keep]
        mx = max(logits)
        e = [math.exp(v - mx) for v in logits]
        z = math.fsum(e)
        pos = (math.fsum(ei * p[0] for ei, p in zip(e, pts)) / z,
               math.fsum(ei * p[1] for ei, p in zip(e, pts)) / z)
        status = STATUS_OK
    else:
        raise ValueError(f"unknown mode {mode!r}")
    return dict(pos=pos, status=status, C=C, counts=counts, ranked=ranked[:n_top],
                circles=circles, winner=best, r2max=r2max)


def aggregate_2d(cand_idx, xy, dist=None, **kw):
    """Final position (x, y) and status of one window (Algorithm 2)."""
    d = aggregate_details(cand_idx, xy, dist, **kw)
    return d["pos"][0], d["pos"][1], d["status"]


def aggregate_windows(cands, xy, dists=None, **kw):
    """Algorithm 2 on every window; returns xy (nw, 2) float64 and status (nw,)."""
    out = np.empty((len(cands), 2), dtype=np.float64)
    st = np.empty(len(cands), dtype=np.int32)
    for w, c in enumerate(cands):
        x, y, s = aggregate_2d(c, xy, None if dists is None else dists[w], **kw)
        out[w] = (x, y)
        st[w] = s
    return out, st
