"""Synthetic floor plan, feature field, database and query frames.

Recipe (stands in for the paper's one-floor, five-path capture of §4):

* Path: a serpentine polyline of parallel corridors ``corridor_len`` metres
  long and ``corridor_gap`` metres apart (the paper models a floor with
  parallel capture paths, §4), joined at alternating ends by connectors of
  length ``corridor_gap``. Database locations sit every ``spacing`` metres of
  arc length. Coordinates are >= ``margin`` > 0.
* Feature field: each of the D feature dimensions is an independent zero-mean,
  unit-variance Gaussian random field over (x, y) with squared-exponential
  correlation length ``ell`` (2 m). It is realised with R shared random Fourier
  features, f(p) = sqrt(2/R) cos(p @ omega.T + b) @ A with omega ~ N(0, I/ell^2),
  b ~ U[0, 2 pi) and A ~ N(0, 1), so it can be evaluated at any off-grid
  position (query frames are 0.3 m apart, the database 0.5 m).
* Scene aliasing: a fraction of database locations is given the feature of a
  uniformly chosen location at least ``alias_min_dist`` metres away plus
  N(0, alias_sigma^2) per dimension (the paper's scene-similarity problem,
  §3.2).
* Queries: single frames are a database row's feature plus N(0, sigma^2);
  windows are m consecutive frames ``frame_spacing`` apart along the path,
  each the field at that position plus N(0, sigma^2); the window's reference
  position is frame floor(m/2) (the centred q_m of §3.1).

Randomness comes from numpy's PCG64 ``default_rng`` with the seeds in
``CONFIGS`` (database 1000 + i, queries 2000 + i).
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

# Synthetic workloads (sizes of the five configurations the build targets).
CONFIGS = {
    "tiny": dict(index=0, n=2_000, dim=128, nq=16, k=10, m=1),
    "hierarchical": dict(index=1, n=100_000, dim=256, coarse_dim=32, shortlist=512, k=20, m=5),
    "precision": dict(index=2, n=2_000_000, dim=256, nq=1024, k=20, rerank_width=64),
    "differentiation": dict(index=3, n=200_000, dim=256, nw=256, m=5, k=32),
    "serving": dict(index=4, n=1_000_000, dim=256, streams=64, fps=15.0, m_lo=3, m_hi=10, k=20),
}


def db_seed(index: int) -> int:
    return 1000 + index


def query_seed(index: int) -> int:
    return 2000 + index


def path_length(n: int, spacing: float = 0.5) -> float:
    return spacing * max(n - 1, 0)


def path_positions(s: np.ndarray, corridor_len: float = 100.0, corridor_gap: float = 3.0,
                   margin: float = 1.0) -> np.ndarray:
    """(x, y) in metres of the points at arc lengths ``s`` along the serpentine."""
    s = np.asarray(s, dtype=np.float64)
    period = corridor_len + corridor_gap
    c = np.floor(s / period)
    r = s - c * period
    east = (c.astype(np.int64) % 2) == 0
    on_corr = r < corridor_len
    x = np.where(on_corr,
                 np.where(east, margin + r, margin + corridor_len - r),
                 np.where(east, margin + corridor_len, margin))
    y = margin + c * corridor_gap + np.where(on_corr, 0.0, r - corridor_len)
    return np.stack([x, y], axis=1)


@dataclass
class FeatureField:
    """Smooth Gaussian random field R^2 -> R^D (random Fourier features)."""
    omega: np.ndarray  # (R, 2) float32
    b: np.ndarray      # (R,) float32
    A: np.ndarray      # (R, D) float32

    @staticmethod
    def make(dim: int, rng: np.random.Generator, ell: float = 2.0, n_basis: int = 256) -> "FeatureField":
        omega = (rng.standard_normal((n_basis, 2)) / ell).astype(np.float32)
        b = rng.uniform(0.0, 2.0 * math.pi, n_basis).astype(np.float32)
        A = rng.standard_normal((n_basis, dim)).astype(np.float32)
        return FeatureField(omega, b, A)

    @property
    def dim(self) -> int:
        return self.A.shape[1]

    def __call__(self, pos: np.ndarray, chunk: int = 1 << 15) -> np.ndarray:
        pos = np.asarray(pos, dtype=np.float32)
        out = np.empty((pos.shape[0], self.dim), dtype=np.float32)
        scale = np.float32(math.sqrt(2.0 / self.omega.shape[0]))
        om = self.omega.astype(np.float64)
        b = self.b.astype(np.float64)

        def one(s):
            p = pos[s:s + chunk].astype(np.float64)
            # phase in binary64 (the products of binary32 values are exact), rounded once to binary32
            phase = (p[:, 0:1] * om[:, 0] + p[:, 1:2] * om[:, 1] + b).astype(np.float32)
            np.cos(phase, out=phase)
            phase *= scale
            np.matmul(phase, self.A, out=out[s:s + chunk])

        starts = range(0, pos.shape[0], chunk)
        if pos.shape[0] <= chunk:
            for s in starts:
                one(s)
        else:
            # chunks are independent and write disjoint rows: the bytes do not depend on the thread count
            import concurrent.futures as cf
            with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
                list(ex.map(one, starts))
        return out


@dataclass
class Database:
    feats: np.ndarray         # (n, D) float32, row-major
    xy: np.ndarray            # (n, 2) float64, floor-plan metres
    arc: np.ndarray           # (n,) float64 arc length of each location
    aliased: np.ndarray       # (n,) bool: feature copied from a distant location
    alias_src: np.ndarray     # (n,) int64 source row of the copy, -1 if none
    field: FeatureField
    spacing: float
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.feats.shape[0]

    @property
    def dim(self) -> int:
        return self.feats.shape[1]


def make_database(n: int, dim: int, seed: int, spacing: float = 0.5, alias_frac: float = 0.10,
                  alias_min_dist: float = 10.0, alias_sigma: float = 0.01,
                  ell: float = 2.0) -> Database:
    rng = np.random.default_rng(seed)
    fld = FeatureField.make(dim, rng, ell=ell)
    arc = spacing * np.arange(n, dtype=np.float64)
    xy = path_positions(arc)
    feats = fld(xy)
    n_alias = int(round(alias_frac * n))
    aliased = np.zeros(n, dtype=bool)
    alias_src = np.full(n, -1, dtype=np.int64)
    if n_alias > 0 and n > 1:
        rows = rng.choice(n, size=n_alias, replace=False)
        src = rng.integers(0, n, size=n_alias)
        # Redraw sources closer than alias_min_dist (Euclidean, floor plan).
        for _ in range(64):
            bad = np.hypot(*(xy[src] - xy[rows]).T) < alias_min_dist
            if not bad.any():
                break
            src[bad] = rng.integers(0, n, size=int(bad.sum()))
        ok = np.hypot(*(xy[src] - xy[rows]).T) >= alias_min_dist
        rows, src = rows[ok], src[ok]
        noise = rng.standard_normal((rows.size, dim)).astype(np.float32) * np.float32(alias_sigma)
        # feats[src] is gathered before any row is overwritten: every copy is of the field's own value
        feats[rows] = feats[src] + noise
        aliased[rows] = True
        alias_src[rows] = src
    return Database(feats=np.ascontiguousarray(feats), xy=xy, arc=arc, aliased=aliased,
                    alias_src=alias_src, field=fld, spacing=spacing,
                    meta=dict(seed=seed, alias_frac=alias_frac, alias_sigma=alias_sigma, ell=ell))


def make_point_queries(db: Database, nq: int, seed: int, sigma: float = 0.05):
    """Single-frame queries: a database row's feature + N(0, sigma^2) noise.

    Returns (q float32 (nq, D), true_row int64 (nq,), true_xy float64 (nq, 2)).
    """
    rng = np.random.default_rng(seed)
    rows = rng.choice(db.n, size=nq, replace=nq > db.n)
    noise = rng.standard_normal((nq, db.dim)).astype(np.float32) * np.float32(sigma)
    q = db.feats[rows] + noise
    return np.ascontiguousarray(q), rows.astype(np.int64), db.xy[rows].copy()


@dataclass
class Windows:
    frames: np.ndarray    # (W, D) float32, frames of all windows back to back
    offsets: np.ndarray   # (nw + 1,) int32 CSR offsets of each window's frames
    true_xy: np.ndarray   # (nw, 2) float64 position of each window's reference frame
    frame_xy: np.ndarray  # (W, 2) float64 position of every frame

    @property
    def nw(self) -> int:
        return self.offsets.size - 1

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)


def make_windows(db: Database, nw: int, m, seed: int, sigma: float = 0.05,
                 frame_spacing: float = 0.3) -> Windows:
    """Query windows of consecutive frames along the path.

    ``m`` is an int (every window has m frames) or a (lo, hi) pair, in which
    case each window's length is uniform in lo..hi inclusive.
    """
    rng = np.random.default_rng(seed)
    if isinstance(m, (tuple, list)):
        lens = rng.integers(int(m[0]), int(m[1]) + 1, size=nw)
    else:
        lens = np.full(nw, int(m), dtype=np.int64)
    offsets = np.zeros(nw + 1, dtype=np.int32)
    offsets[1:] = np.cumsum(lens)
    total = path_length(db.n, db.spacing)
    s_all = np.empty(int(offsets[-1]), dtype=np.float64)
    true_xy = np.empty((nw, 2), dtype=np.float64)
    for w in range(nw):
        span = frame_spacing * (lens[w] - 1)
        s0 = rng.uniform(0.0, max(total - span, 0.0))
        s = s0 + frame_spacing * np.arange(lens[w], dtype=np.float64)
        s_all[offsets[w]:offsets[w + 1]] = s
        true_xy[w] = path_positions(s[lens[w] // 2:lens[w] // 2 + 1])[0]
    frame_xy = path_positions(s_all)
    feats = db.field(frame_xy)
    feats += rng.standard_normal(feats.shape).astype(np.float32) * np.float32(sigma)
    return Windows(frames=np.ascontiguousarray(feats), offsets=offsets, true_xy=true_xy,
                   frame_xy=frame_xy)
