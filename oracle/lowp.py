"""Oracle for the low-precision form: per-vector BF16 / FP8-e4m3 quantisation,
low-precision scores, widened shortlist, exact re-rank.

TEST INFRASTRUCTURE ONLY -- imported by tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the library.

This form is not in the paper (which scores FP features directly, §3.1); it
is the build's precision variant, so the oracle states its steps:

1. Per database row i: scale s_i = amax_i / QMAX in binary32 (QMAX = 448 for
   e4m3, the largest finite e4m3 value; 1 for BF16; s_i = 1 when amax_i = 0),
   and code x^_ij = round_to_format(x_ij / s_i) with the divide in binary32,
   round to nearest even, saturating at +-QMAX. The queries of one batch share
   one scale s_Q: the smallest power of two >= (max over the batch of |q_j|) /
   QMAX (that divide in binary32; at least 2^-126; 1 for an all-zero batch),
   codes q^_j = round_to_format(q_j / s_Q) (an exact divide). Because s_Q is a
   power of two, s_Q q^ does not depend on which batch a query came in (as long
   as no code falls below the format's normal range). (A quantised code is an
   integer decision, so it is taken in binary32 as the kernel takes it.)
2. Score of row i for query q (FP64 here):
   ||q||^2 + s_i^2 ||x^_i||^2 - 2 s_q s_i (q^ . x^_i), i.e. the expansion of
   ||q - x||^2 with both vectors replaced by their quantised forms except for
   ||q||^2, which does not change the order.
3. Shortlist: the ``width`` smallest scores, ties by row.
4. Re-rank: exact squared distance of the FP32 query to the FP32 rows of the
   shortlist; the ``k`` smallest by (distance, row).
"""
from __future__ import annotations

import numpy as np

from .retrieval import sq_dist, top_n

QMAX = {"bf16": 1.0, "e4m3": 448.0}


def round_bf16(v) -> np.ndarray:
    """binary32 -> bfloat16 (round to nearest, ties to even), returned as float32."""
    v = np.ascontiguousarray(v, dtype=np.float32)
    u = v.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) >> np.uint64(16) << np.uint64(16)
    return (u & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)


def round_e4m3(v) -> np.ndarray:
    """binary32 -> FP8 e4m3 (OCP 'fn': bias 7, no infinities, max 448), RNE and
    saturation to +-448, returned as float32.

    Normal values 2^e (1 + m/8), e in [-6, 8]; subnormals m/8 * 2^-6, so the
    grid step is 2^(e-3) at and above 2^-6 and 2^-9 below it.
    """
    v = np.asarray(v, dtype=np.float32).astype(np.float64)
    a = np.abs(v)
    _, ex = np.frexp(a)                      # a = f 2^ex, f in [0.5, 1)
    e = np.maximum(ex - 1, -6)               # binade exponent, clamped at the subnormal range
    step = np.ldexp(1.0, e - 3)
    q = np.rint(a / step) * step             # rint: ties to even
    q = np.minimum(q, 448.0)
    return (np.sign(v) * q).astype(np.float32)


def quantize_rows(X, fmt: str):
    """Per-row scale s (float32 (n,)) and codes (float32 (n, D), exactly representable
    in ``fmt``) following step 1."""
    X = np.asarray(X, dtype=np.float32)
    amax = np.abs(X).max(axis=1)
    qmax = np.float32(QMAX[fmt])
    s = np.where(amax > 0, amax / qmax, np.float32(1.0)).astype(np.float32)
    v = (X / s[:, None]).astype(np.float32)
    codes = round_bf16(v) if fmt == "bf16" else round_e4m3(v)
    return s, codes


def batch_scale(Q, fmt: str) -> np.float32:
    """The shared power-of-two query scale s_Q of step 1."""
    amax = np.float32(np.abs(np.asarray(Q, dtype=np.float32)).max()) if np.size(Q) else np.float32(0.0)
    if amax == 0:
        return np.float32(1.0)
    x = max(float(amax / np.float32(QMAX[fmt])), 2.0 ** -126)  # binary32 divide, then exact in binary64
    f, e = np.frexp(x)                                          # x = f 2^e, f in [0.5, 1)
    return np.float32(np.ldexp(1.0, int(e) - 1) if f == 0.5 else np.ldexp(1.0, int(e)))


def quantize_queries(Q, fmt: str, scale=None):
    """Shared scale s_Q (float32) and codes (float32 (nq, D), exactly representable in
    ``fmt``) of a query batch following step 1; ``scale`` overrides s_Q (the scale
    of the batch a query was served in)."""
    Q = np.atleast_2d(np.asarray(Q, dtype=np.float32))
    s = batch_scale(Q, fmt) if scale is None else np.float32(scale)
    v = (Q / s).astype(np.float32)
    codes = round_bf16(v) if fmt == "bf16" else round_e4m3(v)
    return s, codes


def lowp_scores(q, s_q, q_code, s_rows, codes) -> np.ndarray:
    """Step 2 in FP64 for one query against every row."""
    q64 = np.asarray(q, dtype=np.float64)
    qc = np.asarray(q_code, dtype=np.float64)
    c = np.asarray(codes, dtype=np.float64)
    s = np.asarray(s_rows, dtype=np.float64)
    norms = s * s * (c * c).sum(axis=1)
    return q64 @ q64 + norms - 2.0 * float(s_q) * s * (c @ qc)


def lowp_topk(Q, X, fmt: str, width: int, k: int, codes=None, s_rows=None, q_scale=None):
    """Steps 1-4 for every query of the batch Q (``q_scale``: the batch's s_Q when Q
    is part of a larger batch). Returns idx (nq, k), dist (nq, k) FP64 and the
    shortlist rows (nq, width) in score order."""
    Q = np.atleast_2d(np.asarray(Q, dtype=np.float32))
    X = np.asarray(X, dtype=np.float32)
    if codes is None:
        s_rows, codes = quantize_rows(X, fmt)
    s_Q, q_codes = quantize_queries(Q, fmt, q_scale)
    rows = np.arange(X.shape[0], dtype=np.int64)
    idx = np.empty((Q.shape[0], k), dtype=np.int64)
    dist = np.empty((Q.shape[0], k), dtype=np.float64)
    short = np.empty((Q.shape[0], width), dtype=np.int64)
    for i in range(Q.shape[0]):
        sc = lowp_scores(Q[i], s_Q, q_codes[i], s_rows, codes)
        sl, _ = top_n(sc, rows, width)
        short[i] = sl
        valid = sl[sl >= 0]
        idx[i], dist[i] = top_n(sq_dist(Q[i], X[valid]), valid, k)
    return idx, dist, short
