"""Oracle for the soft (differentiable) retrieval form and its FP64 gradients.

TEST INFRASTRUCTURE ONLY -- imported by tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the library.

Not in the paper: it is the build's differentiable relaxation of §3.1's
retrieval and §3.2's aggregation. Per window b of frames f:

* each frame's top-k rows are chosen by the weighted squared distance
  d_i = sum_j w_j (q_fj - x_ij)^2 (the choice itself is held fixed);
* logits l_i = -d_i / tau over the window's m*k candidates (one joint
  softmax), p = softmax(l), y^_b = sum_i p_i xy_i;
* loss L = (1/B) sum_b ||y^_b - y_b||^2.

Analytic gradients (g_b = 2 (y^_b - y_b) / B):
  dL/dl_i   = p_i g_b . (xy_i - y^_b)
  dL/dd_i   = -(1/tau) dL/dl_i
  dL/dtau   = sum_i dL/dl_i d_i / tau^2
  dL/dw_j   = sum_i dL/dd_i (q_f(i)j - x_ij)^2
  dL/dq_fj  = sum_{i in f} dL/dd_i 2 w_j (q_fj - x_ij)
"""
from __future__ import annotations

import numpy as np

from .retrieval import sq_dist, top_n


def select(frames, offsets, X, w, k):
    """Per-frame top-k rows by weighted distance: idx (W, k)."""
    frames = np.asarray(frames)
    rows = np.arange(np.asarray(X).shape[0], dtype=np.int64)
    out = np.empty((frames.shape[0], k), dtype=np.int64)
    for f in range(frames.shape[0]):
        out[f], _ = top_n(sq_dist(frames[f], X, w), rows, k)
    return out


def forward_backward(frames, offsets, X, xy, y_true, w, tau, idx=None, k=None):
    """Loss and gradients (dq (W, D), dw (D,), dtau) in FP64."""
    frames = np.asarray(frames, dtype=np.float64)
    X = np.asarray(X)
    xy = np.asarray(xy, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    offsets = np.asarray(offsets, dtype=np.int64)
    B = offsets.size - 1
    if idx is None:
        idx = select(frames, offsets, X, w, k)
    loss = 0.0
    dq = np.zeros_like(frames)
    dw = np.zeros_like(w)
    dtau = 0.0
    yhat_all = np.empty((B, 2))
    for b in range(B):
        fr = np.arange(offsets[b], offsets[b + 1])
        cand = idx[fr].reshape(-1)
        owner = np.repeat(fr, idx.shape[1])
        diff = frames[owner] - X[cand].astype(np.float64)        # (C, D)
        d = (w * diff * diff).sum(axis=1)
        logit = -d / tau
        p = np.exp(logit - logit.max())
        p /= p.sum()
        yhat = p @ xy[cand]
        yhat_all[b] = yhat
        r = yhat - y_true[b]
        loss += r @ r / B
        g = 2.0 * r / B
        dl = p * ((xy[cand] - yhat) @ g)
        dd = -dl / tau
        dtau += float((dl * d).sum()) / (tau * tau)
        dw += (dd[:, None] * diff * diff).sum(axis=0)
        np.add.at(dq, owner, dd[:, None] * 2.0 * w * diff)
    return dict(loss=loss, dq=dq, dw=dw, dtau=dtau, idx=idx, yhat=yhat_all)
