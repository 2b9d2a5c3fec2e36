"""Python binding of liblhr.so (include/lhr.h): argument marshalling only.

Every step of retrieval and aggregation runs in the library's CUDA kernels;
this module passes pointers, sizes and torch's current CUDA stream. PyTorch
supplies device memory and streams. There is no CPU fallback: if liblhr.so
is missing or fails to load, import raises.

Names follow the C ABI: lhr_build_db, lhr_query, lhr_query_window,
lhr_aggregate_2d, lhr_db_error, lhr_last_error.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblhr.so")

LHR_OK = 0
LHR_WARN_LOW_CONFIDENCE = 1
LHR_ERR_INVALID_ARG = -1
LHR_ERR_CUDA = -2
LHR_ERR_OOM = -3
LHR_ERR_TIMEOUT = -4
LHR_ERR_UNSUPPORTED = -5

LHR_F32, LHR_BF16, LHR_FP8_E4M3 = 0, 1, 2
LHR_AGG_TILE, LHR_AGG_TILE_CENTROID, LHR_AGG_SOFTMAX = 0, 1, 2
LHR_LOWP_BF16, LHR_LOWP_FP8 = 1, 2

_SCORE = {"f32": LHR_F32, "bf16": LHR_BF16, "fp8": LHR_FP8_E4M3, "e4m3": LHR_FP8_E4M3}
_MODE = {"tile": LHR_AGG_TILE, "centroid": LHR_AGG_TILE_CENTROID, "softmax": LHR_AGG_SOFTMAX}


class DbConfig(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("coarse_dim", ctypes.c_int32), ("lowp", ctypes.c_uint32),
                ("reserved", ctypes.c_int32), ("tile_m", ctypes.c_double)]


class QueryParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("shortlist", ctypes.c_int32), ("score", ctypes.c_int32),
                ("rerank_width", ctypes.c_int32)]


class AggParams(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("top_c", ctypes.c_int32), ("radius_m", ctypes.c_double),
                ("toler_pct", ctypes.c_int32), ("tau", ctypes.c_float)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int32), ("max_window", ctypes.c_int32), ("ring_frames", ctypes.c_int32),
                ("max_batch_frames", ctypes.c_int32), ("n_lanes", ctypes.c_int32), ("k", ctypes.c_int32),
                ("shortlist", ctypes.c_int32), ("score", ctypes.c_int32), ("mem_budget_bytes", ctypes.c_int64),
                ("agg", AggParams), ("rerank_width", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ring_mem_bytes", ctypes.c_int64)]


class ServerResult(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_int64), ("stream_id", ctypes.c_int32), ("m", ctypes.c_int32),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_int32), ("xy", ctypes.c_double * 2),
                ("latency_us", ctypes.c_double)]


class LhrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lhr status {status}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(paper_2006_08861_gb300.build_ext.build())")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "lhr_build_db": [P, P, P, I64, ctypes.POINTER(DbConfig), P, ctypes.POINTER(P)],
        "lhr_free_db": [P],
        "lhr_db_info": [P, ctypes.POINTER(I64), ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32)],
        "lhr_query": [P, P, I32, ctypes.POINTER(QueryParams), P, P, P],
        "lhr_query_window": [P, P, P, I32, I32, ctypes.POINTER(QueryParams), ctypes.POINTER(AggParams),
                             P, P, P, P, P],
        "lhr_aggregate_2d": [P, P, P, I64, P, I32, ctypes.POINTER(AggParams), P, P, P],
        "lhr_db_error": [P, ctypes.POINTER(I32), P],
        "lhr_query_static": [P, P, I32, I32, P, P, P],
        "lhr_query_weighted": [P, P, I32, I32, P, P, P, P],
        "lhr_soft_forward": [P, P, P, I32, I32, I32, P, P, P, P, P, P, P],
        "lhr_soft_backward": [P, P, P, I32, I32, I32, P, P, P, P, P, P, P, P, P, P, P],
        "lhr_loc_mse": [P, P, I32, P, P, P, P],
        "lhr_server_create": [P, ctypes.POINTER(ServerConfig), ctypes.POINTER(P)],
        "lhr_server_submit": [P, I32, P, I32, I64],
        "lhr_server_poll": [P, ctypes.POINTER(ServerResult), I32, ctypes.POINTER(I32), I32],
        "lhr_server_drain": [P, I32],
        "lhr_server_open_stream": [P, ctypes.POINTER(I32)],
        "lhr_server_close_stream": [P, I32, I32],
        "lhr_server_destroy": [P],
        "lhr_profile_enable": [I32],
        "lhr_profile_read": [ctypes.c_char_p, ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_double), I32],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.lhr_last_error.argtypes = []
    lib.lhr_last_error.restype = ctypes.c_char_p
    return lib


_lib = _load()


def lhr_last_error() -> str:
    return _lib.lhr_last_error().decode()


def _check(st: int):
    if st < 0:
        raise LhrError(st, lhr_last_error())
    return st


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())


def _dev_tensor(x, dtype, name):
    torch = _torch()
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype != dtype or not x.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    return x


def _out_tensor(x, dtype, shape, device, name):
    """A caller-supplied output: contiguous, on `device`, of this dtype and exact shape (the
    library writes that many elements through its pointer)."""
    torch = _torch()
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.device != device:
        raise TypeError(f"{name} must be a CUDA tensor on {device}")
    if x.dtype != dtype or not x.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    if tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(x.shape)}")
    return x


def _frames(db, x, name):
    """Query frames: a contiguous float32 CUDA tensor of shape (nq, db.dim)."""
    torch = _torch()
    x = _dev_tensor(x, torch.float32, name)
    if x.dim() != 2 or x.shape[1] != db.dim:
        raise ValueError(f"{name} must have shape (n, {db.dim}), got {tuple(x.shape)}")
    return x


class Database:
    """Owns an lhr_db handle (freed with the object)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        n, d, dc, ns = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.lhr_db_info(self._h, ctypes.byref(n), ctypes.byref(d), ctypes.byref(dc), ctypes.byref(ns)))
        self.n, self.dim, self.coarse_dim, self.n_subspaces = n.value, d.value, dc.value, ns.value

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.lhr_free_db(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_or_dev(x, np_dtype, torch_dtype, name):
    torch = _torch()
    if isinstance(x, torch.Tensor):
        if x.dtype != torch_dtype or not x.is_contiguous():
            raise TypeError(f"{name} must be a contiguous {torch_dtype} tensor")
        return x
    a = np.ascontiguousarray(x, dtype=np_dtype)
    return a


def lhr_build_db(feats, xy, subspace=None, coarse_dim: int = 0, lowp: int = 0, tile_m: float = 0.30,
                 stream=None) -> Database:
    """Builds a device database from features (n x D float32) and floor-plan
    coordinates (n x 2 float64), host arrays or CUDA tensors."""
    torch = _torch()
    f = _host_or_dev(feats, np.float32, torch.float32, "feats")
    c = _host_or_dev(xy, np.float64, torch.float64, "xy")
    s = None if subspace is None else _host_or_dev(subspace, np.int32, torch.int32, "subspace")
    n, dim = f.shape
    cfg = DbConfig(dim, coarse_dim, lowp, 0, tile_m)
    h = ctypes.c_void_p()
    _check(_lib.lhr_build_db(_ptr(f), _ptr(c), _ptr(s), n, ctypes.byref(cfg), _stream(stream), ctypes.byref(h)))
    return Database(h)


def query_params(k: int, shortlist: int = 0, score: str = "f32", rerank_width: int = 64) -> QueryParams:
    return QueryParams(k, shortlist, _SCORE[score], rerank_width)


def agg_params(mode: str = "tile", top_c: int = 10, radius_m: float = 3.0, toler_pct: int = 20,
               tau: float = 1.0) -> AggParams:
    return AggParams(_MODE[mode], top_c, radius_m, toler_pct, tau)


def lhr_query(db: Database, q, k: int, shortlist: int = 0, score: str = "f32", rerank_width: int = 64,
              out=None, stream=None):
    """Top-k rows per query frame: returns (idx int64 [nq, n_s, k], dist float32 [nq, n_s, k])."""
    torch = _torch()
    q = _frames(db, q, "q")
    nq = q.shape[0]
    if out is None:
        idx = torch.empty((nq, db.n_subspaces, k), dtype=torch.int64, device=q.device)
        dist = torch.empty((nq, db.n_subspaces, k), dtype=torch.float32, device=q.device)
    else:
        idx = _out_tensor(out[0], torch.int64, (nq, db.n_subspaces, k), q.device, "idx")
        dist = _out_tensor(out[1], torch.float32, (nq, db.n_subspaces, k), q.device, "dist")
    p = query_params(k, shortlist, score, rerank_width)
    _check(_lib.lhr_query(db.handle, _ptr(q), nq, ctypes.byref(p), _ptr(idx), _ptr(dist), _stream(stream)))
    return idx, dist


def lhr_query_static(db: Database, q, k: int, out, stream=None):
    """Exhaustive FP32 top-k that allocates nothing: scratch is the library's
    fixed 4 MiB device array, shared by every call (serialize overlapping
    calls). ``out`` = (idx int64 [nq, n_s, k], dist float32 [nq, n_s, k]),
    preallocated by the caller."""
    torch = _torch()
    q = _frames(db, q, "q")
    nq = q.shape[0]
    idx = _out_tensor(out[0], torch.int64, (nq, db.n_subspaces, k), q.device, "idx")
    dist = _out_tensor(out[1], torch.float32, (nq, db.n_subspaces, k), q.device, "dist")
    _check(_lib.lhr_query_static(db.handle, _ptr(q), q.shape[0], k, _ptr(idx), _ptr(dist), _stream(stream)))
    return idx, dist


def lhr_query_window(db: Database, frames, offsets, k: int, shortlist: int = 0, score: str = "f32",
                     rerank_width: int = 64, mode: str = "tile", top_c: int = 10, radius_m: float = 3.0,
                     toler_pct: int = 20, tau: float = 1.0, out=None, stream=None):
    """Retrieval for every frame, then Algorithm 2 per window.
    Returns (idx, dist, xy float64 [nw, 2], status int32 [nw])."""
    torch = _torch()
    frames = _frames(db, frames, "frames")
    offsets = _dev_tensor(offsets, torch.int32, "offsets")
    if offsets.dim() != 1 or offsets.shape[0] < 2:
        raise ValueError("offsets must be a 1-D tensor of nw + 1 >= 2 entries")
    W, nw = frames.shape[0], offsets.shape[0] - 1
    dev = frames.device
    if out is None:
        idx = torch.empty((W, db.n_subspaces, k), dtype=torch.int64, device=dev)
        dist = torch.empty((W, db.n_subspaces, k), dtype=torch.float32, device=dev)
        xy = torch.empty((nw, 2), dtype=torch.float64, device=dev)
        status = torch.empty((nw,), dtype=torch.int32, device=dev)
    else:
        idx = _out_tensor(out[0], torch.int64, (W, db.n_subspaces, k), dev, "idx")
        dist = _out_tensor(out[1], torch.float32, (W, db.n_subspaces, k), dev, "dist")
        xy = _out_tensor(out[2], torch.float64, (nw, 2), dev, "xy")
        status = _out_tensor(out[3], torch.int32, (nw,), dev, "status")
    p = query_params(k, shortlist, score, rerank_width)
    a = agg_params(mode, top_c, radius_m, toler_pct, tau)
    _check(_lib.lhr_query_window(db.handle, _ptr(frames), _ptr(offsets), W, nw, ctypes.byref(p), ctypes.byref(a),
                                 _ptr(idx), _ptr(dist), _ptr(xy), _ptr(status), _stream(stream)))
    return idx, dist, xy, status


def lhr_aggregate_2d(db: Database, idx, cand_offsets, dist=None, mode: str = "tile", top_c: int = 10,
                     radius_m: float = 3.0, toler_pct: int = 20, tau: float = 1.0, out=None, stream=None):
    """Algorithm 2 on caller candidates. Returns (xy float64 [nw, 2], status int32 [nw])."""
    torch = _torch()
    idx = _dev_tensor(idx, torch.int64, "idx")
    cand_offsets = _dev_tensor(cand_offsets, torch.int32, "cand_offsets")
    if dist is not None:
        dist = _dev_tensor(dist, torch.float32, "dist")
    if cand_offsets.dim() != 1 or cand_offsets.shape[0] < 2:
        raise ValueError("cand_offsets must be a 1-D tensor of nw + 1 >= 2 entries")
    if dist is not None and dist.numel() != idx.numel():
        raise ValueError("dist must hold one distance per candidate")
    nw = cand_offsets.shape[0] - 1
    if out is None:
        xy = torch.empty((nw, 2), dtype=torch.float64, device=idx.device)
        status = torch.empty((nw,), dtype=torch.int32, device=idx.device)
    else:
        xy = _out_tensor(out[0], torch.float64, (nw, 2), idx.device, "xy")
        status = _out_tensor(out[1], torch.int32, (nw,), idx.device, "status")
    a = agg_params(mode, top_c, radius_m, toler_pct, tau)
    _check(_lib.lhr_aggregate_2d(db.handle, _ptr(idx), _ptr(dist), idx.numel(), _ptr(cand_offsets), nw,
                                 ctypes.byref(a), _ptr(xy), _ptr(status), _stream(stream)))
    return xy, status


def lhr_profile_enable(on: bool) -> None:
    """Per-kernel CUDA-event timing of every later launch (process-wide)."""
    _check(_lib.lhr_profile_enable(1 if on else 0))


def lhr_profile_read(kernel: str | None = None, reset: bool = True):
    """(launches, total device ms) of profiled kernels whose name contains `kernel`."""
    n, ms = ctypes.c_int64(), ctypes.c_double()
    _check(_lib.lhr_profile_read(None if kernel is None else kernel.encode(), ctypes.byref(n), ctypes.byref(ms),
                                 1 if reset else 0))
    return n.value, ms.value


def lhr_db_error(db: Database, stream=None) -> int:
    """Reads and clears the database's device error word (synchronizes)."""
    e = ctypes.c_int32()
    _check(_lib.lhr_db_error(db.handle, ctypes.byref(e), _stream(stream)))
    return e.value


# ------------------------------------------------------------------ soft retrieval
def lhr_query_weighted(db: Database, q, k: int, w, out=None, stream=None):
    """Exhaustive top-k by the weighted distance sum_j w_j (q_j - x_j)^2:
    (idx int64 [nq, n_s, k], dist float32 [nq, n_s, k])."""
    torch = _torch()
    q = _frames(db, q, "q")
    w = _out_tensor(w, torch.float32, (db.dim,), q.device, "w")
    nq = q.shape[0]
    if out is None:
        idx = torch.empty((nq, db.n_subspaces, k), dtype=torch.int64, device=q.device)
        dist = torch.empty((nq, db.n_subspaces, k), dtype=torch.float32, device=q.device)
    else:
        idx = _out_tensor(out[0], torch.int64, (nq, db.n_subspaces, k), q.device, "idx")
        dist = _out_tensor(out[1], torch.float32, (nq, db.n_subspaces, k), q.device, "dist")
    _check(_lib.lhr_query_weighted(db.handle, _ptr(q), nq, k, _ptr(w), _ptr(idx), _ptr(dist), _stream(stream)))
    return idx, dist


def lhr_soft_forward(db: Database, frames, offsets, k: int, w, tau, stream=None):
    """Selection by the weighted distance, then the window softmax:
    (idx [W, n_s, k], dist [W, n_s, k], p float64 [W, n_s, k], yhat float64 [nw, 2])."""
    torch = _torch()
    frames = _dev_tensor(frames, torch.float32, "frames")
    offsets = _dev_tensor(offsets, torch.int32, "offsets")
    w = _dev_tensor(w, torch.float32, "w")
    tau = _dev_tensor(tau, torch.float32, "tau")
    W, nw = frames.shape[0], offsets.shape[0] - 1
    dev = frames.device
    idx = torch.empty((W, db.n_subspaces, k), dtype=torch.int64, device=dev)
    dist = torch.empty((W, db.n_subspaces, k), dtype=torch.float32, device=dev)
    p = torch.empty((W, db.n_subspaces, k), dtype=torch.float64, device=dev)
    yhat = torch.empty((nw, 2), dtype=torch.float64, device=dev)
    _check(_lib.lhr_soft_forward(db.handle, _ptr(frames), _ptr(offsets), W, nw, k, _ptr(w), _ptr(tau), _ptr(idx),
                                 _ptr(dist), _ptr(p), _ptr(yhat), _stream(stream)))
    return idx, dist, p, yhat


def lhr_soft_backward(db: Database, frames, offsets, k: int, w, tau, idx, dist, p, yhat, g_yhat, stream=None):
    """Gradients (dq float32 [W, D], dw float32 [D], dtau float32 [1]) given dL/dyhat."""
    torch = _torch()
    frames = _dev_tensor(frames, torch.float32, "frames")
    g_yhat = _dev_tensor(g_yhat, torch.float64, "g_yhat")
    W, nw = frames.shape[0], offsets.shape[0] - 1
    dq = torch.empty_like(frames)
    dw = torch.empty_like(w)
    dtau = torch.empty((1,), dtype=torch.float32, device=frames.device)
    _check(_lib.lhr_soft_backward(db.handle, _ptr(frames), _ptr(offsets), W, nw, k, _ptr(w), _ptr(tau), _ptr(idx),
                                  _ptr(dist), _ptr(p), _ptr(yhat), _ptr(g_yhat), _ptr(dq), _ptr(dw), _ptr(dtau),
                                  _stream(stream)))
    return dq, dw, dtau


def lhr_loc_mse(yhat, y, scale=None, loss=True, grad=False, stream=None):
    """L = mean_b ||yhat_b - y_b||^2 (float64 [1]) and/or scale * dL/dyhat (float64 [nw, 2])."""
    torch = _torch()
    yhat = _dev_tensor(yhat, torch.float64, "yhat")
    y = _dev_tensor(y, torch.float64, "y")
    nw = yhat.shape[0]
    lo = torch.empty((1,), dtype=torch.float64, device=yhat.device) if loss else None
    gr = torch.empty_like(yhat) if grad else None
    sc = None if scale is None else _dev_tensor(scale, torch.float64, "scale")
    _check(_lib.lhr_loc_mse(_ptr(yhat), _ptr(y), nw, _ptr(sc), _ptr(lo), _ptr(gr), _stream(stream)))
    return lo, gr


def _make_autograd():
    torch = _torch()

    class SoftRetrieval(torch.autograd.Function):
        """y^ = soft_retrieval(frames, w, tau): forward and backward are the
        library's kernels (lhr_soft_forward / lhr_soft_backward)."""

        @staticmethod
        def forward(ctx, frames, w, tau, db, offsets, k):
            frames, w, tau = frames.contiguous(), w.contiguous(), tau.contiguous()
            idx, dist, p, yhat = lhr_soft_forward(db, frames, offsets, k, w, tau)
            ctx.save_for_backward(frames, w, tau, offsets, idx, dist, p, yhat)
            ctx.db, ctx.k = db, k
            ctx.tau_shape = tau.shape
            return yhat

        @staticmethod
        def backward(ctx, g):
            frames, w, tau, offsets, idx, dist, p, yhat = ctx.saved_tensors
            dq, dw, dtau = lhr_soft_backward(ctx.db, frames, offsets, ctx.k, w, tau, idx, dist, p, yhat,
                                             g.contiguous().to(torch.float64))
            return dq, dw, dtau.reshape(ctx.tau_shape), None, None, None

    class LocMSE(torch.autograd.Function):
        """L = mean_b ||y^_b - y_b||^2 (lhr_loc_mse)."""

        @staticmethod
        def forward(ctx, yhat, y):
            yhat, y = yhat.contiguous(), y.contiguous()
            loss, _ = lhr_loc_mse(yhat, y, loss=True, grad=False)
            ctx.save_for_backward(yhat, y)
            return loss.reshape(())

        @staticmethod
        def backward(ctx, g):
            yhat, y = ctx.saved_tensors
            _, grad = lhr_loc_mse(yhat, y, scale=g.reshape(1).to(torch.float64).contiguous(), loss=False, grad=True)
            return grad, None

    return SoftRetrieval, LocMSE


_AUTOGRAD = None


def soft_retrieval(db: Database, frames, offsets, w, tau, k: int):
    """Differentiable window positions y^ (float64 [nw, 2]) w.r.t. frames, w and tau."""
    global _AUTOGRAD
    if _AUTOGRAD is None:
        _AUTOGRAD = _make_autograd()
    return _AUTOGRAD[0].apply(frames, w, tau, db, offsets, k)


def loc_mse(yhat, y):
    """Differentiable mean squared 2-D error of the window positions."""
    global _AUTOGRAD
    if _AUTOGRAD is None:
        _AUTOGRAD = _make_autograd()
    return _AUTOGRAD[1].apply(yhat, y)


# ------------------------------------------------------------------ serving
class Server:
    """Continuous-batching request loop over one database (lhr_server_*).

    submit() queues one frame of a user stream (a float32 host array of D
    values) and optionally asks for the position of that stream's last m
    frames; poll() returns finished windows as dicts (request_id, stream_id,
    m, status, xy, latency_us)."""

    def __init__(self, db: Database, n_streams: int, max_window: int, k: int, shortlist: int = 0,
                 ring_frames: int | None = None, max_batch_frames: int = 64, n_lanes: int = 2,
                 mem_budget_bytes: int = 1 << 30, mode: str = "tile", top_c: int = 10, radius_m: float = 3.0,
                 toler_pct: int = 20, tau: float = 1.0, score: str = "f32", rerank_width: int = 64,
                 ring_mem_bytes: int = 0):
        self.db = db
        ring = ring_frames if ring_frames is not None else 2 * max_window + max_batch_frames
        cfg = ServerConfig(n_streams, max_window, ring, max_batch_frames, n_lanes, k, shortlist, _SCORE[score],
                           mem_budget_bytes, agg_params(mode, top_c, radius_m, toler_pct, tau), rerank_width, 0,
                           ring_mem_bytes)
        h = ctypes.c_void_p()
        _check(_lib.lhr_server_create(db.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._buf = (ServerResult * 4096)()

    def submit(self, stream_id: int, frame, window_m: int = 0, request_id: int = -1):
        f = np.ascontiguousarray(frame, dtype=np.float32)
        if f.size != self.db.dim:
            raise ValueError(f"frame must hold {self.db.dim} values")
        _check(_lib.lhr_server_submit(self._h, stream_id, ctypes.c_void_p(f.ctypes.data), window_m, request_id))

    def poll(self, wait_ms: int = 0, max_results: int = 4096):
        n = ctypes.c_int32()
        _check(_lib.lhr_server_poll(self._h, self._buf, min(max_results, 4096), ctypes.byref(n), wait_ms))
        return [dict(request_id=r.request_id, stream_id=r.stream_id, m=r.m, status=r.status,
                     xy=(r.xy[0], r.xy[1]), latency_us=r.latency_us) for r in self._buf[:n.value]]

    def drain(self, timeout_ms: int = 60000):
        _check(_lib.lhr_server_drain(self._h, timeout_ms))

    def open_stream(self) -> int:
        """Admits a new stream if a device ring is free (LhrError LHR_ERR_OOM otherwise)."""
        sid = ctypes.c_int32()
        _check(_lib.lhr_server_open_stream(self._h, ctypes.byref(sid)))
        return sid.value

    def close_stream(self, stream_id: int, timeout_ms: int = 60000):
        """Closes a stream; its ring returns once its frames are done."""
        _check(_lib.lhr_server_close_stream(self._h, stream_id, timeout_ms))

    def close(self):
        if getattr(self, "_h", None):
            _lib.lhr_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lhr_server_create(db: Database, **cfg) -> Server:
    return Server(db, **cfg)


def lhr_server_submit(server: Server, stream_id: int, frame, window_m: int = 0, request_id: int = -1):
    server.submit(stream_id, frame, window_m, request_id)


def lhr_server_poll(server: Server, wait_ms: int = 0, max_results: int = 4096):
    return server.poll(wait_ms, max_results)


def lhr_server_drain(server: Server, timeout_ms: int = 60000):
    server.drain(timeout_ms)


def lhr_server_open_stream(server: Server) -> int:
    return server.open_stream()


def lhr_server_close_stream(server: Server, stream_id: int, timeout_ms: int = 60000):
    server.close_stream(stream_id, timeout_ms)


def lhr_server_destroy(server: Server):
    server.close()
