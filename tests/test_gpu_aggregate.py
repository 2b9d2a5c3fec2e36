"""Algorithm 2 on the GPU (lhr_aggregate_2d and the aggregation step of
lhr_query_window) against the hand-derived cases and the FP64 oracle."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import aggregate as oagg
from oracle import retrieval as oret
from tests.parity import XY_ATOL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "aggregation_cases.json")


@pytest.fixture(scope="module")
def lhr():
    import paper_2006_08861_gb300 as m
    return m


def _db_for_xy(lhr, xy):
    n = len(xy)
    return lhr.lhr_build_db(np.zeros((n, 4), np.float32), np.asarray(xy, np.float64))


def _agg(lhr, db, cands, mode, dists=None, **kw):
    flat = np.concatenate([np.asarray(c, np.int64) for c in cands])
    offs = np.concatenate([[0], np.cumsum([len(c) for c in cands])]).astype(np.int32)
    idx = torch.from_numpy(flat).cuda()
    d = None if dists is None else torch.from_numpy(np.concatenate(dists).astype(np.float32)).cuda()
    xy, st = lhr.lhr_aggregate_2d(db, idx, torch.from_numpy(offs).cuda(), dist=d, mode=mode, **kw)
    torch.cuda.synchronize()
    return xy.cpu().numpy(), st.cpu().numpy()


def test_golden_cases(lhr):
    g = json.load(open(GOLDEN))
    for case in g["cases"]:
        kw = dict(top_c=case.get("top_c", g["defaults"]["top_c"]), radius_m=g["defaults"]["radius_m"],
                  toler_pct=g["defaults"]["toler_pct"])
        db = _db_for_xy(lhr, case["xy"])
        exp = case["expect"]
        xy, st = _agg(lhr, db, [case["cand"]], "tile", **kw)
        t = g["defaults"]["tile_m"]
        assert st[0] == exp["status"], case["name"]
        assert xy[0].tolist() == [(exp["tile"][0] + 0.5) * t, (exp["tile"][1] + 0.5) * t], case["name"]
        xy, st = _agg(lhr, db, [case["cand"]], "centroid", **kw)
        assert st[0] == exp["status"], case["name"]
        assert np.max(np.abs(xy[0] - exp["centroid"])) <= 1e-9, case["name"]


@pytest.mark.parametrize("mode", ["tile", "centroid", "softmax"])
def test_random_windows_against_oracle(lhr, mode):
    rng = np.random.default_rng(11)
    n = 500
    xy = rng.uniform(0, 30, size=(n, 2))
    xy[:50] = rng.uniform(10, 12, size=(50, 2))  # a dense area
    db = _db_for_xy(lhr, xy)
    cands, dists = [], []
    for w in range(40):
        # sizes on both sides of 1024 (the kernel's warp and block paths)
        c = rng.integers(0, n, size=int(rng.integers(1, 3000)))
        if w % 3 == 0:
            c[: len(c) // 2] = rng.integers(0, 50, size=len(c) // 2)
        if w % 7 == 0:
            c[::5] = -1  # padding rows are skipped
            c[0] = 3
        cands.append(c)
        dists.append(rng.uniform(0.1, 5.0, size=len(c)).astype(np.float32))  # both sides get FP32 inputs
    gxy, gst = _agg(lhr, db, cands, mode, dists=dists if mode == "softmax" else None, tau=0.7)
    # the C ABI's tau is a float: the oracle gets the same float32 value
    oxy, ost = oagg.aggregate_windows(cands, xy, dists=dists if mode == "softmax" else None, mode=mode,
                                      tau=float(np.float32(0.7)))
    assert np.array_equal(gst, ost)
    tol = 0.0 if mode == "tile" else 1e-9
    assert np.max(np.abs(gxy - oxy)) <= tol


@pytest.mark.parametrize("mode", ["tile", "centroid", "softmax"])
def test_small_windows_against_oracle(lhr, mode):
    # windows of 1..128 slots (the register path: 32, 64 and 128 slots per
    # warp), with padding rows and repeated rows
    rng = np.random.default_rng(13)
    n = 400
    xy = rng.uniform(0, 20, size=(n, 2))
    xy[:40] = rng.uniform(5, 6, size=(40, 2))
    db = _db_for_xy(lhr, xy)
    cands, dists = [], []
    for size in [1, 2, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129]:
        c = rng.integers(0, n, size=size)
        if size > 2:
            c[::4] = rng.integers(0, 40, size=len(c[::4]))
            c[1::7] = -1
        cands.append(c)
        dists.append(rng.uniform(0.1, 5.0, size=size).astype(np.float32))
    gxy, gst = _agg(lhr, db, cands, mode, dists=dists if mode == "softmax" else None, tau=0.7)
    oxy, ost = oagg.aggregate_windows(cands, xy, dists=dists if mode == "softmax" else None, mode=mode,
                                      tau=float(np.float32(0.7)))
    assert np.array_equal(gst, ost)
    tol = 0.0 if mode == "tile" else 1e-9
    assert np.max(np.abs(gxy - oxy)) <= tol


def test_parameters_top_c_radius_toler(lhr):
    rng = np.random.default_rng(12)
    xy = rng.uniform(0, 8, size=(300, 2))
    db = _db_for_xy(lhr, xy)
    cands = [rng.integers(0, 300, size=200) for _ in range(10)]
    for kw in (dict(top_c=1, radius_m=0.0, toler_pct=1), dict(top_c=25, radius_m=1.0, toler_pct=50),
               dict(top_c=3, radius_m=2.2, toler_pct=0), dict(top_c=10, radius_m=0.31, toler_pct=5)):
        gxy, gst = _agg(lhr, db, cands, "centroid", **kw)
        oxy, ost = oagg.aggregate_windows(cands, xy, mode="centroid", **kw)
        assert np.array_equal(gst, ost), kw
        assert np.max(np.abs(gxy - oxy)) <= 1e-9, kw


def test_invalid_windows_get_error_status(lhr):
    xy = np.array([[1.0, 1.0], [2.0, 2.0]])
    db = _db_for_xy(lhr, xy)
    idx = torch.tensor([0, 1, -1, -1, 1], dtype=torch.int64, device="cuda")
    # window 0 empty, window 1 only padding, window 2 fine, window 3 past the end
    offs = torch.tensor([0, 0, 2, 4, 9], dtype=torch.int32, device="cuda")
    offs2 = torch.tensor([0, 0, 2, 4, 5], dtype=torch.int32, device="cuda")
    xyo, st = lhr.lhr_aggregate_2d(db, idx, offs2)
    torch.cuda.synchronize()
    assert st.cpu().tolist() == [lhr.LHR_ERR_INVALID_ARG, 0, lhr.LHR_ERR_INVALID_ARG, 0]
    xyo, st = lhr.lhr_aggregate_2d(db, idx, offs)
    torch.cuda.synchronize()
    assert st.cpu().tolist()[3] == lhr.LHR_ERR_INVALID_ARG
    # a row outside the table is skipped and recorded in the error word
    bad = torch.tensor([0, 7], dtype=torch.int64, device="cuda")
    xyo, st = lhr.lhr_aggregate_2d(db, bad, torch.tensor([0, 2], dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    assert st.cpu().tolist() == [0]
    assert lhr.lhr_db_error(db) == lhr.LHR_ERR_INVALID_ARG
    assert lhr.lhr_db_error(db) == 0


def test_window_pipeline_tiny_configuration(lhr):
    # N = 2,000, D = 128, one-frame windows, k = 10, weighted 2-D centroid
    db = synth.make_database(2000, 128, seed=1000)
    q, rows, txy = synth.make_point_queries(db, 16, seed=2000)
    h = lhr.lhr_build_db(db.feats, db.xy)
    offs = torch.arange(17, dtype=torch.int32, device="cuda")
    idx, dist, xy, st = lhr.lhr_query_window(h, torch.from_numpy(q).cuda(), offs, 10, mode="centroid")
    torch.cuda.synchronize()
    gi = idx.cpu().numpy()[:, 0]
    o_idx, _ = oret.exhaustive_topk(q, db.feats, 10)
    cands = oret.window_candidates(gi, np.arange(17))
    oxy, ost = oagg.aggregate_windows(cands, db.xy, mode="centroid")
    assert np.array_equal(st.cpu().numpy(), ost)
    assert np.max(np.abs(xy.cpu().numpy() - oxy)) <= XY_ATOL
    # the oracle's own candidates give the same answer wherever the lists agree
    same = np.all(gi == o_idx[:, 0], axis=1)
    o2, _ = oagg.aggregate_windows(oret.window_candidates(o_idx[:, 0], np.arange(17)), db.xy, mode="centroid")
    assert np.max(np.abs(xy.cpu().numpy()[same] - o2[same]), initial=0.0) <= XY_ATOL
    assert same.mean() >= 0.8


def test_window_pipeline_uneven_lengths(lhr):
    db = synth.make_database(30_000, 128, seed=41)
    win = synth.make_windows(db, 25, (3, 10), seed=42)
    h = lhr.lhr_build_db(db.feats, db.xy)
    idx, dist, xy, st = lhr.lhr_query_window(h, torch.from_numpy(win.frames).cuda(),
                                             torch.from_numpy(win.offsets).cuda(), 20, mode="tile")
    torch.cuda.synchronize()
    gi = idx.cpu().numpy()[:, 0]
    oxy, ost = oagg.aggregate_windows(oret.window_candidates(gi, win.offsets), db.xy, mode="tile")
    assert np.array_equal(st.cpu().numpy(), ost)
    assert np.max(np.abs(xy.cpu().numpy() - oxy)) <= XY_ATOL
