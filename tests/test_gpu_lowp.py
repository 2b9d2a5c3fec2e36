"""Low-precision form (BF16 / FP8-e4m3 codes with per-row scales, tensor-core
scores, fused top-W shortlist, FP32 re-rank) against the FP64 oracle of the
same heuristic, and recall@k against exhaustive search."""
import numpy as np
import pytest

import synth
from oracle import lowp as olowp
from oracle import retrieval as oret
from tests.parity import check_list

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FMT = {"bf16": ("bf16", 1), "fp8": ("e4m3", 2)}


@pytest.fixture(scope="module")
def lhr():
    import paper_2006_08861_gb300 as m
    return m


def _shortlist_separated(q, X, fmt, W, s_rows, codes, s_Q):
    """The oracle's W-th and (W+1)-th scores differ by more than the FP32
    accumulation error of the tensor-core score (so both sides shortlist the
    same rows). s_Q: the shared scale of the batch the query was served in."""
    _, qc = olowp.quantize_queries(q[None], fmt, s_Q)
    sc = np.sort(olowp.lowp_scores(q, s_Q, qc[0], s_rows, codes))
    if W >= sc.size:
        return True
    scale = float(q.astype(np.float64) @ q) + float(np.max(s_rows.astype(np.float64) ** 2 * (codes.astype(np.float64) ** 2).sum(1)))
    return sc[W] - sc[W - 1] > 1e-5 * scale


@pytest.mark.parametrize("fmt_name", ["bf16", "fp8"])
@pytest.mark.parametrize("n,dim,nq,W,k", [
    (1000, 128, 130, 64, 10),     # two query blocks, ragged query block
    (5003, 256, 40, 64, 20),      # ragged last tile, several chunks
    (700, 128, 3, 32, 32),        # shortlist of 32, k = 32
    (3000, 256, 129, 128, 20),    # widest shortlist
])
def test_against_oracle(lhr, fmt_name, n, dim, nq, W, k):
    fmt, bit = FMT[fmt_name]
    rng = np.random.default_rng(n + nq + W)
    X = rng.standard_normal((n, dim)).astype(np.float32)
    Q = (X[rng.integers(0, n, nq)] + 0.3 * rng.standard_normal((nq, dim))).astype(np.float32)
    db = lhr.lhr_build_db(X, np.zeros((n, 2)), lowp=bit)
    idx, dist = lhr.lhr_query(db, torch.from_numpy(Q).cuda(), k, score=fmt_name, rerank_width=W)
    torch.cuda.synchronize()
    assert lhr.lhr_db_error(db) == 0
    gi, gd = idx.cpu().numpy()[:, 0], dist.cpu().numpy()[:, 0]
    s_rows, codes = olowp.quantize_rows(X, fmt)
    s_Q = olowp.batch_scale(Q, fmt)
    o_idx, o_dist, _ = olowp.lowp_topk(Q, X, fmt, W, min(k + 1, W), codes=codes, s_rows=s_rows)
    checked = 0
    for qi in range(nq):
        if not _shortlist_separated(Q[qi], X, fmt, W, s_rows, codes, s_Q):
            continue
        check_list(Q[qi], X, gi[qi], gd[qi], o_idx[qi], o_dist[qi], k, where=f"{fmt_name} q{qi}")
        checked += 1
    assert checked >= int(0.9 * nq)


@pytest.mark.parametrize("fmt_name", ["bf16", "fp8"])
def test_sampled_threshold_path_against_oracle(lhr, fmt_name):
    # 300,000 rows: large enough for the pilot sample (every 64th row), so the
    # shortlist comes from the thresholded main pass. Query 0 is copied into
    # most rows off the sample grid: its candidate count overflows the buffer
    # and the exact per-chunk fallback must give the same answer.
    fmt, bit = FMT[fmt_name]
    rng = np.random.default_rng(31)
    n, dim, nq, W, k = 300_000, 128, 130, 64, 10
    X = rng.standard_normal((n, dim)).astype(np.float32)
    Q = (X[rng.integers(0, n, nq)] + 0.3 * rng.standard_normal((nq, dim))).astype(np.float32)
    dup = np.arange(100, 200_000)
    dup = dup[dup % 64 != 0]
    X[dup] = X[5]
    Q[0] = X[5]
    db = lhr.lhr_build_db(X, np.zeros((n, 2)), lowp=bit)
    idx, dist = lhr.lhr_query(db, torch.from_numpy(Q).cuda(), k, score=fmt_name, rerank_width=W)
    torch.cuda.synchronize()
    assert lhr.lhr_db_error(db) == 0
    gi, gd = idx.cpu().numpy()[:, 0], dist.cpu().numpy()[:, 0]
    s_rows, codes = olowp.quantize_rows(X, fmt)
    s_Q = olowp.batch_scale(Q, fmt)
    sample = np.random.default_rng(32).choice(np.arange(1, nq), size=24, replace=False)
    for qi in [0] + sample.tolist():
        if qi and not _shortlist_separated(Q[qi], X, fmt, W, s_rows, codes, s_Q):
            continue
        o_idx, o_dist, _ = olowp.lowp_topk(Q[qi:qi + 1], X, fmt, W, k + 1, codes=codes, s_rows=s_rows,
                                           q_scale=s_Q)
        check_list(Q[qi], X, gi[qi], gd[qi], o_idx[0], o_dist[0], k, where=f"{fmt_name} q{qi}")
    # query 0: exact copies at distance 0, lowest rows first
    assert gi[0, 0] == 5 and np.all(gd[0] == 0.0)


def test_fp8_main_pass_dense_candidates(lhr):
    # FP8 at D = 256 over a sampled database (the thresholded main pass), 300
    # queries: a ragged last 256-query block. Rows 1000 .. 2199 are near-copies
    # of row 7 that query 1 sits on: about 1,200 candidates inside one row
    # chunk, far past what the epilogue stages per query before a flush, all
    # below the candidate buffer's 2,048.
    fmt, bit = FMT["fp8"]
    rng = np.random.default_rng(77)
    n, dim, nq, W, k = 300_000, 256, 300, 64, 20
    X = rng.standard_normal((n, dim)).astype(np.float32)
    X[1000:2200] = X[7] + 0.02 * rng.standard_normal((1200, dim)).astype(np.float32)
    Q = (X[rng.integers(0, n, nq)] + 0.3 * rng.standard_normal((nq, dim))).astype(np.float32)
    Q[1] = X[7] + 0.01 * rng.standard_normal(dim).astype(np.float32)
    db = lhr.lhr_build_db(X, np.zeros((n, 2)), lowp=bit)
    idx, dist = lhr.lhr_query(db, torch.from_numpy(Q).cuda(), k, score="fp8", rerank_width=W)
    torch.cuda.synchronize()
    assert lhr.lhr_db_error(db) == 0
    gi, gd = idx.cpu().numpy()[:, 0], dist.cpu().numpy()[:, 0]
    s_rows, codes = olowp.quantize_rows(X, fmt)
    s_Q = olowp.batch_scale(Q, fmt)
    sample = [1, 255, 256, 299] + np.random.default_rng(78).choice(np.arange(2, nq), size=16, replace=False).tolist()
    checked = 0
    for qi in sample:
        if not _shortlist_separated(Q[qi], X, fmt, W, s_rows, codes, s_Q):
            continue
        o_idx, o_dist, _ = olowp.lowp_topk(Q[qi:qi + 1], X, fmt, W, k + 1, codes=codes, s_rows=s_rows,
                                           q_scale=s_Q)
        check_list(Q[qi], X, gi[qi], gd[qi], o_idx[0], o_dist[0], k, where=f"fp8 q{qi}")
        checked += 1
    assert checked >= len(sample) // 2
    # query 1's answers are among the near-copies of row 7
    assert np.all((gi[1] == 7) | ((gi[1] >= 1000) & (gi[1] < 2200)))


def test_width_equal_to_database_is_exhaustive(lhr):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((100, 128)).astype(np.float32)
    Q = rng.standard_normal((5, 128)).astype(np.float32)
    db = lhr.lhr_build_db(X, np.zeros((100, 2)), lowp=3)
    for f in ("bf16", "fp8"):
        idx, dist = lhr.lhr_query(db, torch.from_numpy(Q).cuda(), 20, score=f, rerank_width=128)
        ei, ed = lhr.lhr_query(db, torch.from_numpy(Q).cuda(), 20)
        torch.cuda.synchronize()
        assert np.array_equal(idx.cpu().numpy(), ei.cpu().numpy())
        assert np.array_equal(dist.cpu().numpy(), ed.cpu().numpy())


def test_invalid_low_precision_requests(lhr):
    X = np.zeros((10, 128), np.float32)
    db = lhr.lhr_build_db(X, np.zeros((10, 2)), lowp=1)
    q = torch.zeros((1, 128), device="cuda")
    with pytest.raises(lhr.LhrError):
        lhr.lhr_query(db, q, 5, score="fp8")        # no FP8 copy
    with pytest.raises(lhr.LhrError):
        lhr.lhr_query(db, q, 5, score="bf16", rerank_width=4)  # W < k
    with pytest.raises(lhr.LhrError):
        lhr.lhr_build_db(np.zeros((10, 96), np.float32), np.zeros((10, 2)), lowp=2)  # D % 128 for FP8


def _oracle_topk_threads(Q, X, k):
    """The FP64 oracle's exhaustive top-k of each query, one query per host thread."""
    import concurrent.futures as cf
    import os

    def one(i):
        return oret.exhaustive_topk(Q[i:i + 1], X, k)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        res = list(ex.map(one, range(Q.shape[0])))
    return np.stack([r[0][0, 0] for r in res]), np.stack([r[1][0, 0] for r in res])


def test_precision_configuration_recall_and_positions(lhr):
    # N = 2,000,000, D = 256, Q = 1,024 frames (noise 0.05), top-64 shortlist,
    # FP32 re-rank to k = 20, then Algorithm 2 on each frame's 20 candidates.
    # Every query: recall@20 of the BF16 / FP8 forms against the exhaustive FP32
    # scan, and their final positions against the FP32 form's. Sampled queries
    # (64, one per host thread): every form against the FP64 oracle, lists by
    # the parity rule and positions against Algorithm 2 on the oracle's list.
    from oracle import aggregate as oagg
    cfg = synth.CONFIGS["precision"]
    k = cfg["k"]
    db = synth.make_database(cfg["n"], cfg["dim"], seed=synth.db_seed(cfg["index"]))
    q, rows, _ = synth.make_point_queries(db, cfg["nq"], seed=synth.query_seed(cfg["index"]))
    h = lhr.lhr_build_db(db.feats, db.xy, lowp=3)
    qt = torch.from_numpy(q).cuda()
    offs = torch.arange(0, cfg["nq"] * k + 1, k, dtype=torch.int32, device="cuda")
    results = {}
    for f in ("f32", "bf16", "fp8"):
        kw = {} if f == "f32" else dict(score=f, rerank_width=cfg["rerank_width"])
        li, ld = lhr.lhr_query(h, qt, k, **kw)
        xy, st = lhr.lhr_aggregate_2d(h, li.view(-1), offs, mode="tile")
        torch.cuda.synchronize()
        results[f] = (li.cpu().numpy()[:, 0], ld.cpu().numpy()[:, 0], xy.cpu().numpy(), st.cpu().numpy())
    assert lhr.lhr_db_error(h) == 0
    ex, _, ex_xy, ex_st = results["f32"]
    for f in ("bf16", "fp8"):
        li, ld, xy, st = results[f]
        same_set = np.array([set(li[i]) == set(ex[i]) for i in range(cfg["nq"])])
        recall = np.mean([len(set(li[i]) & set(ex[i])) / k for i in range(cfg["nq"])])
        assert recall >= 0.999, (f, recall)
        assert np.mean(li[:, 0] == ex[:, 0]) >= 0.999, f
        # identical candidate sets give identical positions (Algorithm 2 reads the set only)
        dev_m = np.max(np.abs(xy - ex_xy), axis=1)
        assert np.all(dev_m[same_set] <= 1e-9) and np.all(st[same_set] == ex_st[same_set]), f
        assert np.mean((dev_m <= 1e-3) & (st == ex_st)) >= 0.999, (f, np.mean(dev_m <= 1e-3))
    sample = np.random.default_rng(5).choice(cfg["nq"], size=64, replace=False)
    o_idx, o_dist = _oracle_topk_threads(q[sample], db.feats, k + 1)
    o_xy, o_st = oagg.aggregate_windows([o_idx[j, :k] for j in range(sample.size)], db.xy, mode="tile")
    hits = {f: 0 for f in results}
    for j, qi in enumerate(sample):
        sep = o_dist[j, k] - o_dist[j, k - 1] > 1e-4 * o_dist[j, k - 1]
        for f, (li, ld, xy, st) in results.items():
            same = set(li[qi]) == set(o_idx[j, :k])
            hits[f] += len(set(li[qi]) & set(o_idx[j, :k]))
            if f == "f32" or same:
                check_list(q[qi], db.feats, li[qi], ld[qi], o_idx[j], o_dist[j], k, where=f"{f} q{qi}")
            if sep and (f == "f32" or same):
                assert np.max(np.abs(xy[qi] - o_xy[j])) <= 1e-3 and st[qi] == o_st[j], (f, qi)
    for f in ("bf16", "fp8"):
        assert hits[f] / (k * sample.size) >= 0.995, (f, hits[f])
    h.close()


@pytest.mark.parametrize("fmt_name", ["bf16", "fp8"])
def test_batch_outlier_keeps_recall(lhr, fmt_name):
    # The queries of one batch share one power-of-two scale, set by the batch's
    # largest |q_j|. One query 100x larger than the rest pushes the others'
    # codes 100x down (FP8: partly into the e4m3 subnormal range): the others'
    # recall@20 against the exhaustive FP32 scan must stay >= 0.999, and the
    # outlier's own list must equal the scan's.
    fmt, bit = FMT[fmt_name]
    cfg = synth.CONFIGS["precision"]
    k = cfg["k"]
    db = synth.make_database(300_000, 256, seed=4242)
    q, _, _ = synth.make_point_queries(db, 256, seed=4343)
    q[17] *= np.float32(100.0)
    h = lhr.lhr_build_db(db.feats, db.xy, lowp=bit)
    qt = torch.from_numpy(q).cuda()
    ei, ed = lhr.lhr_query(h, qt, k)
    li, ld = lhr.lhr_query(h, qt, k, score=fmt_name, rerank_width=cfg["rerank_width"])
    torch.cuda.synchronize()
    assert lhr.lhr_db_error(h) == 0
    ex, got = ei.cpu().numpy()[:, 0], li.cpu().numpy()[:, 0]
    rest = [i for i in range(q.shape[0]) if i != 17]
    recall = np.mean([len(set(got[i]) & set(ex[i])) / k for i in rest])
    assert recall >= 0.999, recall
    assert set(got[17]) == set(ex[17])
    # the batch scale really moved: the outlier's amax sets it (the oracle's statement of the scale)
    assert olowp.batch_scale(q, fmt) >= 64 * olowp.batch_scale(np.delete(q, 17, axis=0), fmt)
    h.close()
