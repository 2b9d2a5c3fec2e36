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


def test_precision_configuration_recall(lhr):
    # N = 2,000,000, D = 256, Q = 1,024 frames (noise 0.05), top-64 shortlist,
    # FP32 re-rank to k = 20: recall@20 against the exhaustive FP32 scan (which
    # is parity-tested against the oracle) on every query, and against the FP64
    # oracle itself on sampled queries.
    cfg = synth.CONFIGS["precision"]
    db = synth.make_database(cfg["n"], cfg["dim"], seed=1002)
    q, rows, _ = synth.make_point_queries(db, cfg["nq"], seed=2002)
    h = lhr.lhr_build_db(db.feats, db.xy, lowp=3)
    qt = torch.from_numpy(q).cuda()
    ei, ed = lhr.lhr_query(h, qt, cfg["k"])
    results = {}
    for f in ("bf16", "fp8"):
        li, ld = lhr.lhr_query(h, qt, cfg["k"], score=f, rerank_width=cfg["rerank_width"])
        torch.cuda.synchronize()
        results[f] = (li.cpu().numpy()[:, 0], ld.cpu().numpy()[:, 0])
    ex = ei.cpu().numpy()[:, 0]
    for f, (li, ld) in results.items():
        recall = np.mean([len(set(li[i]) & set(ex[i])) / cfg["k"] for i in range(cfg["nq"])])
        assert recall >= 0.999, (f, recall)
        assert np.mean(li[:, 0] == ex[:, 0]) >= 0.999, f
    for qi in (0, 511):
        o_idx, o_dist = oret.exhaustive_topk(q[qi:qi + 1], db.feats, cfg["k"] + 1)
        for f, (li, ld) in results.items():
            check_list(q[qi], db.feats, li[qi], ld[qi], o_idx[0, 0], o_dist[0, 0], cfg["k"], where=f"{f} q{qi}")
    assert lhr.lhr_db_error(h) == 0
    h.close()
