"""Coarse-to-fine retrieval (prefix over every row -> S-row shortlist ->
full re-rank -> top k) against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import aggregate as oagg
from oracle import retrieval as oret
from tests.parity import GAP, XY_ATOL, check_hier_ambiguous, check_list

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lhr():
    import paper_2006_08861_gb300 as m
    return m


def _shortlist_separated(q, X, dc, S):
    d = np.sort(oret.sq_dist(q[:dc], X[:, :dc]))
    return S >= X.shape[0] or (d[S] - d[S - 1]) > GAP * max(d[S - 1], 1e-12)


def test_full_shortlist_equals_exhaustive(lhr):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((600, 64)).astype(np.float32)
    Q = (X[rng.integers(0, 600, 6)] + 0.3 * rng.standard_normal((6, 64))).astype(np.float32)
    db = lhr.lhr_build_db(X, np.zeros((600, 2)), coarse_dim=16)
    q = torch.from_numpy(Q).cuda()
    hi, hd = lhr.lhr_query(db, q, 10, shortlist=600)
    ei, ed = lhr.lhr_query(db, q, 10)
    torch.cuda.synchronize()
    assert np.array_equal(hi.cpu().numpy(), ei.cpu().numpy())
    assert np.array_equal(hd.cpu().numpy(), ed.cpu().numpy())


@pytest.mark.parametrize("n,dim,dc,S,k,nq", [
    (20_000, 64, 16, 256, 10, 5),
    (9_001, 128, 32, 100, 20, 3),
    (3_000, 36, 4, 64, 7, 9),      # prefix of one float4, more than 8 frames
    (5_000, 256, 128, 4096, 32, 2),  # widest prefix, largest shortlist
    (8_000, 128, 64, 500, 32, 6),    # fused path: k = 32 of a 500-row shortlist (warp merges)
    (7_000, 64, 16, 33, 32, 4),      # fused path: shortlist just above k
])
def test_against_oracle(lhr, n, dim, dc, S, k, nq):
    rng = np.random.default_rng(n + S)
    X = rng.standard_normal((n, dim)).astype(np.float32)
    Q = (X[rng.integers(0, n, nq)] + 0.3 * rng.standard_normal((nq, dim))).astype(np.float32)
    db = lhr.lhr_build_db(X, np.zeros((n, 2)), coarse_dim=dc)
    idx, dist = lhr.lhr_query(db, torch.from_numpy(Q).cuda(), k, shortlist=S)
    torch.cuda.synchronize()
    gi, gd = idx.cpu().numpy()[:, 0], dist.cpu().numpy()[:, 0]
    o_idx, o_dist, _ = oret.hierarchical_topk(Q, X, dc, S, k + 1)
    checked = 0
    for qi in range(nq):
        if not _shortlist_separated(Q[qi], X, dc, S):
            continue
        # the oracle's k+1 list comes from the same shortlist
        check_list(Q[qi], X, gi[qi], gd[qi], o_idx[qi], o_dist[qi], k, where=f"q{qi}")
        checked += 1
    assert checked >= nq - 1


def test_boundary_bin_overflow_refines_to_rows(lhr):
    # Every row has the same prefix, so all coarse distances are equal and the
    # shortlist is decided by the row tie rule alone: rows 0..S-1.
    rng = np.random.default_rng(2)
    n, dim, dc, S, k = 12_000, 64, 8, 300, 10
    X = rng.standard_normal((n, dim)).astype(np.float32)
    X[:, :dc] = 0.5
    Q = rng.standard_normal((3, dim)).astype(np.float32)
    db = lhr.lhr_build_db(X, np.zeros((n, 2)), coarse_dim=dc)
    idx, dist = lhr.lhr_query(db, torch.from_numpy(Q).cuda(), k, shortlist=S)
    torch.cuda.synchronize()
    gi = idx.cpu().numpy()[:, 0]
    o_idx, o_dist, short = oret.hierarchical_topk(Q, X, dc, S, k + 1)
    assert np.array_equal(short, np.tile(np.arange(S), (3, 1)))
    for qi in range(3):
        check_list(Q[qi], X, gi[qi], dist.cpu().numpy()[qi, 0], o_idx[qi], o_dist[qi], k)
        assert np.all(gi[qi] < S)


def test_fused_small_requests(lhr):
    # Requests of at most 8 frames take the single-launch fused path: one
    # window of m = 5 frames per call (the building-scale benchmark's call),
    # and one call carrying two windows of 3 and 4 frames.
    cfg = synth.CONFIGS["hierarchical"]
    db = synth.make_database(cfg["n"], cfg["dim"], seed=1001)
    h = lhr.lhr_build_db(db.feats, db.xy, coarse_dim=cfg["coarse_dim"])
    wins = synth.make_windows(db, 4, cfg["m"], seed=2101)
    two = synth.make_windows(db, 2, (3, 4), seed=2102)
    calls = [(wins.frames[wins.offsets[w]:wins.offsets[w + 1]], np.array([0, 5], np.int32)) for w in range(4)]
    calls.append((two.frames, two.offsets))
    for frames, offs in calls:
        idx, dist, xy, st = lhr.lhr_query_window(h, torch.from_numpy(np.ascontiguousarray(frames)).cuda(),
                                                 torch.from_numpy(offs).cuda(), cfg["k"],
                                                 shortlist=cfg["shortlist"], mode="tile")
        torch.cuda.synchronize()
        gi, gd = idx.cpu().numpy()[:, 0], dist.cpu().numpy()[:, 0]
        o_idx, o_dist, _ = oret.hierarchical_topk(frames, db.feats, cfg["coarse_dim"], cfg["shortlist"],
                                                  cfg["k"] + 1)
        for f in range(frames.shape[0]):
            if _shortlist_separated(frames[f], db.feats, cfg["coarse_dim"], cfg["shortlist"]):
                check_list(frames[f], db.feats, gi[f], gd[f], o_idx[f], o_dist[f], cfg["k"], where=f"f{f}")
        o_xy, o_st = oagg.aggregate_windows(oret.window_candidates(gi, offs), db.xy, mode="tile")
        assert np.array_equal(st.cpu().numpy(), o_st)
        assert np.max(np.abs(xy.cpu().numpy() - o_xy)) <= XY_ATOL
    assert lhr.lhr_db_error(h) == 0


def test_hierarchical_configuration_windows(lhr):
    # Building scale: N = 100,000, D = 256, coarse prefix 32, shortlist 512,
    # k = 20, windows of m = 5 frames 0.3 m apart, aggregated in 2-D.
    cfg = synth.CONFIGS["hierarchical"]
    db = synth.make_database(cfg["n"], cfg["dim"], seed=1001)
    win = synth.make_windows(db, 8, cfg["m"], seed=2001)
    h = lhr.lhr_build_db(db.feats, db.xy, coarse_dim=cfg["coarse_dim"])
    frames = torch.from_numpy(win.frames).cuda()
    offs = torch.from_numpy(win.offsets).cuda()
    idx, dist, xy, st = lhr.lhr_query_window(h, frames, offs, cfg["k"], shortlist=cfg["shortlist"],
                                             mode="tile")
    torch.cuda.synchronize()
    gi, gd = idx.cpu().numpy()[:, 0], dist.cpu().numpy()[:, 0]
    o_idx, o_dist, _ = oret.hierarchical_topk(win.frames, db.feats, cfg["coarse_dim"], cfg["shortlist"],
                                              cfg["k"] + 1)
    strict = 0
    for f in range(win.frames.shape[0]):
        if _shortlist_separated(win.frames[f], db.feats, cfg["coarse_dim"], cfg["shortlist"]):
            check_list(win.frames[f], db.feats, gi[f], gd[f], o_idx[f], o_dist[f], cfg["k"], where=f"f{f}")
            strict += 1
        else:
            # the shortlist boundary nearly ties (about a third of the frames at S = 512 of 100,000):
            # the list must still be the exact top k of a valid shortlist
            check_hier_ambiguous(win.frames[f], db.feats, cfg["coarse_dim"], cfg["shortlist"], gi[f], gd[f],
                                 cfg["k"], where=f"f{f}")
    assert strict >= win.frames.shape[0] // 2, strict
    # Algorithm 2 on the GPU's candidates equals the oracle's on the same candidates
    cands = oret.window_candidates(gi, win.offsets)
    o_xy, o_st = oagg.aggregate_windows(cands, db.xy, mode="tile")
    assert np.array_equal(st.cpu().numpy(), o_st)
    assert np.max(np.abs(xy.cpu().numpy() - o_xy)) <= XY_ATOL
    # and the localization is right for most windows (error < 3 m)
    err = np.hypot(*(xy.cpu().numpy() - win.true_xy).T)
    assert np.mean(err < 3.0) >= 0.75
    h.close()


def test_subspaces_coarse_to_fine_papers_experiment_shape(lhr):
    # §4's experiment shape through the coarse-to-fine path: P = 5 paths
    # (subspaces, interleaved in the database so rows are permuted), windows of
    # M = 11 frames, top N = 15 per frame and path: 825 candidates per window,
    # then Algorithm 2. Per frame and path against the FP64 oracle (the
    # coarse-to-fine form run over each subspace alone); positions against
    # Algorithm 2 of the oracle on the same candidates.
    n, dim, dc, S, k, P, M = 30_000, 128, 32, 256, 15, 5, 11
    db = synth.make_database(n, dim, seed=81)
    corridor = np.floor(db.arc / 103.0).astype(np.int64)          # 100 m corridors + 3 m connectors
    sub = (corridor % P).astype(np.int32)
    win = synth.make_windows(db, 3, M, seed=82)
    h = lhr.lhr_build_db(db.feats, db.xy, subspace=sub, coarse_dim=dc)
    assert h.n_subspaces == P
    frames = torch.from_numpy(win.frames).cuda()
    offs = torch.from_numpy(win.offsets).cuda()
    idx, dist, xy, st = lhr.lhr_query_window(h, frames, offs, k, shortlist=S, mode="tile")
    torch.cuda.synchronize()
    assert lhr.lhr_db_error(h) == 0
    gi, gd = idx.cpu().numpy(), dist.cpu().numpy()
    assert gi.shape == (win.frames.shape[0], P, k) and (gi >= 0).all()
    o_idx, o_dist = oret.hierarchical_topk_subspaces(win.frames, db.feats, dc, S, k + 1, sub, P)
    strict = 0
    for s in range(P):
        rows = np.nonzero(sub == s)[0]
        Xs = db.feats[rows]
        pos = {int(r): i for i, r in enumerate(rows)}
        for f in range(win.frames.shape[0]):
            if _shortlist_separated(win.frames[f], Xs, dc, S):
                check_list(win.frames[f], db.feats, gi[f, s], gd[f, s], o_idx[f, s], o_dist[f, s], k, rows=rows,
                           where=f"f{f} s{s}")
                strict += 1
            else:
                assert np.isin(gi[f, s], rows).all()
                check_hier_ambiguous(win.frames[f], Xs, dc, S, np.array([pos[int(r)] for r in gi[f, s]]), gd[f, s],
                                     k, where=f"f{f} s{s}")
    assert strict >= (win.frames.shape[0] * P) // 2, strict
    cands = oret.window_candidates(gi, win.offsets)
    assert all(c.size == 825 for c in cands)   # N x M x P of §4
    o_xy, o_st = oagg.aggregate_windows(cands, db.xy, mode="tile")
    assert np.array_equal(st.cpu().numpy(), o_st)
    assert np.max(np.abs(xy.cpu().numpy() - o_xy)) <= XY_ATOL
    # the shortlist may not exceed a subspace's rows
    with pytest.raises(lhr.LhrError):
        lhr.lhr_query_window(h, frames, offs, k, shortlist=int(np.bincount(sub).min()) + 1)
    h.close()


def test_fused_control_blocks_left_zeroed(lhr):
    # The fused kernel's zero-initialised words (histograms, per-frame
    # counters, grid barrier) live in a per-stream control block that each
    # launch leaves zeroed, in place of a memset before it. Calls in a row on
    # one stream, calls on more streams than there are blocks (the others take
    # scratch and a memset), a captured graph replayed several times, and the
    # two-window form all give the first call's results, bit for bit.
    cfg = synth.CONFIGS["hierarchical"]
    db = synth.make_database(40_000, cfg["dim"], seed=1301)
    h = lhr.lhr_build_db(db.feats, db.xy, coarse_dim=cfg["coarse_dim"])
    win = synth.make_windows(db, 2, (3, 4), seed=1302)
    frames = torch.from_numpy(win.frames).cuda()
    offs = torch.from_numpy(win.offsets).cuda()
    S, k = cfg["shortlist"], cfg["k"]

    def call(stream=None, out=None):
        return lhr.lhr_query_window(h, frames, offs, k, shortlist=S, mode="centroid", stream=stream, out=out)

    ref = [t.clone() for t in call()]
    torch.cuda.synchronize()

    def same(res):
        for a, b in zip(ref, res):
            assert torch.equal(a, b)

    for _ in range(4):
        same(call())
    streams = [torch.cuda.Stream() for _ in range(12)]
    outs = []
    for s in streams:
        with torch.cuda.stream(s):
            outs.append(call(stream=s))
    torch.cuda.synchronize()
    for res in outs:
        same(res)
    for s in streams[:3]:  # again on streams that hold a block
        with torch.cuda.stream(s):
            res = call(stream=s)
        s.synchronize()
        same(res)
    out = [torch.empty_like(t) for t in ref]
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        call(stream=side, out=out)  # warm-up outside the capture
        side.synchronize()
        with torch.cuda.graph(g, stream=side):
            call(stream=side, out=out)
    for _ in range(3):
        for t in out:
            t.zero_()
        g.replay()
        torch.cuda.synchronize()
        same(out)
    assert lhr.lhr_db_error(h) == 0
    # and the first call agrees with the oracle
    o_idx, o_dist, _ = oret.hierarchical_topk(win.frames, db.feats, cfg["coarse_dim"], S, k + 1)
    gi, gd = ref[0].cpu().numpy()[:, 0], ref[1].cpu().numpy()[:, 0]
    checked = 0
    for f in range(win.frames.shape[0]):
        if _shortlist_separated(win.frames[f], db.feats, cfg["coarse_dim"], S):
            check_list(win.frames[f], db.feats, gi[f], gd[f], o_idx[f], o_dist[f], k, where=f"f{f}")
            checked += 1
    assert checked >= 1
    h.close()


@pytest.mark.parametrize("k,m", [(20, (3, 4)), (32, (4, 4)), (32, (3, 5))])
def test_fused_window_draws_against_oracle(lhr, k, m):
    # Algorithm 2 inside the fused launch, with parameters that make the draws
    # run past the first tile or fail (status 1: the first tile is kept):
    # windows of at most 128 candidate slots take the table form, larger ones
    # the sorting form. Positions and statuses against the oracle's Algorithm 2
    # on the same candidates.
    cfg = synth.CONFIGS["hierarchical"]
    db = synth.make_database(30_000, cfg["dim"], seed=1401)
    h = lhr.lhr_build_db(db.feats, db.xy, coarse_dim=cfg["coarse_dim"])
    win = synth.make_windows(db, 2, m, seed=1402 + k)
    frames = torch.from_numpy(win.frames).cuda()
    offs = torch.from_numpy(win.offsets).cuda()
    for mode in ("tile", "centroid"):
        for kw in (dict(top_c=10, radius_m=3.0, toler_pct=20), dict(top_c=10, radius_m=3.0, toler_pct=100),
                   dict(top_c=4, radius_m=0.3, toler_pct=30), dict(top_c=1, radius_m=0.0, toler_pct=0)):
            idx, _, xy, st = lhr.lhr_query_window(h, frames, offs, k, shortlist=cfg["shortlist"], mode=mode, **kw)
            torch.cuda.synchronize()
            cands = oret.window_candidates(idx.cpu().numpy()[:, 0], win.offsets)
            o_xy, o_st = oagg.aggregate_windows(cands, db.xy, mode=mode, **kw)
            assert np.array_equal(st.cpu().numpy(), o_st), (mode, kw)
            assert np.max(np.abs(xy.cpu().numpy() - o_xy)) <= XY_ATOL, (mode, kw)
    assert lhr.lhr_db_error(h) == 0
    h.close()
