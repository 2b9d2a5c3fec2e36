"""Serving runtime (continuous batching over many user streams): every
window's result in the mix equals the same window computed alone with
lhr_query_window, for coarse-to-fine and exhaustive retrieval, several
aggregation modes, uneven window lengths, a memory budget that admits one
tick at a time, and bad arguments."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lhr():
    import paper_2006_08861_gb300 as m
    return m


def _streams(db, n_streams, frames_per_stream, seed):
    """Each stream walks its own stretch of the path: frames along it."""
    out = []
    for s in range(n_streams):
        w = synth.make_windows(db, 1, frames_per_stream, seed=seed + s)
        out.append(w.frames)
    return out


def _run_mix(lhr, h, streams, lens, k, shortlist, mode, **kw):
    srv = lhr.Server(h, n_streams=len(streams), max_window=max(lens), k=k, shortlist=shortlist, mode=mode, **kw)
    order = []
    nfr = streams[0].shape[0]
    rid = 0
    expect = {}
    rng = np.random.default_rng(5)
    # interleave the streams' frames in a shuffled round-robin
    for t in range(nfr):
        for s in rng.permutation(len(streams)):
            m = lens[s]
            srv.submit(int(s), streams[s][t], window_m=m, request_id=rid)
            lo = max(0, t - m + 1)
            expect[rid] = (int(s), lo, t + 1)
            rid += 1
    srv.drain(120000)
    res = []
    while True:
        got = srv.poll(wait_ms=0)
        if not got:
            break
        res += got
    srv.close()
    assert len(res) == rid
    return res, expect


@pytest.mark.parametrize("shortlist,mode,kw", [
    (256, "tile", dict(max_batch_frames=16, n_lanes=2)),
    (256, "centroid", dict(max_batch_frames=7, n_lanes=3)),
    (0, "tile", dict(max_batch_frames=40, n_lanes=2)),
    (256, "tile", dict(max_batch_frames=5, n_lanes=2, mem_budget_bytes=1)),  # one tick at a time
])
def test_mix_equals_alone(lhr, shortlist, mode, kw):
    db = synth.make_database(20_000, 128, seed=61)
    h = lhr.lhr_build_db(db.feats, db.xy, coarse_dim=32)
    streams = _streams(db, 12, 14, seed=620)
    lens = [3 + (s * 5) % 8 for s in range(12)]  # 3 .. 10
    k = 10
    res, expect = _run_mix(lhr, h, streams, lens, k, shortlist, mode, **kw)
    for r in res:
        s, lo, hi = expect[r["request_id"]]
        assert r["stream_id"] == s and r["m"] == hi - lo
        fr = torch.from_numpy(np.ascontiguousarray(streams[s][lo:hi])).cuda()
        offs = torch.tensor([0, hi - lo], dtype=torch.int32, device="cuda")
        _, _, xy, st = lhr.lhr_query_window(h, fr, offs, k, shortlist=shortlist, mode=mode)
        torch.cuda.synchronize()
        assert r["status"] == int(st.item()), r
        assert tuple(xy.cpu().numpy()[0]) == r["xy"], (r, xy)
        assert r["latency_us"] > 0
    assert lhr.lhr_db_error(h) == 0


def test_server_bad_arguments(lhr):
    db = synth.make_database(3000, 64, seed=63)
    h = lhr.lhr_build_db(db.feats, db.xy, coarse_dim=16)
    with pytest.raises(lhr.LhrError):
        lhr.Server(h, n_streams=2, max_window=4, k=5, shortlist=64, n_lanes=1)
    with pytest.raises(lhr.LhrError):
        lhr.Server(h, n_streams=2, max_window=4, k=5, shortlist=64, ring_frames=4)
    srv = lhr.Server(h, n_streams=2, max_window=4, k=5, shortlist=64)
    f = db.feats[0]
    with pytest.raises(lhr.LhrError):
        srv.submit(2, f, window_m=1)
    with pytest.raises(lhr.LhrError):
        srv.submit(0, f, window_m=5)
    srv.submit(0, f, window_m=1, request_id=9)
    srv.drain(30000)
    r = srv.poll(wait_ms=100)
    assert len(r) == 1 and r[0]["request_id"] == 9 and r[0]["m"] == 1
    srv.close()


def _ring_bytes(ring_frames, dim, k):
    return ring_frames * (dim * 4 + k * 12)


def test_stream_admission_by_ring_memory(lhr):
    # Rings for two streams: a third stream is refused until one closes; the
    # admitted stream then starts from no frames and its windows are right.
    db = synth.make_database(20_000, 128, seed=64)
    h = lhr.lhr_build_db(db.feats, db.xy, coarse_dim=32)
    k, mw, mb = 10, 4, 8
    ring = 2 * mw + mb
    srv = lhr.Server(h, n_streams=4, max_window=mw, k=k, shortlist=256, max_batch_frames=mb,
                     ring_mem_bytes=2 * _ring_bytes(ring, 128, k) + 100)
    walks = _streams(db, 3, 6, seed=640)
    a, b = srv.open_stream(), srv.open_stream()
    assert {a, b} == {0, 1}
    with pytest.raises(lhr.LhrError) as e:
        srv.open_stream()
    assert e.value.status == lhr.LHR_ERR_OOM
    with pytest.raises(lhr.LhrError):
        srv.submit(2, walks[2][0], window_m=1)        # never opened
    for t in range(6):
        srv.submit(a, walks[0][t], window_m=3, request_id=100 + t)
        srv.submit(b, walks[1][t], window_m=3, request_id=200 + t)
    srv.close_stream(a)
    with pytest.raises(lhr.LhrError):
        srv.submit(a, walks[0][0], window_m=1)        # closed
    c = srv.open_stream()                              # admitted once a ring is free
    assert c == a
    for t in range(6):
        srv.submit(c, walks[2][t], window_m=4, request_id=300 + t)
    srv.drain(60000)
    res = []
    while True:
        got = srv.poll(wait_ms=0)
        if not got:
            break
        res += got
    srv.close()
    assert len(res) == 18
    for r in res:
        base, t = divmod(r["request_id"], 100)
        walk, m = {1: (walks[0], 3), 2: (walks[1], 3), 3: (walks[2], 4)}[base]
        lo = max(0, t - m + 1)
        assert r["m"] == t + 1 - lo
        fr = torch.from_numpy(np.ascontiguousarray(walk[lo:t + 1])).cuda()
        offs = torch.tensor([0, t + 1 - lo], dtype=torch.int32, device="cuda")
        _, _, xy, st = lhr.lhr_query_window(h, fr, offs, k, shortlist=256)
        torch.cuda.synchronize()
        assert r["status"] == int(st.item()) and tuple(xy.cpu().numpy()[0]) == r["xy"], r
    assert lhr.lhr_db_error(h) == 0


def test_low_precision_serving_mix_equals_alone(lhr):
    # BF16-resident retrieval per tick (tensor-core scores, top-64, FP32 re-rank):
    # the batch's shared power-of-two query scale leaves BF16 codes times scale
    # unchanged, so every window equals the same window alone.
    db = synth.make_database(300_000, 256, seed=66)
    h = lhr.lhr_build_db(db.feats, db.xy, lowp=1)
    streams = _streams(db, 6, 10, seed=660)
    lens = [3, 5, 8, 10, 4, 6]
    k = 20
    res, expect = _run_mix(lhr, h, streams, lens, k, 0, "tile", score="bf16", rerank_width=64,
                           max_batch_frames=24, n_lanes=2)
    for r in res:
        s, lo, hi = expect[r["request_id"]]
        fr = torch.from_numpy(np.ascontiguousarray(streams[s][lo:hi])).cuda()
        offs = torch.tensor([0, hi - lo], dtype=torch.int32, device="cuda")
        _, _, xy, st = lhr.lhr_query_window(h, fr, offs, k, score="bf16", rerank_width=64)
        torch.cuda.synchronize()
        assert r["status"] == int(st.item()) and tuple(xy.cpu().numpy()[0]) == r["xy"], r
    assert lhr.lhr_db_error(h) == 0


def test_serving_configuration_against_oracle(lhr):
    # 1,000,000 x 256 database, coarse prefix 32, shortlist 512, k = 20; user
    # streams send frames with windows m in 3..10. Sampled served windows are
    # checked against the FP64 oracle: coarse-to-fine top-k of every frame
    # (oracle.retrieval) and Algorithm 2 on their candidates (oracle.aggregate).
    import concurrent.futures as cf
    import os

    from oracle import aggregate as oagg
    from oracle import retrieval as oret
    from tests.parity import GAP, XY_ATOL
    cfg = synth.CONFIGS["serving"]
    db = synth.make_database(cfg["n"], cfg["dim"], seed=synth.db_seed(cfg["index"]))
    h = lhr.lhr_build_db(db.feats, db.xy, coarse_dim=32)
    k, S = cfg["k"], 512
    n_streams, per = 8, 12
    streams = _streams(db, n_streams, per, seed=synth.query_seed(cfg["index"]))
    rng = np.random.default_rng(7)
    lens = rng.integers(cfg["m_lo"], cfg["m_hi"] + 1, size=n_streams)
    res, expect = _run_mix(lhr, h, streams, list(lens), k, S, "tile", max_batch_frames=32, n_lanes=3)
    byid = {r["request_id"]: r for r in res}
    sample = sorted(rng.choice(sorted(byid), size=32, replace=False).tolist())

    def oracle_frame(f):
        # The oracle's shortlist boundary may nearly tie (then rounding picks the boundary rows), so the
        # frame's top k counts as determined only when the top k over every row that any valid shortlist
        # could hold is made of rows every valid shortlist holds, with its k-th / (k+1)-th gap separated.
        o_idx, o_dist, _ = oret.hierarchical_topk(f[None], db.feats, 32, S, k + 1)
        dc = oret.sq_dist(f[:32], db.feats[:, :32])
        cS = np.partition(dc, S - 1)[S - 1]
        sure = np.nonzero(dc < cS * (1 - 2 * GAP))[0]
        band = np.nonzero((dc >= cS * (1 - 2 * GAP)) & (dc <= cS * (1 + 2 * GAP)))[0]
        possible = np.concatenate([sure, band])
        p_idx, p_dist = oret.top_n(oret.sq_dist(f, db.feats[possible]), possible, k + 1)
        determined = (not np.isin(p_idx[:k], band).any() and
                      (p_dist[k] - p_dist[k - 1]) > GAP * p_dist[k - 1] and
                      np.array_equal(np.sort(p_idx[:k]), np.sort(o_idx[0, :k])))
        return o_idx[0, :k], determined

    frames = {}
    for rid in sample:
        s, lo, hi = expect[rid]
        for t in range(lo, hi):
            frames[(s, t)] = None
    keys = list(frames)
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        for key, out in zip(keys, ex.map(lambda kk: oracle_frame(streams[kk[0]][kk[1]]), keys)):
            frames[key] = out
    compared = 0
    for rid in sample:
        s, lo, hi = expect[rid]
        if not all(frames[(s, t)][1] for t in range(lo, hi)):
            continue  # a frame's top k depends on which near-tied rows enter its shortlist
        cands = np.concatenate([frames[(s, t)][0] for t in range(lo, hi)])
        o_xy, o_st = oagg.aggregate_windows([cands], db.xy, mode="tile")
        r = byid[rid]
        assert r["status"] == int(o_st[0]), (rid, r)
        assert np.max(np.abs(np.array(r["xy"]) - o_xy[0])) <= XY_ATOL, (rid, r, o_xy)
        compared += 1
    # about a third of the windows have every frame determined (windows hold 3-10 frames)
    assert compared >= 6, compared
    assert lhr.lhr_db_error(h) == 0
