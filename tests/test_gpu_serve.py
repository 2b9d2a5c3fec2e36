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
