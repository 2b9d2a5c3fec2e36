"""Exhaustive FP32 scan + fused top-k (§3.1, Algorithm 1) against the FP64
oracle: several tiles and chunks, ragged tails, every query-block width,
subspaces, padding, exact ties, and the 2M-row database on sampled queries."""
import numpy as np
import pytest

import synth
from oracle import retrieval as oret
from tests.parity import check_list

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lhr():
    import paper_2006_08861_gb300 as m
    return m


def _run(lhr, X, Q, k, subspace=None, xy=None):
    if xy is None:
        xy = np.zeros((X.shape[0], 2))
    db = lhr.lhr_build_db(X, xy, subspace=subspace)
    q = torch.from_numpy(np.ascontiguousarray(Q, dtype=np.float32)).cuda()
    idx, dist = lhr.lhr_query(db, q, k)
    torch.cuda.synchronize()
    assert lhr.lhr_db_error(db) == 0
    return db, idx.cpu().numpy(), dist.cpu().numpy()


def _compare(X, Q, k, g_idx, g_dist, subspace=None, n_sub=None):
    o_idx, o_dist = oret.exhaustive_topk(Q, X, k + 1, subspace=subspace, n_subspaces=n_sub)
    groups = None
    if subspace is not None:
        groups = [np.nonzero(subspace == s)[0] for s in range(o_idx.shape[1])]
    exact = 0
    for qi in range(Q.shape[0]):
        for s in range(g_idx.shape[1]):
            exact += check_list(Q[qi], X, g_idx[qi, s], g_dist[qi, s], o_idx[qi, s], o_dist[qi, s], k,
                                rows=None if groups is None else groups[s], where=f"q{qi} s{s}")
    return exact


def test_tiny_configuration(lhr):
    # N=2,000 locations, D=128, Q=16 single frames, k=10 (the tiny workload)
    db = synth.make_database(2000, 128, seed=1000)
    q, rows, _ = synth.make_point_queries(db, 16, seed=2000)
    _, gi, gd = _run(lhr, db.feats, q, 10, xy=db.xy)
    assert gi.shape == (16, 1, 10)
    exact = _compare(db.feats, q, 10, gi, gd)
    assert exact >= 16 * 8
    # the true row is found first for these low-noise queries
    assert np.mean(gi[:, 0, 0] == rows) >= 0.75  # scene aliasing puts a copy first now and then


@pytest.mark.parametrize("n,dim,nq,k", [
    (1237, 36, 5, 7),      # ragged everything; lanes partly idle
    (4099, 128, 16, 16),   # query block of 16
    (50_003, 256, 3, 20),  # many chunks, ragged stage tail
    (3001, 512, 4, 32),    # widest rows, k = 32
    (4000, 128, 37, 12),   # several query blocks
    (997, 64, 1, 1),       # single query, k = 1
    (2500, 256, 8, 20),    # query block of 8 on 1 KB rows
    (700, 8, 2, 5),        # tiny rows
])
def test_shapes(lhr, n, dim, nq, k):
    rng = np.random.default_rng(n + dim + nq + k)
    X = rng.standard_normal((n, dim)).astype(np.float32)
    Q = (X[rng.integers(0, n, nq)] + 0.3 * rng.standard_normal((nq, dim))).astype(np.float32)
    _, gi, gd = _run(lhr, X, Q, k)
    _compare(X, Q, k, gi, gd)


@pytest.mark.parametrize("offset", [100.0, -3000.0])
def test_large_common_offset(lhr, offset):
    # ||x||^2 + ||q||^2 - 2 q.x cancels badly when every vector sits far from
    # the origin; the scan's filter must still never drop a true neighbour.
    rng = np.random.default_rng(9)
    X = (offset + rng.standard_normal((6000, 64))).astype(np.float32)
    Q = (X[rng.integers(0, 6000, 6)] + 0.1 * rng.standard_normal((6, 64))).astype(np.float32)
    _, gi, gd = _run(lhr, X, Q, 16)
    _compare(X, Q, 16, gi, gd)


def test_exact_ties_break_by_lower_row(lhr):
    # Integer-valued rows with many duplicates: FP32 distances are exact, so
    # the order must equal the oracle's (distance, row) order bit for bit.
    rng = np.random.default_rng(5)
    base = rng.integers(-2, 3, size=(40, 16)).astype(np.float32)
    X = base[rng.integers(0, 40, size=3000)]
    Q = rng.integers(-2, 3, size=(6, 16)).astype(np.float32)
    _, gi, gd = _run(lhr, X, Q, 25)
    o_idx, o_dist = oret.exhaustive_topk(Q, X, 25)
    assert np.array_equal(gi, o_idx)
    assert np.array_equal(gd.astype(np.float64), o_dist)


def test_k_larger_than_database_pads(lhr):
    rng = np.random.default_rng(6)
    X = rng.standard_normal((5, 8)).astype(np.float32)
    Q = rng.standard_normal((3, 8)).astype(np.float32)
    _, gi, gd = _run(lhr, X, Q, 10)
    o_idx, o_dist = oret.exhaustive_topk(Q, X, 10)
    assert np.array_equal(gi, o_idx)
    assert np.all(np.isinf(gd[:, :, 5:])) and np.all(gi[:, :, 5:] == -1)


def test_subspaces_per_subspace_topk(lhr):
    # §3.1: the database is divided into subspaces searched independently;
    # §4: top N per frame and per path. Ids are shuffled (not grouped), one
    # subspace is empty and one is smaller than k.
    rng = np.random.default_rng(7)
    n, dim, k = 3000, 64, 15
    X = rng.standard_normal((n, dim)).astype(np.float32)
    sub = rng.choice([0, 1, 3, 4], size=n, p=[0.4, 0.3, 0.297, 0.003]).astype(np.int32)
    sub[:2] = 4
    Q = (X[rng.integers(0, n, 5)] + 0.2 * rng.standard_normal((5, dim))).astype(np.float32)
    db, gi, gd = _run(lhr, X, Q, k, subspace=sub)
    assert db.n_subspaces == 5 and gi.shape == (5, 5, k)
    assert np.all(gi[:, 2] == -1)  # empty subspace 2
    _compare(X, Q, k, gi, gd, subspace=sub, n_sub=5)


def test_paper_candidate_shape_825(lhr):
    # §4: N = 15 per frame, M = 11 frames, P = 5 paths -> 825 candidates.
    db = synth.make_database(5000, 128, seed=33)
    sub = np.minimum(np.arange(db.n) * 5 // db.n, 4).astype(np.int32)
    win = synth.make_windows(db, 2, 11, seed=34)
    h = lhr.lhr_build_db(db.feats, db.xy, subspace=sub)
    frames = torch.from_numpy(win.frames).cuda()
    idx, dist = lhr.lhr_query(h, frames, 15)
    torch.cuda.synchronize()
    gi = idx.cpu().numpy()
    cands = oret.window_candidates(gi, win.offsets)
    assert [c.size for c in cands] == [825, 825] and np.all(gi >= 0)
    _compare(db.feats, win.frames, 15, gi, dist.cpu().numpy(), subspace=sub, n_sub=5)


def test_invalid_arguments_raise(lhr):
    rng = np.random.default_rng(8)
    X = rng.standard_normal((100, 16)).astype(np.float32)
    db = lhr.lhr_build_db(X, np.zeros((100, 2)))
    q = torch.zeros((2, 16), device="cuda")
    for bad in (dict(k=0), dict(k=33), dict(k=5, shortlist=3)):
        with pytest.raises(lhr.LhrError) as e:
            lhr.lhr_query(db, q, **bad)
        assert e.value.status == lhr.LHR_ERR_INVALID_ARG
    with pytest.raises(lhr.LhrError):
        lhr.lhr_query(db, q, 5, shortlist=64)  # no coarse level
    Xn = X.copy()
    Xn[3, 4] = np.nan
    with pytest.raises(lhr.LhrError) as e:
        lhr.lhr_build_db(Xn, np.zeros((100, 2)))
    assert e.value.status == lhr.LHR_ERR_INVALID_ARG
    with pytest.raises(lhr.LhrError):
        lhr.lhr_build_db(np.zeros((10, 6), np.float32), np.zeros((10, 2)))  # D % 4 != 0


def test_two_million_rows_sampled(lhr):
    # The 2,000,000 x 256 database of the precision workload, plain FP32 scan
    # with 8 frames per pass (the launch the HBM benchmark times); two sampled
    # queries are checked against the oracle in full.
    db = synth.make_database(2_000_000, 256, seed=1002)
    q, rows, _ = synth.make_point_queries(db, 8, seed=2002)
    h = lhr.lhr_build_db(db.feats, db.xy)
    qt = torch.from_numpy(q).cuda()
    idx, dist = lhr.lhr_query(h, qt, 20)
    torch.cuda.synchronize()
    gi, gd = idx.cpu().numpy(), dist.cpu().numpy()
    for qi in (0, 5):
        o_idx, o_dist = oret.exhaustive_topk(q[qi:qi + 1], db.feats, 21)
        check_list(q[qi], db.feats, gi[qi, 0], gd[qi, 0], o_idx[0, 0], o_dist[0, 0], 20, where=f"q{qi}")
    # most queries find their own row first (aliased copies sometimes win)
    assert np.mean(gi[:, 0, 0] == rows) >= 0.75
    h.close()


# ------------------------------------------------------------------ pilot sample
# Databases of >= 65,536 rows carry a pilot sample (every 64th row); its k-th
# distances seed the scan's thresholds. Results must not change.
def test_pilot_seeded_scan_matches_oracle(lhr):
    rng = np.random.default_rng(41)
    n, dim, nq, k = 70_001, 64, 9, 32
    X = rng.standard_normal((n, dim)).astype(np.float32)
    Q = (X[rng.integers(0, n, nq)] + 0.3 * rng.standard_normal((nq, dim))).astype(np.float32)
    _, gi, gd = _run(lhr, X, Q, k)
    _compare(X, Q, k, gi, gd)


def test_pilot_with_subspaces_small_and_empty(lhr):
    # subspace 1 holds fewer than k sample rows (its pilot bound is +inf),
    # subspace 2 is empty, ids are shuffled
    rng = np.random.default_rng(42)
    n, dim, k = 90_000, 32, 20
    X = rng.standard_normal((n, dim)).astype(np.float32)
    sub = rng.choice([0, 1, 3], size=n, p=[0.6, 0.01, 0.39]).astype(np.int32)
    Q = (X[rng.integers(0, n, 6)] + 0.2 * rng.standard_normal((6, dim))).astype(np.float32)
    db, gi, gd = _run(lhr, X, Q, k, subspace=sub)
    assert db.n_subspaces == 4 and np.all(gi[:, 2] == -1)
    _compare(X, Q, k, gi, gd, subspace=sub, n_sub=4)


def test_pilot_exact_ties(lhr):
    # integer rows with many exact duplicates: the pilot bound lands on tied
    # distances; order must still equal the oracle's bit for bit
    rng = np.random.default_rng(43)
    base = rng.integers(-2, 3, size=(60, 16)).astype(np.float32)
    X = base[rng.integers(0, 60, size=80_000)]
    Q = rng.integers(-2, 3, size=(5, 16)).astype(np.float32)
    _, gi, gd = _run(lhr, X, Q, 30)
    o_idx, o_dist = oret.exhaustive_topk(Q, X, 30)
    assert np.array_equal(gi, o_idx)
    assert np.array_equal(gd.astype(np.float64), o_dist)


def test_many_frames_match_oracle(lhr):
    # >= 64 frames over a sampled database take the register-tiled many-frame
    # pass: three frame blocks (the last ragged), k = 20
    rng = np.random.default_rng(45)
    n, dim, nq, k = 70_003, 128, 150, 20
    X = rng.standard_normal((n, dim)).astype(np.float32)
    Q = (X[rng.integers(0, n, nq)] + 0.3 * rng.standard_normal((nq, dim))).astype(np.float32)
    _, gi, gd = _run(lhr, X, Q, k)
    _compare(X, Q, k, gi, gd)


def test_many_frames_exact_ties(lhr):
    # integer rows with many exact duplicates through the many-frame pass:
    # equal to the oracle bit for bit (ties by lower row)
    rng = np.random.default_rng(46)
    base = rng.integers(-2, 3, size=(60, 64)).astype(np.float32)
    X = base[rng.integers(0, 60, size=80_000)]
    Q = rng.integers(-2, 3, size=(70, 64)).astype(np.float32)
    _, gi, gd = _run(lhr, X, Q, 30)
    o_idx, o_dist = oret.exhaustive_topk(Q, X, 30)
    assert np.array_equal(gi, o_idx)
    assert np.array_equal(gd.astype(np.float64), o_dist)


@pytest.mark.parametrize("n,dim,nq,k,weighted", [
    (100_003, 256, 300, 32, False),  # 8 K slices, three frame blocks of 128 and a padded fourth
    (70_001, 192, 257, 10, True),    # 6 K slices, weighted, one frame past a 256-frame sort unit
    (66_000, 64, 64, 1, False),      # 2 K slices, a single frame block, k = 1
])
def test_many_frames_tensor_core_filter(lhr, n, dim, nq, k, weighted):
    # many frames go through the TF32 tensor-core filter; frames with very
    # different thresholds (noise 0.01 .. 3) share 32-frame groups only after
    # the threshold sort, so an unsorted or wrong group bound loses rows here
    rng = np.random.default_rng(n + nq)
    X = rng.standard_normal((n, dim)).astype(np.float32)
    noise = np.exp(rng.uniform(np.log(0.01), np.log(3.0), nq)).astype(np.float32)[:, None]
    Q = (X[rng.integers(0, n, nq)] + noise * rng.standard_normal((nq, dim))).astype(np.float32)
    if weighted:
        w = rng.uniform(0.5, 1.5, dim).astype(np.float32)
        db = lhr.lhr_build_db(X, np.zeros((n, 2)))
        gi, gd = lhr.lhr_query_weighted(db, torch.from_numpy(Q).cuda(), k, torch.from_numpy(w).cuda())
        torch.cuda.synchronize()
        assert lhr.lhr_db_error(db) == 0
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
        oi, od = oret.exhaustive_topk(Q, X, k + 1, w=w)
        exact = sum(check_list(Q[qi], X, gi[qi, 0], gd[qi, 0], oi[qi, 0], od[qi, 0], k, where=f"q{qi}", w=w)
                    for qi in range(nq))
    else:
        _, gi, gd = _run(lhr, X, Q, k)
        exact = _compare(X, Q, k, gi, gd)
    assert exact >= nq * k // 2  # ranks separated from both neighbours, compared bit-exactly


def test_many_frames_wide_dynamic_range(lhr):
    # dimensions of magnitude 1e-6 .. 1e3 and weights 1e-2 .. 1e2 through the
    # FP16 tensor-core filter: the power-of-two scales keep the largest values
    # below FP16's overflow, most small ones fall into its subnormal range, and
    # the filter's margin (with its subnormal term) must still keep every row of
    # the exact weighted top k
    rng = np.random.default_rng(91)
    n, dim, nq, k = 70_000, 64, 80, 16
    mag = (10.0 ** rng.uniform(-6, 3, dim)).astype(np.float32)
    X = (rng.standard_normal((n, dim)) * mag).astype(np.float32)
    Q = (X[rng.integers(0, n, nq)] + 0.05 * mag * rng.standard_normal((nq, dim))).astype(np.float32)
    w = (10.0 ** rng.uniform(-2, 2, dim)).astype(np.float32)
    db = lhr.lhr_build_db(X, np.zeros((n, 2)))
    gi, gd = lhr.lhr_query_weighted(db, torch.from_numpy(Q).cuda(), k, torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    assert lhr.lhr_db_error(db) == 0
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    oi, od = oret.exhaustive_topk(Q, X, k + 1, w=w)
    exact = sum(check_list(Q[qi], X, gi[qi, 0], gd[qi, 0], oi[qi, 0], od[qi, 0], k, where=f"q{qi}", w=w)
                for qi in range(nq))
    assert exact >= nq * k // 2


def test_pilot_and_plain_scan_agree(lhr):
    # lhr_query seeds from the pilot; lhr_query_static never does
    rng = np.random.default_rng(44)
    X = rng.standard_normal((100_000, 128)).astype(np.float32)
    db = lhr.lhr_build_db(X, np.zeros((100_000, 2)))
    q = torch.from_numpy((X[:7] + 0.1 * rng.standard_normal((7, 128))).astype(np.float32)).cuda()
    i1, d1 = lhr.lhr_query(db, q, 24)
    out_i = torch.empty((7, 1, 24), dtype=torch.int64, device="cuda")
    out_d = torch.empty((7, 1, 24), dtype=torch.float32, device="cuda")
    lhr.lhr_query_static(db, q, 24, (out_i, out_d))
    torch.cuda.synchronize()
    assert torch.equal(i1, out_i) and torch.equal(d1, out_d)


def test_binding_rejects_mismatched_buffers(lhr):
    # the binding checks shapes, dtypes and devices before the library writes through a pointer
    X = np.random.default_rng(9).standard_normal((500, 64)).astype(np.float32)
    db = lhr.lhr_build_db(X, np.zeros((500, 2)))
    q = torch.zeros((3, 64), device="cuda")
    k = 5
    good = (torch.empty((3, 1, k), dtype=torch.int64, device="cuda"),
            torch.empty((3, 1, k), dtype=torch.float32, device="cuda"))
    lhr.lhr_query(db, q, k, out=good)
    lhr.lhr_query_static(db, q, k, out=good)
    with pytest.raises(ValueError):
        lhr.lhr_query(db, torch.zeros((3, 32), device="cuda"), k)          # D differs from the database's
    with pytest.raises(ValueError):
        lhr.lhr_query(db, q, k, out=(good[0][:2], good[1][:2]))            # too few rows
    with pytest.raises(ValueError):
        lhr.lhr_query_static(db, q, k + 1, out=good)                        # k differs
    with pytest.raises(TypeError):
        lhr.lhr_query(db, q, k, out=(good[0], good[1].double()))            # wrong dtype
    with pytest.raises(TypeError):
        lhr.lhr_query(db, q, k, out=(good[0].cpu(), good[1]))               # host tensor
    torch.cuda.synchronize()
    assert lhr.lhr_db_error(db) == 0
