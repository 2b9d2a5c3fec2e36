"""Pins of the FP64 oracle against facts fixed outside the oracle itself:
hand-computed distances, brute force on tiny inputs, invariants of the method,
library special cases, and hand-derived Algorithm 2 cases (tests/golden)."""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import aggregate, lowp, retrieval, soft

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "aggregation_cases.json")


# ---------------------------------------------------------------- O1 distance
def test_distance_hand_computed():
    # (1-2)^2 + (2-0)^2 + (3-3)^2 + (4-7)^2 = 1 + 4 + 0 + 9 = 14
    q = [1.0, 2.0, 3.0, 4.0]
    X = np.array([[2.0, 0.0, 3.0, 7.0], [1.0, 2.0, 3.0, 4.0], [0.0, 0.0, 0.0, 0.0]])
    d = retrieval.sq_dist(q, X)
    assert d.tolist() == [14.0, 0.0, 30.0]
    # weights 1, 1/2, 2, 1/4: 1 + 2 + 0 + 2.25 = 5.25
    w = [1.0, 0.5, 2.0, 0.25]
    assert retrieval.sq_dist(q, X[:1], w).tolist() == [5.25]


def test_distance_exact_on_integer_vectors():
    rng = np.random.default_rng(7)
    Q = rng.integers(-50, 50, size=(5, 16))
    X = rng.integers(-50, 50, size=(40, 16))
    for q in Q:
        exact = [sum(int(a - b) ** 2 for a, b in zip(q, x)) for x in X]
        assert retrieval.sq_dist(q.astype(np.float32), X.astype(np.float32)).tolist() == exact


# ---------------------------------------------------------------- O2 top-k
def _brute_topk(d, k):
    """Selection by repeated minimum of (distance, row) -- a different algorithm
    from the oracle's sort."""
    taken, out = set(), []
    for _ in range(min(k, len(d))):
        best = None
        for i, v in enumerate(d):
            if i in taken:
                continue
            if best is None or (v, i) < (d[best], best):
                best = i
        taken.add(best)
        out.append(best)
    return out


def test_topk_ties_break_by_row():
    d = np.array([1.0, 0.0, 1.0, 0.0, 2.0])
    idx, dist = retrieval.top_n(d, np.arange(5), 4)
    assert idx.tolist() == [1, 3, 0, 2]
    assert dist.tolist() == [0.0, 0.0, 1.0, 1.0]


def test_topk_padding_when_k_exceeds_rows():
    idx, dist = retrieval.top_n(np.array([3.0, 1.0]), np.array([10, 11]), 4)
    assert idx.tolist() == [11, 10, -1, -1]
    assert dist[:2].tolist() == [1.0, 3.0] and np.isinf(dist[2:]).all()


def test_exhaustive_topk_equals_brute_force():
    rng = np.random.default_rng(11)
    for n, dim, k in [(1, 4, 1), (7, 3, 3), (33, 8, 5), (64, 8, 64), (20, 2, 25)]:
        X = rng.integers(-3, 4, size=(n, dim)).astype(np.float32)   # many exact ties
        Q = rng.integers(-3, 4, size=(3, dim)).astype(np.float32)
        idx, dist = retrieval.exhaustive_topk(Q, X, k)
        for qi in range(3):
            d = [sum(float(a - b) ** 2 for a, b in zip(Q[qi], x)) for x in X]
            want = _brute_topk(d, k)
            got = idx[qi, 0].tolist()
            assert got[:len(want)] == want
            assert all(v == -1 for v in got[len(want):])


def test_exhaustive_topk_equals_numpy_stable_argsort():
    rng = np.random.default_rng(12)
    X = rng.standard_normal((500, 16)).astype(np.float32)
    Q = rng.standard_normal((4, 16)).astype(np.float32)
    idx, dist = retrieval.exhaustive_topk(Q, X, 50)
    for qi in range(4):
        d = ((X.astype(np.float64) - Q[qi].astype(np.float64)) ** 2).sum(1)
        want = np.argsort(d, kind="stable")[:50]
        assert idx[qi, 0].tolist() == want.tolist()


def test_per_subspace_topk_equals_topk_of_each_subspace_alone():
    rng = np.random.default_rng(13)
    X = rng.standard_normal((300, 8)).astype(np.float32)
    sub = rng.integers(0, 5, size=300)
    Q = rng.standard_normal((3, 8)).astype(np.float32)
    idx, dist = retrieval.exhaustive_topk(Q, X, 15, subspace=sub, n_subspaces=5)
    assert idx.shape == (3, 5, 15)
    for s in range(5):
        rows = np.nonzero(sub == s)[0]
        ii, dd = retrieval.exhaustive_topk(Q, X[rows], 15)
        mapped = np.where(ii[:, 0] >= 0, rows[np.maximum(ii[:, 0], 0)], -1)
        assert (idx[:, s] == mapped).all()


# ---------------------------------------------------------------- O3 coarse-to-fine
def test_hierarchical_with_full_shortlist_equals_exhaustive():
    rng = np.random.default_rng(14)
    X = rng.standard_normal((400, 32)).astype(np.float32)
    Q = rng.standard_normal((5, 32)).astype(np.float32)
    ex_i, ex_d = retrieval.exhaustive_topk(Q, X, 10)
    h_i, h_d, _ = retrieval.hierarchical_topk(Q, X, coarse_dim=8, shortlist=400, k=10)
    assert (h_i == ex_i[:, 0]).all() and np.array_equal(h_d, ex_d[:, 0])


def test_hierarchical_with_full_prefix_equals_exhaustive():
    rng = np.random.default_rng(15)
    X = rng.standard_normal((400, 32)).astype(np.float32)
    Q = rng.standard_normal((5, 32)).astype(np.float32)
    ex_i, _ = retrieval.exhaustive_topk(Q, X, 10)
    h_i, _, _ = retrieval.hierarchical_topk(Q, X, coarse_dim=32, shortlist=10, k=10)
    assert (h_i == ex_i[:, 0]).all()


def test_hierarchical_uses_the_prefix_and_the_shortlist():
    # row 0: prefix exact, tail far (d = 200); row 1: prefix far, total d = 50.
    X = np.array([[0, 0, 10, 10], [5, 5, 0, 0]], dtype=np.float32)
    q = np.zeros((1, 4), dtype=np.float32)
    h_i, h_d, short = retrieval.hierarchical_topk(q, X, coarse_dim=2, shortlist=1, k=1)
    assert short.tolist() == [[0]] and h_i.tolist() == [[0]] and h_d.tolist() == [[200.0]]
    ex_i, ex_d = retrieval.exhaustive_topk(q, X, 1)
    assert ex_i[0, 0].tolist() == [1] and ex_d[0, 0].tolist() == [50.0]


def test_hierarchical_per_subspace_with_full_shortlists_equals_exhaustive_per_subspace():
    # shortlists as large as the largest subspace reduce the coarse-to-fine form
    # to exhaustive search, subspace by subspace (the exhaustive per-subspace
    # oracle is pinned above against each subspace alone)
    rng = np.random.default_rng(16)
    X = rng.standard_normal((500, 24)).astype(np.float32)
    sub = rng.integers(0, 4, 500).astype(np.int32)
    Q = rng.standard_normal((6, 24)).astype(np.float32)
    big = int(np.bincount(sub).max())
    h_i, h_d = retrieval.hierarchical_topk_subspaces(Q, X, 8, big, 7, sub, 4)
    ex_i, ex_d = retrieval.exhaustive_topk(Q, X, 7, subspace=sub, n_subspaces=4)
    assert (h_i == ex_i).all() and np.array_equal(h_d, ex_d)
    # and every returned row lies in its subspace
    assert all((sub[h_i[:, s]] == s).all() for s in range(4))


def test_hierarchical_per_subspace_uses_each_subspaces_own_shortlist():
    # subspace 0 holds rows 0, 2; subspace 1 holds rows 1, 3. With S = 1 the
    # prefix picks row 2 in subspace 0 (prefix exact, tail far) and row 1 in
    # subspace 1, although rows 0 and 3 are nearer over the whole feature.
    X = np.array([[4, 4, 0, 0], [0, 1, 9, 9], [0, 0, 9, 9], [3, 3, 0, 0]], dtype=np.float32)
    sub = np.array([0, 1, 0, 1], dtype=np.int32)
    q = np.zeros((1, 4), dtype=np.float32)
    h_i, h_d = retrieval.hierarchical_topk_subspaces(q, X, 2, 1, 1, sub)
    assert h_i.tolist() == [[[2], [1]]] and h_d.tolist() == [[[162.0], [163.0]]]
    ex_i, ex_d = retrieval.exhaustive_topk(q, X, 1, subspace=sub)
    assert ex_i.tolist() == [[[0], [3]]] and ex_d.tolist() == [[[32.0], [18.0]]]


# ---------------------------------------------------------------- O4 windows
def test_candidate_count_of_the_papers_experiment():
    # §4: N = 15 candidates per frame, M = 11 frames, P = 5 paths -> 825.
    k, m, ns = 15, 11, 5
    frame_idx = np.arange(m * ns * k).reshape(m, ns, k)
    cands = retrieval.window_candidates(frame_idx, np.array([0, m]))
    assert len(cands) == 1 and cands[0].size == 825 == k * m * ns


def test_window_candidates_keep_duplicates_and_order():
    frame_idx = np.array([[3, 4], [4, 5], [9, 9]])
    cands = retrieval.window_candidates(frame_idx, np.array([0, 2, 3]))
    assert cands[0].tolist() == [3, 4, 4, 5] and cands[1].tolist() == [9, 9]


# ---------------------------------------------------------------- O5/O6 Algorithm 2
def _golden_cases():
    with open(GOLDEN) as f:
        g = json.load(f)
    for c in g["cases"]:
        yield pytest.param(c, g["defaults"], id=c["name"])


@pytest.mark.parametrize("case,defaults", list(_golden_cases()))
def test_aggregation_golden(case, defaults):
    kw = dict(defaults)
    for key in ("tile_m", "top_c", "radius_m", "toler_pct"):
        if key in case:
            kw[key] = case[key]
    xy = np.array(case["xy"], dtype=np.float64)
    cand = np.array(case["cand"])
    det = aggregate.aggregate_details(cand, xy, mode="tile", **kw)
    exp = case["expect"]
    assert list(det["winner"]) == exp["tile"]
    assert det["status"] == exp["status"]
    assert det["C"] == exp["C"]
    t = kw["tile_m"]
    assert det["pos"] == ((exp["tile"][0] + 0.5) * t, (exp["tile"][1] + 0.5) * t)
    x, y, s = aggregate.aggregate_2d(cand, xy, mode="centroid", **kw)
    assert s == exp["status"]
    assert abs(x - exp["centroid"][0]) <= 1e-12 and abs(y - exp["centroid"][1]) <= 1e-12


def test_aggregation_is_permutation_invariant():
    rng = np.random.default_rng(16)
    xy = rng.uniform(0, 20, size=(200, 2))
    cand = rng.integers(0, 200, size=120)
    cand[:40] = 5          # a dense cluster
    base = aggregate.aggregate_2d(cand, xy, mode="centroid")
    for _ in range(5):
        p = rng.permutation(cand)
        got = aggregate.aggregate_2d(p, xy, mode="centroid")
        assert got[2] == base[2] and abs(got[0] - base[0]) < 1e-9 and abs(got[1] - base[1]) < 1e-9


def test_aggregation_ignores_padding_rows():
    xy = np.array([[1.0, 1.0]])
    assert aggregate.aggregate_2d([0, -1, -1], xy, mode="centroid") == (1.0, 1.0, 0)
    with pytest.raises(ValueError):
        aggregate.aggregate_2d([-1, -1], xy)


def test_circle_limit_for_paper_constants():
    # 3 m radius over 30 cm tiles = 10 tiles -> squared limit 100 (§3.2).
    assert aggregate.circle_r2_limit(3.0, 0.30) == 100
    assert aggregate.circle_r2_limit(1.0, 0.30) == 11      # (10/3)^2 = 11.1
    assert aggregate.circle_r2_limit(0.0, 0.30) == 0


def test_symmetric_clusters_give_the_midpoint():
    # Two equal clusters within one circle of each other: centroid is their midpoint.
    xy = np.array([[5.05, 5.05], [6.25, 5.05]])   # tiles (16,16) and (20,16)
    x, y, s = aggregate.aggregate_2d([0, 0, 0, 1, 1, 1], xy, mode="centroid")
    assert s == 0 and abs(x - 5.65) < 1e-12 and abs(y - 5.05) < 1e-12


def test_softmax_mode_limits():
    xy = np.array([[1.0, 2.0], [5.0, 6.0], [9.0, -1.0]])
    d = np.array([0.5, 0.25, 3.0])
    # tau -> 0: the nearest candidate's coordinates
    x, y, _ = aggregate.aggregate_2d([0, 1, 2], xy, d, mode="softmax", tau=1e-6)
    assert (x, y) == (5.0, 6.0)
    # tau -> inf: the plain mean
    x, y, _ = aggregate.aggregate_2d([0, 1, 2], xy, d, mode="softmax", tau=1e12)
    assert abs(x - 5.0) < 1e-9 and abs(y - 7.0 / 3.0) < 1e-9


# ---------------------------------------------------------------- low precision
def test_bf16_rounding_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(17)
    v = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10,
                        np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0, 1e-30],
                                 dtype=np.float32)])
    want = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(lowp.round_bf16(v), want)


def test_bf16_hand_values():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1.
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: ties to even -> 1 + 2^-6.
    got = lowp.round_bf16(np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8], dtype=np.float32))
    assert got.tolist() == [1.0, 1 + 2 ** -6]


def test_e4m3_hand_values():
    v = [0.5, 448.0, 500.0, -500.0, 2 ** -9, 2 ** -10, 3 * 2 ** -10, 17.0, 19.0, 1.0625, 1.1875, 0.0]
    # 17 lies halfway between 16 and 18 (step 2 in [16, 32)): even mantissa -> 16.
    # 19 lies halfway between 18 and 20: even -> 20. 1.0625 = 1 + 1/16: tie -> 1.
    # 1.1875 = 1 + 3/16: tie between 1.125 and 1.25 -> 1.25. 2^-10: tie 0 / 2^-9 -> 0.
    want = [0.5, 448.0, 448.0, -448.0, 2 ** -9, 0.0, 2 ** -8, 16.0, 20.0, 1.0, 1.25, 0.0]
    assert lowp.round_e4m3(np.array(v, dtype=np.float32)).tolist() == want


def test_e4m3_rounding_matches_torch_conversion_in_range():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8")
    rng = np.random.default_rng(18)
    v = (rng.standard_normal(20000) * 60).astype(np.float32)
    v = np.clip(v, -448, 448)
    want = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    assert np.array_equal(lowp.round_e4m3(v), want)


@pytest.mark.parametrize("fmt,rel", [("bf16", 2 ** -8), ("e4m3", 2 ** -4)])
def test_quantize_rows_reconstructs_within_format_precision(fmt, rel):
    rng = np.random.default_rng(19)
    X = rng.standard_normal((64, 32)).astype(np.float32)
    s, c = lowp.quantize_rows(X, fmt)
    assert np.abs(c).max() <= lowp.QMAX[fmt]
    amax = np.abs(X).max(1)
    err = np.abs(c * s[:, None] - X)
    # absolute error at most half a grid step of the element's binade (<= rel * |x|),
    # plus the subnormal step for tiny elements
    bound = rel * np.abs(X) + s[:, None] * (2.0 ** -10 if fmt == "e4m3" else 0.0) + 1e-7 * amax[:, None]
    assert (err <= bound).all()


def test_lowp_topk_with_full_width_equals_exhaustive():
    rng = np.random.default_rng(20)
    X = rng.standard_normal((300, 16)).astype(np.float32)
    Q = rng.standard_normal((4, 16)).astype(np.float32)
    ex_i, ex_d = retrieval.exhaustive_topk(Q, X, 8)
    for fmt in ("bf16", "e4m3"):
        i, d, short = lowp.lowp_topk(Q, X, fmt, width=300, k=8)
        assert (i == ex_i[:, 0]).all() and np.array_equal(d, ex_d[:, 0])
        assert sorted(short[0].tolist()) == list(range(300))


def test_lowp_score_equals_distance_on_exact_codes():
    # Rows and queries made of values exactly representable after scaling:
    # the low-precision score is then the exact squared distance.
    X = np.array([[448.0, -224.0, 0.0, 8.0], [1.0, 2.0, -4.0, 448.0]], dtype=np.float32)
    q = np.array([[448.0, 0.0, 0.0, 0.0]], dtype=np.float32)
    s, c = lowp.quantize_rows(X, "e4m3")
    sq, cq = lowp.quantize_queries(q, "e4m3")
    assert np.array_equal(c * s[:, None], X)
    sc = lowp.lowp_scores(q[0], sq, cq[0], s, c)
    assert np.allclose(sc, retrieval.sq_dist(q[0], X), rtol=0, atol=1e-9)


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_batch_scale_is_the_smallest_power_of_two_above_the_ratio(fmt):
    qmax = lowp.QMAX[fmt]
    rng = np.random.default_rng(23)
    for _ in range(200):
        Q = (rng.standard_normal((3, 8)) * 10.0 ** rng.uniform(-3, 3)).astype(np.float32)
        s = float(lowp.batch_scale(Q, fmt))
        ratio = float(np.float32(np.abs(Q).max()) / np.float32(qmax))
        f, _ = np.frexp(s)
        assert f == 0.5                        # a power of two
        assert s / 2 < ratio <= s              # the smallest one >= the ratio
    # ratio exactly a power of two: s equals it; an all-zero batch: 1; tiny: 2^-126
    assert lowp.batch_scale(np.array([[qmax * 0.25, -1e-3]], np.float32), fmt) == np.float32(0.25)
    assert lowp.batch_scale(np.zeros((2, 4), np.float32), fmt) == np.float32(1.0)
    assert lowp.batch_scale(np.array([[1e-40]], np.float32), fmt) == np.float32(2.0 ** -126)
    # the batch maximum, not each query's own, sets the scale
    Q = np.array([[qmax, 0.0], [1.0, 0.0]], np.float32)
    s, c = lowp.quantize_queries(Q, fmt)
    assert s == np.float32(1.0) and c[1, 0] == 1.0


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_query_codes_do_not_depend_on_the_batch_power_of_two(fmt):
    # With a power-of-two scale, s_Q q^ is the same whichever batch the query is
    # in (values away from the format's subnormal range).
    rng = np.random.default_rng(24)
    q = (rng.uniform(0.5, 2.0, (1, 16)) * rng.choice([-1.0, 1.0], (1, 16))).astype(np.float32)
    big = np.full((1, 16), 7.5, np.float32)
    s1, c1 = lowp.quantize_queries(q, fmt)
    s2, c2 = lowp.quantize_queries(np.concatenate([q, big]), fmt)
    assert s2 > s1
    assert np.array_equal(c1[0] * s1, c2[0] * s2)


# ---------------------------------------------------------------- soft retrieval
def _soft_problem(seed=21):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((60, 6)).astype(np.float32)
    xy = rng.uniform(0, 10, size=(60, 2))
    frames = rng.standard_normal((6, 6))
    offsets = np.array([0, 3, 6])
    y = rng.uniform(0, 10, size=(2, 2))
    w = rng.uniform(0.5, 1.5, size=6)
    return frames, offsets, X, xy, y, w


def test_soft_gradients_match_central_differences():
    frames, offsets, X, xy, y, w = _soft_problem()
    tau = 2.0
    base = soft.forward_backward(frames, offsets, X, xy, y, w, tau, k=4)
    idx = base["idx"]
    h = 1e-6

    def L(fr=frames, ww=w, t=tau):
        return soft.forward_backward(fr, offsets, X, xy, y, ww, t, idx=idx)["loss"]

    fd_tau = (L(t=tau + h) - L(t=tau - h)) / (2 * h)
    assert abs(fd_tau - base["dtau"]) <= 1e-6 * max(1.0, abs(fd_tau))
    for j in range(w.size):
        e = np.zeros_like(w); e[j] = h
        fd = (L(ww=w + e) - L(ww=w - e)) / (2 * h)
        assert abs(fd - base["dw"][j]) <= 1e-6 * max(1.0, abs(fd))
    for f, j in itertools.product(range(frames.shape[0]), range(frames.shape[1])):
        e = np.zeros_like(frames); e[f, j] = h
        fd = (L(fr=frames + e) - L(fr=frames - e)) / (2 * h)
        assert abs(fd - base["dq"][f, j]) <= 1e-6 * max(1.0, abs(fd))


def test_soft_small_tau_reduces_to_nearest_candidate():
    frames, offsets, X, xy, y, w = _soft_problem(22)
    out = soft.forward_backward(frames, offsets, X, xy, y, w, 1e-9, k=4)
    for b in range(2):
        fr = range(offsets[b], offsets[b + 1])
        best = min(((float((w * (frames[f] - X[i]) ** 2).sum()), i) for f in fr
                    for i in out["idx"][f]))
        assert np.allclose(out["yhat"][b], xy[best[1]], atol=1e-12)


def test_soft_loss_is_mean_squared_error():
    frames, offsets, X, xy, y, w = _soft_problem(23)
    out = soft.forward_backward(frames, offsets, X, xy, y, w, 1.0, k=3)
    mse = np.mean(np.sum((out["yhat"] - y) ** 2, axis=1))
    assert math.isclose(out["loss"], mse, rel_tol=1e-12)
