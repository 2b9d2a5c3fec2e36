"""Soft retrieval (differentiable form) on the GPU against the FP64 oracle:
the weighted selection (indices and distances under the parity rules), the
window softmax and positions, the loss, and the analytic gradients dq, dw,
dtau; central finite differences through the autograd functions; the
differentiation workload's shape (N = 200,000, B = 256 windows of m = 5,
k = 32) on sampled windows."""
import numpy as np
import pytest

import synth
from oracle import retrieval as oret
from oracle import soft
from tests.parity import check_list

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lhr():
    import paper_2006_08861_gb300 as m
    return m


def _weights(rng, dim):
    return rng.uniform(0.5, 1.5, dim).astype(np.float32)


@pytest.mark.parametrize("n,dim,nq,k,subs", [
    (3001, 64, 7, 16, None),      # ragged, no pilot
    (70_003, 32, 9, 32, None),    # pilot sample, two query blocks
    (80_000, 128, 5, 20, 3),      # pilot with subspaces
    (70_003, 128, 130, 32, None), # many frames: the register-tiled pass
])
def test_weighted_selection_matches_oracle(lhr, n, dim, nq, k, subs):
    rng = np.random.default_rng(n + dim)
    X = rng.standard_normal((n, dim)).astype(np.float32)
    Q = (X[rng.integers(0, n, nq)] + 0.3 * rng.standard_normal((nq, dim))).astype(np.float32)
    w = _weights(rng, dim)
    sub = None if subs is None else rng.integers(0, subs, n).astype(np.int32)
    db = lhr.lhr_build_db(X, np.zeros((n, 2)), subspace=sub)
    gi, gd = lhr.lhr_query_weighted(db, torch.from_numpy(Q).cuda(), k, torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    assert lhr.lhr_db_error(db) == 0
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    oi, od = oret.exhaustive_topk(Q, X, k + 1, subspace=sub, n_subspaces=subs, w=w)
    for qi in range(nq):
        for s in range(gi.shape[1]):
            rows = None if sub is None else np.nonzero(sub == s)[0]
            check_list(Q[qi], X, gi[qi, s], gd[qi, s], oi[qi, s], od[qi, s], k, rows=rows, where=f"q{qi} s{s}", w=w)


def test_unit_weights_equal_plain_scan(lhr):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((5000, 64)).astype(np.float32)
    q = torch.from_numpy(X[:6] + 0.1 * rng.standard_normal((6, 64)).astype(np.float32)).cuda()
    db = lhr.lhr_build_db(X, np.zeros((5000, 2)))
    i1, d1 = lhr.lhr_query(db, q, 12)
    i2, d2 = lhr.lhr_query_weighted(db, q, 12, torch.ones(64, device="cuda"))
    torch.cuda.synchronize()
    assert torch.equal(i1, i2) and torch.equal(d1, d2)


def test_negative_weight_is_recorded(lhr):
    rng = np.random.default_rng(4)
    X = rng.standard_normal((500, 16)).astype(np.float32)
    db = lhr.lhr_build_db(X, np.zeros((500, 2)))
    w = torch.ones(16, device="cuda")
    w[3] = -1.0
    lhr.lhr_query_weighted(db, torch.from_numpy(X[:2]).cuda(), 5, w)
    assert lhr.lhr_db_error(db) == lhr.LHR_ERR_INVALID_ARG


def _problem(seed, n=4000, dim=32, nw=6, m=4, k=8):
    db = synth.make_database(n, dim, seed=seed)
    win = synth.make_windows(db, nw, m, seed=seed + 1)
    rng = np.random.default_rng(seed + 2)
    w = rng.uniform(0.7, 1.3, dim).astype(np.float32)
    return db, win, w, k


def _forward(lhr, h, win, w, tau, k):
    frames = torch.from_numpy(win.frames).cuda()
    offs = torch.from_numpy(win.offsets).cuda()
    wt = torch.from_numpy(w).cuda()
    tt = torch.tensor([tau], dtype=torch.float32, device="cuda")
    return frames, offs, wt, tt, lhr.lhr_soft_forward(h, frames, offs, k, wt, tt)


@pytest.mark.parametrize("tau", [0.1, 1.0, 10.0])
def test_forward_backward_match_fp64_oracle(lhr, tau):
    db, win, w, k = _problem(50)
    h = lhr.lhr_build_db(db.feats, db.xy)
    frames, offs, wt, tt, (idx, dist, p, yhat) = _forward(lhr, h, win, w, tau, k)
    gi = idx.cpu().numpy()[:, 0, :]
    oi, od = oret.exhaustive_topk(win.frames, db.feats, k + 1, w=w)
    for f in range(win.frames.shape[0]):
        check_list(win.frames[f], db.feats, gi[f], dist.cpu().numpy()[f, 0], oi[f, 0], od[f, 0], k, where=f"f{f}", w=w)
    y = win.true_xy.astype(np.float64)
    ref = soft.forward_backward(win.frames, win.offsets, db.feats, db.xy, y, w.astype(np.float64), float(np.float32(tau)),
                                idx=gi)
    assert np.allclose(yhat.cpu().numpy(), ref["yhat"], rtol=0, atol=1e-6)
    yt = torch.from_numpy(y).cuda()
    loss, _ = lhr.lhr_loc_mse(yhat, yt)
    _, g = lhr.lhr_loc_mse(yhat, yt, loss=False, grad=True)
    assert abs(loss.item() - ref["loss"]) <= 1e-9 + 1e-6 * ref["loss"]
    dq, dw, dtau = lhr.lhr_soft_backward(h, frames, offs, k, wt, tt, idx, dist, p, yhat, g)
    torch.cuda.synchronize()
    assert lhr.lhr_db_error(h) == 0

    def close(a, b, name):
        a = np.asarray(a, dtype=np.float64)
        scale = max(np.max(np.abs(b)), 1e-12)
        err = np.max(np.abs(a - b)) / scale
        assert err < 2e-4, f"{name}: max error {err:.3g} of the largest entry"

    close(dq.cpu().numpy(), ref["dq"], "dq")
    close(dw.cpu().numpy(), ref["dw"], "dw")
    close(dtau.cpu().numpy()[0], np.array(ref["dtau"]), "dtau")


def test_autograd_against_central_differences(lhr):
    # h = 1e-3 on a few coordinates of w, tau and the frames; samples whose
    # top-k sets change under +-h are skipped (the selection is held fixed)
    db, win, w, k = _problem(60, nw=4, m=3, k=6)
    h = lhr.lhr_build_db(db.feats, db.xy)
    y = torch.from_numpy(win.true_xy.astype(np.float64)).cuda()
    offs = torch.from_numpy(win.offsets).cuda()
    frames0 = torch.from_numpy(win.frames).cuda()
    w0 = torch.from_numpy(w).cuda()
    tau0 = torch.tensor([1.0], device="cuda")

    def loss_of(frames, wv, tv):
        yhat = lhr.soft_retrieval(h, frames, offs, wv, tv, k)
        return lhr.loc_mse(yhat, y)

    fr = frames0.clone().requires_grad_(True)
    wv = w0.clone().requires_grad_(True)
    tv = tau0.clone().requires_grad_(True)
    L = loss_of(fr, wv, tv)
    L.backward()
    base_idx = lhr.lhr_soft_forward(h, frames0, offs, k, w0, tau0)[0]

    def fd(which, i, step=1e-3):
        vals = []
        for sgn in (1, -1):
            f2, w2, t2 = frames0.clone(), w0.clone(), tau0.clone()
            tgt = {"q": f2.view(-1), "w": w2, "tau": t2}[which]
            tgt[i] += sgn * step
            idx2 = lhr.lhr_soft_forward(h, f2, offs, k, w2, t2)[0]
            if not torch.equal(idx2, base_idx):
                return None
            with torch.no_grad():
                vals.append(loss_of(f2, w2, t2).item())
        return (vals[0] - vals[1]) / (2 * step)

    checked = 0
    for which, grad, coords in (("w", wv.grad, [0, 5, 17]), ("tau", tv.grad, [0]),
                                ("q", fr.grad.view(-1), [3, 40, 100])):
        for i in coords:
            est = fd(which, i)
            if est is None:
                continue
            an = grad[i].item()
            assert abs(est - an) <= 2e-2 * max(abs(an), 1e-3) + 2e-4, f"{which}[{i}]: fd {est} vs analytic {an}"
            checked += 1
    assert checked >= 4


def test_invalid_tau_and_window(lhr):
    db, win, w, k = _problem(70, nw=2, m=2, k=4)
    h = lhr.lhr_build_db(db.feats, db.xy)
    frames, offs, wt, _, _ = _forward(lhr, h, win, w, 1.0, k)
    lhr.lhr_db_error(h)
    _, _, _, yhat = lhr.lhr_soft_forward(h, frames, offs, k, wt, torch.tensor([-1.0], device="cuda"))
    assert torch.isnan(yhat).all()
    assert lhr.lhr_db_error(h) == lhr.LHR_ERR_INVALID_ARG
    with pytest.raises(lhr.LhrError):
        lhr.lhr_soft_forward(h, frames, offs, 0, wt, torch.tensor([1.0], device="cuda"))


def test_differentiation_workload_sampled(lhr):
    # N = 200,000 x 256, B = 256 windows of m = 5, k = 32, w = 1, tau = 0.1:
    # forward + backward; sampled windows against the FP64 oracle
    spec = synth.CONFIGS["differentiation"]
    db = synth.make_database(spec["n"], spec["dim"], seed=synth.db_seed(spec["index"]))
    win = synth.make_windows(db, spec["nw"], spec["m"], seed=synth.query_seed(spec["index"]))
    h = lhr.lhr_build_db(db.feats, db.xy)
    k = spec["k"]
    w = np.ones(spec["dim"], np.float32)
    frames, offs, wt, tt, (idx, dist, p, yhat) = _forward(lhr, h, win, w, 0.1, k)
    y = win.true_xy.astype(np.float64)
    _, g = lhr.lhr_loc_mse(yhat, torch.from_numpy(y).cuda(), loss=False, grad=True)
    dq, dw, dtau = lhr.lhr_soft_backward(h, frames, offs, k, wt, tt, idx, dist, p, yhat, g)
    torch.cuda.synchronize()
    assert lhr.lhr_db_error(h) == 0
    gi = idx.cpu().numpy()[:, 0, :]
    gd = dist.cpu().numpy()[:, 0, :]
    for b in (0, 77, 255):
        fr = np.arange(win.offsets[b], win.offsets[b + 1])
        oi, od = oret.exhaustive_topk(win.frames[fr], db.feats, k + 1, w=w)
        for j, f in enumerate(fr):
            check_list(win.frames[f], db.feats, gi[f], gd[f], oi[j, 0], od[j, 0], k, where=f"b{b} f{f}", w=w)
        sub_off = np.array([0, fr.size], dtype=np.int32)
        ref = soft.forward_backward(win.frames[fr], sub_off, db.feats, db.xy, y[b:b + 1], w.astype(np.float64),
                                    float(np.float32(0.1)), idx=gi[fr])
        assert np.allclose(yhat.cpu().numpy()[b], ref["yhat"][0], atol=1e-6)
        # this window's frames: dq is B-scaled in the full batch (g = 2 (y^ - y) / B)
        scale = 1.0 / spec["nw"]
        dq_ref = ref["dq"] * scale
        err = np.max(np.abs(dq.cpu().numpy()[fr] - dq_ref)) / max(np.max(np.abs(dq_ref)), 1e-12)
        assert err < 2e-4, f"window {b}: dq error {err:.3g}"
    # dw and dtau sum over all 256 windows (the library reduces them in a fixed order): the FP64
    # oracle's gradients over every window, with the GPU's selection held fixed
    ref = soft.forward_backward(win.frames, win.offsets, db.feats, db.xy, y, w.astype(np.float64),
                                float(np.float32(0.1)), idx=gi)
    dw_err = np.max(np.abs(dw.cpu().numpy() - ref["dw"])) / max(np.max(np.abs(ref["dw"])), 1e-30)
    assert dw_err < 2e-4, f"dw error {dw_err:.3g}"
    dtau_ref = ref["dtau"]
    assert abs(float(dtau.cpu().numpy()[0]) - dtau_ref) <= 2e-4 * abs(dtau_ref) + 1e-9, (dtau, dtau_ref)
    assert np.allclose(yhat.cpu().numpy(), ref["yhat"], atol=1e-6)
    h.close()
