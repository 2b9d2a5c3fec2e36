"""lhr_query_static: the exhaustive FP32 query for callers that cannot allocate
device memory (its scratch is a fixed device array inside the library).

Kept in a file that sorts last, so a run that stops at the first failure has
already run every other test. It builds its own database, so it passes alone
in a fresh process as well as after the rest of the suite.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_static_scratch_query_matches_lhr_query_twice_in_a_row():
    import paper_2006_08861_gb300 as lhr
    db = synth.make_database(20_000, 256, seed=77)
    h = lhr.lhr_build_db(db.feats, db.xy)
    k = 20
    # two calls in a row with different inputs: the second must not see the
    # first one's leftovers in the shared scratch array
    for call, nq in enumerate((12, 5)):
        q, _, _ = synth.make_point_queries(db, nq, seed=700 + call)
        qt = torch.from_numpy(q).cuda()
        ref_idx, ref_dist = lhr.lhr_query(h, qt, k)
        idx = torch.full((nq, 1, k), -7, dtype=torch.int64, device="cuda")
        dist = torch.full((nq, 1, k), -7.0, dtype=torch.float32, device="cuda")
        lhr.lhr_query_static(h, qt, k, out=(idx, dist))
        torch.cuda.synchronize()
        assert np.array_equal(idx.cpu().numpy(), ref_idx.cpu().numpy()), call
        np.testing.assert_allclose(dist.cpu().numpy(), ref_dist.cpu().numpy(), rtol=1e-5, atol=0)
    assert lhr.lhr_db_error(h) == 0


def test_static_scratch_rejects_requests_beyond_its_size():
    import paper_2006_08861_gb300 as lhr
    db = synth.make_database(20_000, 256, seed=78)
    h = lhr.lhr_build_db(db.feats, db.xy)
    nq, k = 4096, 32
    q = torch.zeros((nq, 256), device="cuda")
    idx = torch.empty((nq, 1, k), dtype=torch.int64, device="cuda")
    dist = torch.empty((nq, 1, k), dtype=torch.float32, device="cuda")
    with pytest.raises(lhr.LhrError) as e:
        lhr.lhr_query_static(h, q, k, out=(idx, dist))
    assert e.value.status == lhr.LHR_ERR_INVALID_ARG
    assert "scratch" in lhr.lhr_last_error()
