"""Runs one library call repeatedly on a synthetic case, for profilers.

    python -m paper_2006_08861_gb300.profile_case CASE [--n N] [--dim D] [--nq Q] [--fmt bf16|fp8] [--reps R] [--time]

Cases: "scan" (exhaustive FP32 lhr_query on an n x D standard-normal
database, Q frames near database rows), "hier" (lhr_query_window: one window
of 5 frames on the 100,000 x 256 building-scale database, coarse prefix 32,
shortlist 512, k = 20), "lowp" (tensor-core lhr_query, Q frames, BF16/FP8
copies, re-rank width 64), "weighted" (lhr_query_weighted, Q frames, unit
weights), "soft" (the soft-retrieval selection: lhr_query_weighted with unit
weights for 256 windows x 5 frames, k = 32, on the 200,000 x 256 synthetic
floor-plan database). --time prints each kernel's mean device time (event pairs).
"""
import argparse
import os
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("case", choices=["scan", "hier", "lowp", "weighted", "soft"])
    ap.add_argument("--n", type=int, default=500_000)
    ap.add_argument("--dim", type=int, default=256)
    ap.add_argument("--nq", type=int, default=8)
    ap.add_argument("--k", type=int, default=20)
    ap.add_argument("--fmt", default="fp8", choices=["bf16", "fp8"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--time", action="store_true")
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import paper_2006_08861_gb300 as lhr

    dev = torch.device("cuda:0")
    rng = np.random.default_rng(0)
    if a.case == "hier":
        import synth
        db = synth.make_database(100_000, 256, seed=synth.db_seed(1))
        w = synth.make_windows(db, 1, 5, seed=synth.query_seed(1))
        h = lhr.lhr_build_db(db.feats, db.xy, coarse_dim=32)
        ft = torch.from_numpy(w.frames).to(dev)
        offs = torch.from_numpy(w.offsets).to(dev)
        call = lambda: lhr.lhr_query_window(h, ft, offs, 20, shortlist=512)
    elif a.case == "soft":
        import synth
        c = synth.CONFIGS["differentiation"]
        db = synth.make_database(c["n"], c["dim"], seed=synth.db_seed(c["index"]))
        w = synth.make_windows(db, c["nw"], c["m"], seed=synth.query_seed(c["index"]))
        h = lhr.lhr_build_db(db.feats, db.xy)
        ft = torch.from_numpy(w.frames).to(dev)
        wt = torch.ones(c["dim"], device=dev)
        call = lambda: lhr.lhr_query_weighted(h, ft, c["k"], wt)
    else:
        X = rng.standard_normal((a.n, a.dim), dtype=np.float32)
        h = lhr.lhr_build_db(X, np.zeros((a.n, 2)), lowp=3 if a.case == "lowp" else 0)
        qt = torch.from_numpy(X[rng.integers(0, a.n, a.nq)] + 0.05).to(dev)
        if a.case == "scan":
            call = lambda: lhr.lhr_query(h, qt, a.k)
        elif a.case == "lowp":
            call = lambda: lhr.lhr_query(h, qt, a.k, score=a.fmt, rerank_width=64)
        else:
            wt = torch.ones(a.dim, device=dev)
            call = lambda: lhr.lhr_query_weighted(h, qt, a.k, wt)
    for _ in range(a.reps):
        call()
    torch.cuda.synchronize()
    if a.time:
        lhr.lhr_profile_enable(True)
        for _ in range(10):
            call()
        torch.cuda.synchronize()
        lhr.lhr_profile_enable(False)
        for name in ("hier_fused", "scan_pilot", "wnorm", "scan_topk", "many_bound", "f16_prep", "sort_queries",
                     "f16_pilot", "f16_many", "many_select",
                     "small_topk", "coarse_kernel", "collect", "shortlist",
                     "aggregate", "quantize", "tc_pilot", "tau_kernel", "tc_main", "tc_full", "merge_rerank"):
            n, ms = lhr.lhr_profile_read(name, reset=True)
            if n:
                print(f"{a.case} {name}: {n} launches, mean {ms / n * 1e3:.1f} us")
    err = lhr.lhr_db_error(h)
    if err:
        raise SystemExit(f"device error word {err}")


if __name__ == "__main__":
    main()
