#!/usr/bin/env python
"""Throughput benchmark of the localization hot path on synthetic data.

Default workload ("hierarchical"): N = 100,000 database locations, D = 256
FP32 features, coarse prefix 32, shortlist 512, top k = 20, windows of m = 5
consecutive frames, Algorithm 2 per window; one window per library call
(lhr_query_window with nw = 1: coarse kernel, shortlist/re-rank kernel,
aggregation kernel). A step is B = 64 such windows back to back on one stream,
captured once into a CUDA graph and replayed; L2 is flushed (a 256 MB write)
before every step, outside the timed events. The metric is localization
queries (windows) per second over all ranks.

Other workloads (--workload): "hbm_scan" (plain FP32 exhaustive scan of a
2,000,000 x 256 database, 8 frames per pass, k = 20) and "tiny" (2,000 x 128,
16 single-frame queries, k = 10, centroid aggregation).

--impl reference times the FP64 CPU oracle on the same workload instead.
Under torchrun every rank processes its own windows (no collective on the data
path); the elapsed time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "queries/s and % of HBM/TC roofline, low-precision vs FP32 at recall@k≥0.999; p99"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of each workload's dominant
# kernel, from one ncu capture of the current kernel: hier_fused_kernel on this very workload;
# scan_topk_kernel on 500,000 x 256 rows (517.4 MB), scaled by rows to the 2,000,000-row launch;
# tc_main_kernel (FP8) at the full 2,000,000 rows (single metrics: one pass).
# Re-measure (or set None) whenever the kernel changes.
TRAFFIC = {"hierarchical": ("hier_fused_kernel", 14.02e6), "hbm_scan": ("scan_topk_kernel", 4 * 517.4e6),
           "precision": ("tc_main_kernel", 531.3e6 + 5.8e6)}


# ------------------------------------------------------------------ ranks
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard(n: int, rank: int, world: int):
    """Contiguous share [start, stop) of n independent units for this rank."""
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(x: float, world: int) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ workloads
def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


def workload_spec(name: str) -> dict:
    import synth
    if name == "hierarchical":
        c = synth.CONFIGS["hierarchical"]
        return dict(name=name, n=c["n"], dim=c["dim"], coarse_dim=c["coarse_dim"], shortlist=c["shortlist"],
                    k=c["k"], m=c["m"], per_step=64, mode="tile", seed_db=1001, seed_q=2001,
                    unit="windows/s", desc="N=100000 D=256 FP32, coarse prefix 32, shortlist 512, k=20, "
                                           "windows of m=5 frames (0.3 m apart, sigma 0.05), one window per "
                                           "lhr_query_window call, Algorithm 2 tile mode")
    if name == "tiny":
        c = synth.CONFIGS["tiny"]
        return dict(name=name, n=c["n"], dim=c["dim"], coarse_dim=0, shortlist=0, k=c["k"], m=1, per_step=16,
                    mode="centroid", seed_db=1000, seed_q=2000, batch_windows=16, unit="queries/s",
                    desc="N=2000 D=128 FP32, 16 single-frame queries per call, exhaustive k=10, centroid")
    if name == "hbm_scan":
        c = synth.CONFIGS["precision"]
        return dict(name=name, n=c["n"], dim=c["dim"], coarse_dim=0, shortlist=0, k=20, m=1, per_step=8,
                    mode=None, seed_db=1002, seed_q=2002, unit="queries/s",
                    desc="N=2000000 D=256 FP32 exhaustive scan, 8 query frames per pass, k=20")
    raise SystemExit(f"unknown workload {name}")


def make_inputs(spec, n_windows, rank):
    import synth
    db = synth.make_database(spec["n"], spec["dim"], seed=spec["seed_db"])
    if spec["name"] == "hierarchical":
        win = synth.make_windows(db, n_windows, spec["m"], seed=spec["seed_q"] + 7919 * rank)
        return db, win.frames, win.offsets
    q, _, _ = synth.make_point_queries(db, n_windows, seed=spec["seed_q"] + 7919 * rank)
    return db, q, np.arange(n_windows + 1, dtype=np.int32)


# ------------------------------------------------------------------ oracle timing
def oracle_unit(spec, db, frames, offsets, w):
    """The oracle's answer for one unit (window / query) of the workload."""
    from oracle import aggregate as oagg
    from oracle import retrieval as oret
    fr = frames[offsets[w]:offsets[w + 1]]
    if spec["shortlist"]:
        idx, _, _ = oret.hierarchical_topk(fr, db.feats, spec["coarse_dim"], spec["shortlist"], spec["k"])
    else:
        idx, _ = oret.exhaustive_topk(fr, db.feats, spec["k"])
        idx = idx[:, 0]
    if spec["mode"] is None:
        return idx
    return oagg.aggregate_2d(idx.reshape(-1), db.xy, mode=spec["mode"])


def time_oracle(spec, db, frames, offsets, budget_s: float, max_units: int):
    t0 = time.perf_counter()
    done = 0
    while done < max_units:
        oracle_unit(spec, db, frames, offsets, done)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return done / el, done, el


# ------------------------------------------------------------------ ours
def run_ours(args, spec, rank, world, local):
    import torch
    import paper_2006_08861_gb300 as lhr

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    B = spec["per_step"]
    n_units = (args.warmup + args.steps) * B
    db, frames, offsets = make_inputs(spec, n_units, rank)
    h = lhr.lhr_build_db(db.feats, db.xy, coarse_dim=spec["coarse_dim"])
    stream = torch.cuda.current_stream()
    k = spec["k"]
    m = spec["m"]
    d_frames = torch.from_numpy(frames).to(dev)
    one_off = torch.tensor([0, m], dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # output buffers for one step
    if spec["name"] == "hbm_scan":
        out_idx = torch.empty((B, 1, k), dtype=torch.int64, device=dev)
        out_dist = torch.empty((B, 1, k), dtype=torch.float32, device=dev)
    else:
        bw = spec.get("batch_windows", 1)
        out_idx = torch.empty((B * m, 1, k), dtype=torch.int64, device=dev)
        out_dist = torch.empty((B * m, 1, k), dtype=torch.float32, device=dev)
        out_xy = torch.empty((B, 2), dtype=torch.float64, device=dev)
        out_st = torch.empty((B,), dtype=torch.int32, device=dev)
        unit_offs = torch.arange(bw + 1, dtype=torch.int32, device=dev)

    src = torch.empty((B * m, spec["dim"]), dtype=torch.float32, device=dev)

    def issue_step(frames_dev):
        """All library calls of one step (reads `frames_dev`, B units)."""
        if spec["name"] == "hbm_scan":
            lhr.lhr_query(h, frames_dev, k, out=(out_idx, out_dist))
            return 1  # the scan kernel (+ the pilot-sample kernel on large databases: counted below)
        if spec["name"] == "tiny":
            lhr.lhr_query_window(h, frames_dev, unit_offs, k, mode=spec["mode"],
                                 out=(out_idx, out_dist, out_xy, out_st))
            return 2
        launches = 0
        for w in range(B):
            lhr.lhr_query_window(h, frames_dev[w * m:(w + 1) * m], one_off, k, shortlist=spec["shortlist"],
                                 mode=spec["mode"],
                                 out=(out_idx[w * m:(w + 1) * m], out_dist[w * m:(w + 1) * m],
                                      out_xy[w:w + 1], out_st[w:w + 1]))
            launches += 1 if m <= 8 else 4  # fused single launch for requests of <= 8 frames
        return launches

    def load_step(i):
        src.copy_(d_frames[i * B * m:(i + 1) * B * m], non_blocking=True)

    # CUDA graph of one step (the library's launches, replayed without host overhead)
    graph = None
    if not args.no_graph:
        load_step(0)
        issue_step(src)  # warm: pools, function attributes
        torch.cuda.synchronize()
        try:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                launches_per_step = issue_step(src)
        except Exception as e:  # capture unsupported: time eager launches instead
            print(f"# graph capture failed ({e}); timing eager launches", file=sys.stderr)
            graph = None
    if graph is None:
        launches_per_step = issue_step(src)
    torch.cuda.synchronize()

    def replay():
        if graph is not None:
            graph.replay()
        else:
            issue_step(src)

    for i in range(args.warmup):
        load_step(i)
        replay()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    host_t0 = time.perf_counter()
    for i in range(args.steps):
        load_step(args.warmup + i)
        flush.zero_()                       # L2 flush between timed iterations
        torch.cuda.synchronize()
        barrier(world)
        ev0[i].record(stream)
        replay()
        ev1[i].record(stream)
        torch.cuda.synchronize()
    host_el = time.perf_counter() - host_t0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    total_ms = max_over_ranks(sum(step_ms), world)
    units = B * args.steps * world
    value = units / (total_ms / 1e3)

    # per-unit latency (device time of one unit's launches, graph-replayed, warm L2)
    lat = []
    if spec["name"] == "hierarchical":
        g1 = None
        if graph is not None:
            g1 = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g1):
                lhr.lhr_query_window(h, src[:m], one_off, k, shortlist=spec["shortlist"], mode=spec["mode"],
                                     out=(out_idx[:m], out_dist[:m], out_xy[:1], out_st[:1]))
        for i in range(400):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if g1 is not None:
                g1.replay()
            else:
                lhr.lhr_query_window(h, src[:m], one_off, k, shortlist=spec["shortlist"], mode=spec["mode"],
                                     out=(out_idx[:m], out_dist[:m], out_xy[:1], out_st[:1]))
            b.record(stream)
            b.synchronize()
            lat.append(a.elapsed_time(b) * 1e3)

    # dominant kernel: event-timed per launch in an instrumented pass of the same steps
    lhr.lhr_profile_read(None, reset=True)
    lhr.lhr_profile_enable(True)
    for i in range(args.steps):
        load_step(args.warmup + i)
        flush.zero_()
        issue_step(src)
    torch.cuda.synchronize()
    lhr.lhr_profile_enable(False)
    kern = {}
    for name in ("hier_fused_kernel", "coarse_kernel", "collect_kernel", "shortlist_kernel", "aggregate_kernel",
                 "scan_pilot", "scan_topk_kernel", "small_topk_kernel"):
        cnt, tot = lhr.lhr_profile_read(name, reset=True)
        if cnt:
            kern[name] = (cnt, tot)
    # the library's own launch count per step (every kernel is under a profiling scope)
    launches_per_step = max(launches_per_step, round(sum(v[0] for v in kern.values()) / args.steps))
    dom = max(kern, key=lambda n: kern[n][1])
    n_launch, tot_ms = kern[dom]
    avg_s = tot_ms / n_launch / 1e3
    D, Dc, S = spec["dim"], spec["coarse_dim"], spec["shortlist"]
    if dom == "hier_fused_kernel":
        # one window per launch: the coarse slab plus the shortlisted rows of its m frames
        alg_bytes = spec["n"] * Dc * 4 + m * S * D * 4
    elif dom == "coarse_kernel":
        alg_bytes = spec["n"] * Dc * 4 + m * D * 4
    elif dom == "shortlist_kernel":
        alg_bytes = S * D * 4 + D * 4           # one frame's shortlist rows per CTA; m CTAs per launch
        alg_bytes *= m
    elif dom in ("scan_topk_kernel", "small_topk_kernel"):
        alg_bytes = spec["n"] * D * 4 + (B if spec["name"] == "hbm_scan" else B * m) * D * 4
    else:
        alg_bytes = m * k * 8
    hbm_peak, _, peak_src = load_peaks()
    achieved = alg_bytes / avg_s / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm_peak,
                "peak_source": peak_src, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                "traffic": (TRAFFIC[spec["name"]][1] if spec["name"] in TRAFFIC and TRAFFIC[spec["name"]][0] == dom
                            else None),
                "avg_launch_us": round(avg_s * 1e6, 3),
                "algorithmic_bytes_per_launch": alg_bytes,
                "kernel_share": {n: round(v[1] / sum(x[1] for x in kern.values()), 4) for n, v in kern.items()}}

    # end to end through the public API with host buffers (pinned), per step:
    # H2D of the step's frames, the library calls (eager, as a user makes them),
    # D2H of the step's results.
    host_frames = torch.from_numpy(frames).pin_memory()
    if spec["name"] == "hbm_scan":
        host_out = torch.empty((B, 1, k), dtype=torch.int64).pin_memory()
        d2h_bytes = host_out.numel() * 8
    else:
        host_xy = torch.empty((B, 2), dtype=torch.float64).pin_memory()
        host_st = torch.empty((B,), dtype=torch.int32).pin_memory()
        d2h_bytes = B * 16 + B * 4
    e2e_steps = min(args.steps, 10)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        j = args.warmup + i
        src.copy_(host_frames[j * B * m:(j + 1) * B * m], non_blocking=True)
        issue_step(src)
        if spec["name"] == "hbm_scan":
            host_out.copy_(out_idx, non_blocking=True)
        else:
            host_xy.copy_(out_xy, non_blocking=True)
            host_st.copy_(out_st, non_blocking=True)
        torch.cuda.synchronize()
    e2e_el = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": round(B * e2e_steps * world / e2e_el, 1), "unit": spec["unit"],
           "h2d_bytes_per_step": B * m * spec["dim"] * 4, "d2h_bytes_per_step": d2h_bytes,
           "path": "Python binding -> C ABI, eager launches, pinned host buffers"}
    err = lhr.lhr_db_error(h)
    if err != 0:
        raise SystemExit(f"device error word {err}")

    # CPU baseline: the FP64 oracle on a bounded sample of the same units (rank 0)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ncpu = os.cpu_count()
        v, done, el = time_oracle(spec, db, frames, offsets, budget_s=args.cpu_budget, max_units=n_units)
        cpu = {"value": round(v, 3), "unit": spec["unit"], "cores": 1, "kind": "oracle",
               "sample": f"{done} units of the same workload in {el:.1f} s (numpy FP64, one thread; "
                         f"{ncpu} host cores present)"}

    out = {
        "metric": METRIC, "value": round(value, 1), "unit": spec["unit"], "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": spec["name"], "desc": spec["desc"], "units_per_step": B,
                   "l2": "flushed (256 MB write) before every timed step",
                   "launch": "CUDA graph of the step's library launches" if graph is not None else "eager",
                   "parallelism": f"replicas x{world}, independent windows per rank"},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
        "host_wall_s": round(host_el, 3),
    }
    if lat:
        lat.sort()
        out["latency_us"] = {"p50": round(lat[len(lat) // 2], 2), "p99": round(lat[int(len(lat) * 0.99)], 2),
                             "what": "device time of one window (graph-replayed, warm L2)"}
    h.close()
    return out


def run_precision(args, rank, world, local):
    """N = 2,000,000 x 256 database, 1,024 query frames per batch: the BF16 and
    FP8 tensor-core forms (top-64 shortlist by score, FP32 re-rank to k = 20)
    next to the plain FP32 scan on the same data; recall@20 against that FP32
    scan on every query and against the FP64 oracle on sampled queries."""
    import torch
    import paper_2006_08861_gb300 as lhr
    import synth
    from oracle import retrieval as oret

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    c = synth.CONFIGS["precision"]
    db = synth.make_database(c["n"], c["dim"], seed=1002)
    nq, k, W = c["nq"], c["k"], c["rerank_width"]
    batches = args.warmup + args.steps
    q_all, rows_all, xy_all = synth.make_point_queries(db, nq * min(batches, 4), seed=2002 + 7919 * rank)
    h = lhr.lhr_build_db(db.feats, db.xy, lowp=3)
    qd = torch.from_numpy(q_all).to(dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out_i = torch.empty((nq, 1, k), dtype=torch.int64, device=dev)
    out_d = torch.empty((nq, 1, k), dtype=torch.float32, device=dev)
    n_sets = q_all.shape[0] // nq

    def batch(i):
        return qd[(i % n_sets) * nq:(i % n_sets + 1) * nq]

    forms = {}
    results = {}
    for form in ("f32", "bf16", "fp8"):
        kw = {} if form == "f32" else dict(score=form, rerank_width=W)
        for i in range(args.warmup):
            lhr.lhr_query(h, batch(i), k, out=(out_i, out_d), **kw)
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        ms = []
        for i in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            barrier(world)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lhr.lhr_query(h, batch(args.warmup + i), k, out=(out_i, out_d), **kw)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        clk = clocks.stop()
        tot = max_over_ranks(sum(ms), world)
        lhr.lhr_query(h, batch(0), k, out=(out_i, out_d), **kw)
        torch.cuda.synchronize()
        results[form] = out_i.cpu().numpy()[:, 0].copy()
        forms[form] = {"queries_per_s": round(nq * args.steps * world / (tot / 1e3), 1),
                       "ms_per_batch": round(tot / args.steps, 4), "clocks": clk}
    ex = results["f32"]
    true_xy = xy_all[:nq]
    for form in ("bf16", "fp8"):
        got = results[form]
        forms[form]["recall@20_vs_fp32_scan"] = round(float(np.mean(
            [len(set(got[i]) & set(ex[i])) / k for i in range(nq)])), 6)
        forms[form]["top1_location_error_m"] = round(float(np.mean(np.hypot(*(db.xy[got[:, 0]] - true_xy).T))), 4)
    forms["f32"]["top1_location_error_m"] = round(float(np.mean(np.hypot(*(db.xy[ex[:, 0]] - true_xy).T))), 4)
    # FP64 oracle on sampled queries
    sample = [0, 511] if not args.no_cpu_baseline else []
    t0 = time.perf_counter()
    for qi in sample:
        o_idx, _ = oret.exhaustive_topk(q_all[qi:qi + 1], db.feats, k)
        for form in ("f32", "bf16", "fp8"):
            forms[form].setdefault("recall@20_vs_fp64_oracle_sampled", [])
            forms[form]["recall@20_vs_fp64_oracle_sampled"].append(len(set(results[form][qi]) & set(o_idx[0, 0])) / k)
    oracle_s = time.perf_counter() - t0
    # dominant kernel of the FP8 form: the main tensor-core pass, event-timed
    lhr.lhr_profile_read(None, reset=True)
    lhr.lhr_profile_enable(True)
    for i in range(args.steps):
        flush.zero_()
        lhr.lhr_query(h, batch(i), k, out=(out_i, out_d), score="fp8", rerank_width=W)
    torch.cuda.synchronize()
    lhr.lhr_profile_enable(False)
    share = {}
    for name in ("quantize", "tc_pilot", "tau_kernel", "tc_main", "tc_full", "merge_rerank"):
        n_l, t_ms = lhr.lhr_profile_read(name, reset=True)
        if n_l:
            share[name] = (n_l, t_ms)
    n_main, t_main = share.get("tc_main", (1, float("nan")))
    flops = 2.0 * nq * c["n"] * c["dim"]
    _, bf16_peak, src = load_peaks()
    fp8_peak = 2.0 * bf16_peak  # measured BF16 burst x the nominal FP8/BF16 ratio (4.5 / 2.25)
    achieved = flops / (t_main / n_main / 1e3) / 1e12
    best = "fp8" if forms["fp8"]["recall@20_vs_fp32_scan"] >= 0.999 else "bf16"
    cpu = None
    if not args.no_cpu_baseline and sample:
        cpu = {"value": round(len(sample) / oracle_s, 4), "unit": "queries/s", "cores": 1, "kind": "oracle",
               "sample": f"{len(sample)} queries, exhaustive FP64 over 2,000,000 rows (numpy, one thread)"}
    tot_all = sum(v[1] for v in share.values())
    out = {
        "metric": METRIC, "value": forms[best]["queries_per_s"], "unit": "queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": forms[best]["ms_per_batch"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp8" if best == "fp8" else "bf16",
        "data": "synthetic",
        "config": {"workload": "precision", "desc": "N=2000000 D=256, Q=1024 per batch, per-row scaled BF16/FP8 "
                                                    "copies, top-64 by tensor-core score, FP32 re-rank to k=20",
                   "l2": "flushed before every timed batch", "form_reported": best},
        "forms": forms,
        "roofline": {"bound": "tensor", "kernel": "tc_main (fp8)", "achieved": round(achieved, 1),
                     "peak": round(fp8_peak, 1), "peak_source": f"{src} bf16 burst x 2 (nominal fp8/bf16)",
                     "unit": "TFLOP/s", "frac": round(achieved / fp8_peak, 4), "traffic": TRAFFIC["precision"][1],
                     "avg_launch_us": round(t_main / n_main * 1e3, 2),
                     "algorithmic_flops_per_launch": flops,
                     "kernel_share": {n: round(v[1] / tot_all, 4) for n, v in share.items()}},
        "cpu_baseline": cpu,
        "clocks": forms[best].get("clocks"),  # sampled during the reported form's timed batches
        # per batch: query scale, query codes, pilot, tau, main, fallback (exits at once), merge + re-rank
        "gpu_launches": 7 * args.steps,
    }
    h.close()
    return out


def run_differentiation(args, rank, world, local):
    """N = 200,000 x 256 database, B = 256 windows of m = 5 frames, k = 32,
    w = 1, tau = 0.1: one step is the soft retrieval's forward (weighted
    selection + window softmax), the location loss, and the backward (dq, dw,
    dtau), through the autograd functions a user calls."""
    import torch
    import paper_2006_08861_gb300 as lhr
    import synth
    from oracle import soft

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    c = synth.CONFIGS["differentiation"]
    db = synth.make_database(c["n"], c["dim"], seed=synth.db_seed(c["index"]))
    B, m, k = c["nw"], c["m"], c["k"]
    n_sets = 2
    win = synth.make_windows(db, B * n_sets, m, seed=synth.query_seed(c["index"]) + 7919 * rank)
    h = lhr.lhr_build_db(db.feats, db.xy)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    frames_all = torch.from_numpy(win.frames).to(dev)
    y_all = torch.from_numpy(win.true_xy.astype(np.float64)).to(dev)
    offs = torch.arange(0, (B + 1) * m, m, dtype=torch.int32, device=dev)
    w = torch.ones(c["dim"], dtype=torch.float32, device=dev, requires_grad=True)
    tau = torch.full((1,), 0.1, dtype=torch.float32, device=dev, requires_grad=True)

    def step(i):
        j = i % n_sets
        fr = frames_all[j * B * m:(j + 1) * B * m].clone().requires_grad_(True)
        yhat = lhr.soft_retrieval(h, fr, offs, w, tau, k)
        loss = lhr.loc_mse(yhat, y_all[j * B:(j + 1) * B])
        loss.backward()
        return loss, fr

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms = []
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier(world)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(args.warmup + i)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    clk = clocks.stop()
    tot = max_over_ranks(sum(ms), world)
    # per-kernel shares in an instrumented pass
    lhr.lhr_profile_read(None, reset=True)
    lhr.lhr_profile_enable(True)
    for i in range(args.steps):
        flush.zero_()
        step(i)
    torch.cuda.synchronize()
    lhr.lhr_profile_enable(False)
    share = {}
    for name in ("wnorm_kernel", "scan_pilot", "scan_topk_kernel", "many_bound_kernel", "many_kernel",
                 "many_select_kernel", "soft_forward_kernel", "soft_backward_kernel"):
        n_l, t_ms = lhr.lhr_profile_read(name, reset=True)
        if n_l:
            share[name] = (n_l, t_ms)
    # the selection's main kernel: the many-frame pass (>= 64 frames) or the streaming scan
    sel = "many_kernel" if "many_kernel" in share else "scan_topk_kernel"
    n_scan, t_scan = share.get(sel, (1, float("nan")))
    # the selection is FP32 SIMT arithmetic: 3 flops per (frame, row, dim) (sub, fma)
    flops = 3.0 * B * m * c["n"] * c["dim"]
    alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x 2 flops x max SM clock (GHz), TFLOP/s
    achieved = 2.0 * B * m * c["n"] * c["dim"] / (t_scan / n_scan / 1e3) / 1e12
    # gradient check of one window against the FP64 oracle (selection from the GPU)
    loss, fr = step(0)
    g_fr = fr.grad.detach().cpu().numpy()
    idx = lhr.lhr_soft_forward(h, frames_all[:B * m], offs, k, w.detach(), tau.detach())[0].cpu().numpy()[:, 0]
    ref = soft.forward_backward(win.frames[:m], np.array([0, m], np.int32), db.feats, db.xy,
                                win.true_xy[:1].astype(np.float64), np.ones(c["dim"]), float(np.float32(0.1)),
                                idx=idx[:m])
    dq_err = float(np.max(np.abs(g_fr[:m] - ref["dq"] / B)) / max(np.max(np.abs(ref["dq"] / B)), 1e-30))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t0 = time.perf_counter()
        soft.forward_backward(win.frames[:m], np.array([0, m], np.int32), db.feats, db.xy,
                              win.true_xy[:1].astype(np.float64), np.ones(c["dim"]), 0.1, k=k)
        el = time.perf_counter() - t0
        cpu = {"value": round(1.0 / el, 4), "unit": "windows/s (fwd+bwd)", "cores": 1, "kind": "oracle",
               "sample": "1 window of 5 frames: exhaustive FP64 weighted selection over 200,000 rows, softmax, "
                         "analytic gradients (numpy, one thread)"}
    tot_all = sum(v[1] for v in share.values())
    out = {
        "metric": METRIC, "value": round(B * args.steps * world / (tot / 1e3), 1), "unit": "windows/s (fwd+bwd)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "differentiation", "desc": "N=200000 D=256, B=256 windows of m=5, k=32, w=1, "
                                                          "tau=0.1: soft retrieval forward + location loss + backward",
                   "l2": "flushed before every timed step", "launch": "eager (autograd)"},
        "roofline": {"bound": "alu", "kernel": f"{sel} (weighted selection)",
                     "achieved": round(achieved, 2), "peak": round(alu_peak, 1),
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (derived)", "unit": "TFLOP/s",
                     "frac": round(achieved / alu_peak, 4), "traffic": None,
                     "avg_launch_us": round(t_scan / n_scan * 1e3, 1),
                     "algorithmic_flops_per_launch": 2.0 * B * m * c["n"] * c["dim"],
                     "kernel_share": {n: round(v[1] / tot_all, 4) for n, v in share.items()}},
        "grad_check": {"dq_max_rel_err_vs_fp64_window0": dq_err, "loss": float(loss.item())},
        "cpu_baseline": cpu,
        "clocks": clk,
        "gpu_launches": round(sum(v[0] for v in share.values()) / args.steps) + 2,
    }
    h.close()
    return out


def run_serving(args, rank, world, local):
    """N = 1,000,000 x 256 database (coarse prefix 32, shortlist 512, k = 20,
    Algorithm 2 tile mode); 64 user streams, each sending frames with
    exponential inter-arrival times (15 frames/s per stream) and asking, with
    every frame, for the position of its last m frames, m uniform in 3..10.
    The server batches continuously; the arrivals are replayed at 1x, 10x and
    100x speed and all at once (saturation). Beside it, the per-request path:
    each window alone through lhr_query_window, one after another."""
    import torch
    import paper_2006_08861_gb300 as lhr
    import synth

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    c = synth.CONFIGS["serving"]
    db = synth.make_database(c["n"], c["dim"], seed=synth.db_seed(c["index"]))
    h = lhr.lhr_build_db(db.feats, db.xy, coarse_dim=32)
    n_streams, fps, k, S = c["streams"], c["fps"], c["k"], 512
    rng = np.random.default_rng(synth.query_seed(c["index"]) + 7919 * rank)
    per_stream = 64
    walks = [synth.make_windows(db, 1, per_stream, seed=synth.query_seed(c["index"]) + 100 * s + 7919 * rank).frames
             for s in range(n_streams)]
    # arrival schedule: (time s, stream, frame index, window m)
    events = []
    for s in range(n_streams):
        t = 0.0
        for f in range(per_stream):
            t += rng.exponential(1.0 / fps)
            events.append((t, s, f, int(rng.integers(c["m_lo"], c["m_hi"] + 1))))
    events.sort()
    levels = {}

    def run_level(speed):
        srv = lhr.Server(h, n_streams=n_streams, max_window=c["m_hi"], k=k, shortlist=S, max_batch_frames=64,
                         n_lanes=3, mem_budget_bytes=2 << 30)
        t0 = time.perf_counter()
        for i, (t, s, f, m) in enumerate(events):
            if speed is not None:
                due = t0 + t / speed
                while True:
                    now = time.perf_counter()
                    if now >= due:
                        break
                    if due - now > 2e-4:
                        time.sleep(due - now - 1e-4)
            srv.submit(s, walks[s][f], window_m=m, request_id=i)
        srv.drain(600000)
        el = time.perf_counter() - t0
        res = srv.poll(max_results=4096)
        while len(res) < len(events):
            more = srv.poll(wait_ms=100)
            if not more:
                break
            res += more
        srv.close()
        lat = sorted(r["latency_us"] for r in res)
        offered = None if speed is None else round(n_streams * fps * speed, 1)
        return {"windows_per_s": round(len(res) / el, 1), "offered_windows_per_s": offered,
                "p50_us": round(lat[len(lat) // 2], 1), "p99_us": round(lat[int(len(lat) * 0.99)], 1),
                "windows": len(res)}

    run_level(None)  # warm: pools, function attributes
    clocks = ClockSampler(local)
    clocks.start()
    for name, speed in (("1x", 1.0), ("10x", 10.0), ("100x", 100.0), ("saturation", None)):
        if name == "1x" and args.steps < 10:
            continue  # the real-time replay takes the schedule's length (about 4 s); skipped on short runs
        levels[name] = run_level(speed)
    clk = clocks.stop()
    # per-request path: every window alone, synchronously, on a sample of the schedule
    sample = events[:min(len(events), 400)]
    lat = []
    offs = torch.tensor([0, 0], dtype=torch.int32, device=dev)
    frames_dev = [torch.from_numpy(w).to(dev) for w in walks]
    t0 = time.perf_counter()
    for (t, s, f, m) in sample:
        lo = max(0, f - m + 1)
        offs[1] = f + 1 - lo
        a = time.perf_counter()
        lhr.lhr_query_window(h, frames_dev[s][lo:f + 1], offs, k, shortlist=S)
        torch.cuda.synchronize()
        lat.append((time.perf_counter() - a) * 1e6)
    el = time.perf_counter() - t0
    lat.sort()
    per_req = {"windows_per_s": round(len(sample) / el, 1), "p50_us": round(lat[len(lat) // 2], 1),
               "p99_us": round(lat[int(len(lat) * 0.99)], 1), "windows": len(sample),
               "path": "lhr_query_window per window, synchronous, coarse-to-fine FP32"}
    sat = levels["saturation"]
    total = max_over_ranks(len(events) / sat["windows_per_s"], world)
    out = {
        "metric": METRIC, "value": round(len(events) * world / total, 1), "unit": "windows/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 / sat["windows_per_s"], 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serving", "desc": "N=1000000 D=256, coarse prefix 32, shortlist 512, k=20; 64 "
                                                  "streams x 15 fps, Poisson arrivals, window m uniform 3..10 per "
                                                  "request, one window per frame; continuous batching (<= 64 "
                                                  "frames per tick, 3 lanes)",
                   "value_is": "saturation throughput (all arrivals at once)"},
        "load_levels": levels, "per_request_fp32": per_req,
        "latency_us": {"p50": sat["p50_us"], "p99": sat["p99_us"], "what": "submit -> result on the host, saturation"},
        "clocks": clk, "cpu_baseline": None,
        "gpu_launches": None,
    }
    h.close()
    return out


def run_reference(args, spec, rank, world):
    """The FP64 oracle as the reference arm: each step is a bounded sample."""
    if rank != 0:
        return None
    B = 2 if spec["name"] == "hierarchical" else (1 if spec["name"] == "hbm_scan" else spec["per_step"])
    n_units = (args.warmup + args.steps) * B
    db, frames, offsets = make_inputs(spec, n_units, 0)
    for i in range(args.warmup):
        for w in range(i * B, (i + 1) * B):
            oracle_unit(spec, db, frames, offsets, w)
    t0 = time.perf_counter()
    for i in range(args.warmup, args.warmup + args.steps):
        for w in range(i * B, (i + 1) * B):
            oracle_unit(spec, db, frames, offsets, w)
    el = time.perf_counter() - t0
    v = B * args.steps / el
    sample = f"{B} units per step x {args.steps} steps (numpy FP64, one thread)"
    return {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": spec["unit"], "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": spec["name"], "desc": spec["desc"]},
            "cpu_baseline": {"value": round(v, 3), "unit": spec["unit"], "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 3), "unit": spec["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="hierarchical",
                    choices=["hierarchical", "tiny", "hbm_scan", "precision", "differentiation", "serving"])
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work for cpu_baseline")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    if args.workload in ("precision", "differentiation", "serving"):
        run = {"precision": run_precision, "differentiation": run_differentiation,
               "serving": run_serving}[args.workload]
        out = None if args.impl == "reference" else run(args, rank, world, local)
        if args.impl == "reference" and rank == 0:
            out = {"impl": "reference", "unavailable": f"the {args.workload} workload's reference arm is the FP64 "
                                                       "oracle; run --workload hierarchical for the timed reference"}
    else:
        spec = workload_spec(args.workload)
        if args.impl == "reference":
            out = run_reference(args, spec, rank, world)
        else:
            out = run_ours(args, spec, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
