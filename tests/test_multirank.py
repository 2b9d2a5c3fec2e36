"""The N > 1 launch path of bench.py on CPU: two gloo ranks (127.0.0.1) shard
the independent units without overlap or gap, agree on the max-over-ranks
time, and pass the barrier; the reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        lo, hi = bench.shard(1001, r, w)
        t = bench.max_over_ranks(float(10 + 5 * r), w)
        bench.barrier(w)
        q.put((r, w, local, lo, hi, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_agree():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, lo0, hi0, t0), (r1, w1, l1, lo1, hi1, t1) = out
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert lo0 == 0 and hi0 == lo1 and hi1 == 1001 and abs((hi0 - lo0) - (hi1 - lo1)) <= 1
    assert t0 == t1 == 15.0


def test_shard_covers_every_unit_once():
    import bench
    for n in (0, 1, 7, 64, 1001):
        for world in (1, 2, 3, 8):
            spans = [bench.shard(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def test_reference_arm_runs_on_rank_zero_only():
    import bench
    spec = bench.workload_spec("tiny")

    class A:
        warmup, steps = 3, 1

    assert bench.run_reference(A, spec, rank=1, world=2) is None
