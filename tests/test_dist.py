"""The multi-process (N > 1) path of bench.py on CPU: two gloo ranks, as the
torchrun launch would start them. Each rank is a replica of the workload (the
roots partition with no data-path exchange), so the only collectives are the
timing reductions: the max of the elapsed times and the sum of the units."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.dist_env()
    d = bench.init_dist(w, "gloo")
    bench.barrier(d)
    elapsed, units = bench.aggregate(d, 1.0 + rank, 100.0 * (rank + 1))
    out.put((r, elapsed, units))
    # the reference arm: only rank 0 runs and prints; the others return at once
    if r != 0:
        assert bench.run_reference(None, w, r) is None
    d.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # max of (1.0, 2.0) and sum of (100, 200) on both ranks
    assert got == [(0, 2.0, 300.0), (1, 2.0, 300.0)]


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.init_dist(1, "gloo") is None
    assert bench.aggregate(None, 3.5, 42.0) == (3.5, 42.0)
