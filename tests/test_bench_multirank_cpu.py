"""The bench's multi-rank plumbing (one process per GPU, replicas only: no collective on the data
path) on CPU with the gloo backend and world size 2: process-group set-up from the torchrun
environment variables, the barrier, and the whole-job rate (every rank's units over the slowest
rank's time, computed with a SUM and a MAX all-reduce)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "LGP_BENCH_BACKEND": "gloo"})
    import importlib.util
    import torch
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    r, w, local = bench.dist_init(world)
    bench.barrier(w)
    # rank 0 did 3e9 units in 2 s, rank 1 did 5e9 units in 4 s: 8e9 units over the slowest 4 s
    units, secs = (3e9, 2.0) if r == 0 else (5e9, 4.0)
    rate, total = bench.job_rate(units, secs, w, torch.device("cpu"))
    mx = bench.max_over_ranks(secs, w, torch.device("cpu"))
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, w, rate, total, mx))


def test_two_gloo_ranks_aggregate_like_the_bench():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, rate, total, mx in out:
        assert w == 2
        assert total == pytest.approx(4.0) and mx == pytest.approx(4.0)
        assert rate == pytest.approx(8e9 / 4.0)
    assert sorted(o[0] for o in out) == [0, 1]


def test_single_rank_needs_no_process_group():
    import importlib.util
    import torch
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.job_rate(6e9, 3.0, 1, torch.device("cpu")) == (2e9, 3.0)
