"""The bench's multi-rank logic on two gloo ranks (CPU, no GPU).

Ranks are replicas: each simulates its own event (seed offset by the rank) and the job's
throughput is every rank's work over the slowest rank's time.  The reference arm runs on
rank 0 only; other ranks return without work.
"""
import argparse
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_2104_08265_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = [120.0, 150.0][rank]                 # per-rank total time of the timed steps
        m = bench.max_over_ranks(ms, ws, "cpu")
        v = bench.job_throughput(ws, 10, 1000, m)
        seed = bench.rank_params(synth.DriftParams(seed=5), rank).seed
        ran_reference = None
        if rank == 1:
            args = argparse.Namespace(workload="plane128-2k", steps=1, warmup=0, gpus=ws)
            bench.run_reference(args)              # must return at once on rank 1
            ran_reference = False
        q.put((rank, m, v, bench.dist_env(), seed, ran_reference))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_offset_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in procs:
            rank, m, v, env, seed, ref = q.get(timeout=120)
            out[rank] = (m, v, env, seed, ref)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    for rank in (0, 1):
        m, v, env, seed, _ = out[rank]
        assert m == 150.0                                   # the slowest rank's time
        assert v == pytest.approx(2 * 10 * 1000 / 0.150)    # all ranks' depos over it
        assert env == (2, rank, rank)
        assert seed == 5 + rank                             # one event per rank
    assert out[1][4] is False


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_throughput(1, 4, 250, 1000.0) == pytest.approx(1000.0)
