"""bench.py's multi-GPU form on two gloo ranks, on the CPU.

The solver does not shard: for N GPUs bench.py runs N replicas, each rank
serving its own frame sequences (no collective on the data path), and reports
the frames of all ranks over the slowest rank's timed region.  These tests run
exactly the functions bench.py uses for that (per-rank sequence seeds, the
max-over-ranks timing reduction, the whole-job value) as two gloo processes.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, streams, steps, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            init_method=f"tcp://127.0.0.1:{port}")
    try:
        env = bench.dist_env()
        seeds = bench.stream_seeds(rank, streams)
        local_ms = 100.0 + 37.5 * rank             # rank 1 is the slow replica
        slowest = bench.max_over_ranks(local_ms, world)
        value = bench.whole_job_fps(world, streams, steps, slowest)
        every = [None] * world
        dist.all_gather_object(every, seeds)
        q.put({"rank": rank, "env": env, "seeds": seeds, "slowest": slowest, "value": value,
               "every": every})
    finally:
        dist.destroy_process_group()


def test_replicas_on_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port, world, streams, steps = _free_port(), 2, 8, 8
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, streams, steps, q))
             for r in range(world)]
    for p in procs:
        p.start()
    try:
        out = sorted((q.get(timeout=180) for _ in procs), key=lambda r: r["rank"])
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    for r, res in enumerate(out):
        assert res["env"] == (r, world, r)
        # the slowest rank's timed region, seen identically by every rank
        assert res["slowest"] == 137.5
        assert res["value"] == pytest.approx(world * streams * steps / 0.1375, rel=1e-12)
        assert len(set(res["seeds"])) == streams
    # no two streams of the job animate the same sequence
    allseeds = [sd for lst in out[0]["every"] for sd in lst]
    assert len(set(allseeds)) == world * streams
    assert out[0]["every"] == out[1]["every"]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_fps(1, 8, 8, 1000.0) == pytest.approx(64.0)
    assert bench.stream_seeds(0, 3) == [3, 4, 5]
    assert bench.stream_seeds(1, 3) == [6, 7, 8]
