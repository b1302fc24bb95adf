"""The benchmark's multi-rank logic on CPU: two gloo ranks, each with its own replica
field, agree on the slowest rank's time (no data-path collective exists to test)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import argparse
    import bench
    t = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
    cfg = bench.config_of(argparse.Namespace(config=4, size=8, rel=1e-3, tier=None))
    f, fh, xi = bench.workload(cfg, rank)
    assert cfg["seed"] + rank == bench.replica_seed(rank)
    q.put((rank, t, bench.replica_seed(rank), float(f.sum()), xi))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_distinct_fields():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert [g[1] for g in got] == [20.0, 20.0]
    assert got[0][2] != got[1][2]
    assert got[0][3] != got[1][3]


def test_single_process_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
