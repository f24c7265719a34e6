"""The bench's multi-process path on CPU: two gloo ranks reduce their timings (max) and packet
counts (sum) the way `bench.py` does under torchrun, and each rank gets an independent replica of
the workload (same detector parameters, its own traffic seed)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, _ = bench.dist_env()
    ms = bench.max_over_ranks(10.0 * (rank + 1), world)
    pk = bench.sum_over_ranks(1000.0 * (rank + 1), world)
    W = bench.replica_workload("corelink_c2", rank)
    bench.barrier(world)
    q.put((rank, w, r, ms, pk, W["traffic"]["seed"], W["params"]))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_replicate():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[2] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert all(x[3] == 20.0 for x in res)          # max over ranks
    assert all(x[4] == 3000.0 for x in res)        # sum over ranks
    assert res[0][5] != res[1][5]                   # independent traffic per replica
    assert res[0][6] == res[1][6]                   # same detector parameters


def test_single_process_defaults(golden):
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5 and bench.sum_over_ranks(2.0, 1) == 2.0
    g = golden["throughput_units"]   # Sec. 5: 109 Mpps at 800 B reported as 681.25 Gb/s
    assert bench.gbps(g["mpps"])["paper_convention"] == pytest.approx(g["gbps_paper_convention"])
