"""Routers spread over ranks (shard.py), on CPU gloo ranks: the reduce-scatter by recorder range,
the fold by elementwise minimum and the gather to the root give exactly the RSEA one process gets
by merging every router (Algorithm 5, min reading), and so the same list. The sketches come from
the oracle; the fold is a numpy minimum standing in for the library's kernel (the GPU tests check
that kernel), so what is tested here is the partition and the exchange."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ROUTERS = 5
SLOTS = 5


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    import trafficgen as tg
    W = tg.workload("tiny")
    W["traffic"].update(routers=ROUTERS, shared_frac=0.3, n_planted=12, count_a=400, count="fixed")
    return W


def _numpy_min(out, slices):
    import torch
    m = np.minimum.reduce([s.numpy().view(np.uint16) for s in slices])
    out.copy_(torch.from_numpy(m.view(np.int16)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import trafficgen as tg
    from paper_1803_11036_gb300 import shard
    try:
        W = _workload()
        p = oracle.params(W["params"])
        tabs = tg.hash_tables(W["hash_seed"])
        T = tg.Traffic(**W["traffic"])
        mine = [j for j in range(ROUTERS) if j % world == rank]
        sketches = [oracle.new_sketch(p) for _ in range(ROUTERS)]
        ranges = shard.estimator_ranges(p.r << p.q, p.eta, world)
        listed = 0
        for t in range(SLOTS):
            pairs = T.slot(t)
            for j in range(ROUTERS):       # every rank follows every router, to check the root
                if t:
                    oracle.advance(p, sketches[j])
                oracle.scan(p, tabs, sketches[j], pairs[j])
            local = oracle.merge(p, [sketches[j] for j in mine])
            full = torch.from_numpy(local.view(np.int16))
            got = shard.reduce_scatter_min(full, ranges, rank, _numpy_min)
            f, c = ranges[rank]
            want_range = oracle.merge(p, sketches)[f:f + c]
            assert np.array_equal(got.numpy().view(np.uint16), want_range), (rank, t)
            dest = torch.full((p.r * p.C * p.eta,), -1, dtype=torch.int16) if rank == 0 else None
            shard.gather_ranges(got, ranges, rank, 0, dest)
            if rank == 0:
                glob = dest.numpy().view(np.uint16)
                want = oracle.merge(p, sketches)
                assert np.array_equal(glob, want), t
                a = oracle.regain(p, tabs, glob, "pruned")
                b = oracle.regain(p, tabs, want, "pruned")
                assert np.array_equal(a["ips"], b["ips"]) and np.array_equal(a["rk"], b["rk"])
                listed += len(a["ips"])
        q.put((rank, "ok", listed))
    except Exception as e:  # reported to the parent
        q.put((rank, repr(e), 0))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_merge_equals_one_process_merge(world):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(r[1] == "ok" for r in res), res
    assert res[0][2] > 0       # the root regained sliding super points


def test_estimator_ranges_partition_whole_estimators():
    sys.path.insert(0, ROOT)
    from paper_1803_11036_gb300 import shard
    for n, eta, world in [(2560, 64, 3), (5 << 18, 2048, 8), (7, 32, 4), (3, 32, 5), (10, 8, 1)]:
        rg = shard.estimator_ranges(n, eta, world)
        assert len(rg) == world
        assert rg[0][0] == 0 and sum(c for _, c in rg) == n * eta
        for (f0, c0), (f1, _) in zip(rg, rg[1:]):
            assert f0 + c0 == f1                 # contiguous, in rank order
        sizes = [c // eta for _, c in rg]
        assert all(c % eta == 0 for _, c in rg) and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.estimator_ranges(10, 8, 0)
