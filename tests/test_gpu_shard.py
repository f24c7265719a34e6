"""The GPU side of routers spread over ranks (shard.py): the min-merge kernel that folds received
recorder ranges (ssd_min_merge) against numpy's minimum on ragged sizes and every input count up to
the limit, and the whole end of slot - local merge, reduce-scatter by range, gather, regain,
advance - against the oracle. Only one GPU is available, so the exchange runs as one NCCL rank;
several ranks are emulated on the one GPU by folding each range of their local merges with the
same kernel, one after the other (no kernel waits for another)."""
import os
import socket

import numpy as np
import pytest

import oracle
import paper_1803_11036_gb300 as ssd
import trafficgen as tg
from gpu_harness import to_dev
from paper_1803_11036_gb300 import _abi, shard

pytestmark = pytest.mark.gpu


def _u16(rng, n):
    return rng.integers(0, 65536, n, dtype=np.uint32).astype(np.uint16)


@pytest.mark.parametrize("n_in", [1, 3, 9, 128])
@pytest.mark.parametrize("count", [0, 5, 8, 1000, 1_000_003])
def test_min_merge_kernel(n_in, count):
    import torch
    W = tg.workload("tiny")
    ctx = ssd.Context(ssd.make_params(W["params"]), tg.hash_tables(W["hash_seed"]))
    rng = np.random.default_rng(count + n_in)
    host = [_u16(rng, count) for _ in range(n_in)]
    if count > 8:   # runs of 65535 (never touched) and 0 (touched this slot), as in real sketches
        host[0][: count // 3] = 65535
        host[-1][count // 2: count // 2 + 7] = 0
    dev = [torch.from_numpy(h.view(np.int16)).cuda() for h in host]
    out = torch.empty(count, dtype=torch.int16, device="cuda")
    ctx.min_merge(out, dev)
    want = np.minimum.reduce(host) if count else np.empty(0, np.uint16)
    assert np.array_equal(out.cpu().numpy().view(np.uint16), want)
    ctx.min_merge(dev[0], dev)               # in place into one of the inputs
    assert np.array_equal(dev[0].cpu().numpy().view(np.uint16), want)
    ctx.close()


def test_min_merge_refuses_unaligned_and_too_many():
    import torch
    W = tg.workload("tiny")
    ctx = ssd.Context(ssd.make_params(W["params"]), tg.hash_tables(W["hash_seed"]))
    buf = torch.zeros(64, dtype=torch.int16, device="cuda")
    with pytest.raises(ssd.SSDError) as e:
        ctx.min_merge(buf[1:33], [buf[1:33]])       # 2-byte offset: not 16-byte aligned
    assert e.value.code == _abi.SSD_EINVAL
    with pytest.raises(ssd.SSDError) as e:
        ctx.min_merge(buf[:8], [buf[:8]] * (ssd.SSD_MAX_ROUTERS + 1))
    assert e.value.code == _abi.SSD_EINVAL
    ctx.close()


@pytest.mark.parametrize("world", [2, 3, 5])
def test_emulated_ranks_fold_to_the_merged_rsea(world):
    """Routers dealt round-robin to `world` emulated ranks: each rank's local merge (ssd_merge),
    then each range folded from every rank's slice of it (ssd_min_merge), equals the merge of
    every router and the oracle's global RSEA, slot after slot."""
    import torch
    W = tg.workload("edge_small")
    p = oracle.params(W["params"])
    tabs = tg.hash_tables(W["hash_seed"])
    ctx = ssd.Context(ssd.make_params(W["params"]), tabs)
    T = tg.Traffic(**W["traffic"])
    R = T.routers
    routers = [ctx.sketch() for _ in range(R)]
    locals_ = [ctx.sketch() for _ in range(world)]
    pipe = oracle.Pipeline(p, tabs, R)
    ranges = shard.estimator_ranges(p.r << p.q, p.eta, world)
    for t in range(4):
        pairs = T.slot(t)
        pipe.step(pairs, regain_method=None)
        if t:
            ctx.advance(routers)
        ctx.scan_batch(routers, [to_dev(x) for x in pairs])
        for rank in range(world):
            mine = [routers[j] for j in range(R) if j % world == rank]
            if mine:
                ctx.merge(mine, locals_[rank])
        views = [locals_[rank].export_device() for rank in range(world) if any(j % world == rank for j in range(R))]
        glob = torch.empty(p.r * p.C * p.eta, dtype=torch.int16, device="cuda")
        for f, c in ranges:
            ctx.min_merge(glob[f:f + c], [v[f:f + c] for v in views])
        torch.cuda.synchronize()
        assert np.array_equal(glob.cpu().numpy().view(np.uint16), pipe.global_sk), t
    ctx.close()


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_detector_one_nccl_rank():
    """ShardedDetector end to end on one NCCL rank: lists, R_k and the global RSEA equal the
    oracle's every slot, and the routers advance."""
    import torch
    import torch.distributed as dist
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0, world_size=1,
                            device_id=torch.device("cuda", 0))
    try:
        W = tg.workload("edge_small")
        p = oracle.params(W["params"])
        tabs = tg.hash_tables(W["hash_seed"])
        ctx = ssd.Context(ssd.make_params(W["params"]), tabs)
        T = tg.Traffic(**W["traffic"])
        routers = [ctx.sketch() for _ in range(T.routers)]
        det = shard.ShardedDetector(ctx, routers)
        pipe = oracle.Pipeline(p, tabs, T.routers)
        found = 0
        for t in range(W["slots"]):
            pairs = T.slot(t)
            want = pipe.step(pairs, "pruned")
            ctx.scan_batch(routers, [to_dev(x) for x in pairs])
            ips, rk = det.close_slot()
            assert np.array_equal(ips, want["ips"]) and np.array_equal(rk, want["rk"]), t
            assert np.array_equal(det.glob.export(), pipe.global_sk), t
            found += len(ips)
        assert found > 0 and routers[0].slot == W["slots"]
        det.close()
        ctx.close()
    finally:
        dist.destroy_process_group()
