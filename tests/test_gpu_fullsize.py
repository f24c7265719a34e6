"""Parity at the full size of the benchmark workload (one core-link router, 6.25 M packets per
slot, q = 18, a 5 GiB RSEA), in the launch configuration bench.py times: ssd_scan then
ssd_close_slot with no global sketch, every slot.

The full RSEA is too large for the oracle to hold and advance slot by slot, so the oracle follows
a sample of estimators through every packet (Algorithm 2 and the recorder update restricted to
them) and decides, for a sample of hosts, whether each is a sliding super point. With the RHFG[0]
check on, a host is in the list exactly when all r of its estimators RHFG[i](x) are hot and the
union of the r has R_k >= the threshold, which the sampled estimators decide completely."""
import numpy as np
import pytest

import oracle
import paper_1803_11036_gb300 as ssd
import trafficgen as tg
from gpu_harness import to_dev

pytestmark = pytest.mark.gpu

SLOTS = 24


def test_corelink_full_size_sampled():
    import torch
    W = tg.workload("corelink_c2")
    prm = W["params"]
    tabs = tg.hash_tables(W["hash_seed"])
    T = tg.traffic_for(W)
    # A: the bench configuration (literal regain, routers only); B: the same traffic with the
    # RHFG[0] check and the merged sketch written every slot.
    ctx_a = ssd.Context(ssd.make_params(prm), tabs)
    ctx_b = ssd.Context(ssd.make_params(prm, ssd.SSD_VERIFY_H0), tabs)
    ra, rb, gb = ctx_a.sketch(), ctx_b.sketch(), ctx_b.sketch()
    slots = T.fill_many([(t, 0) for t in range(SLOTS)])
    la = lb = None
    for t in range(SLOTS):
        dev = to_dev(slots[t])
        ctx_a.scan(ra, dev)
        la = ctx_a.close_slot([ra])
        ctx_b.scan(rb, dev)
        lb = ctx_b.close_slot([rb], gb)
        del dev
    torch.cuda.synchronize()
    # the two configurations hold the same routers, and the checked list is inside the literal one
    n_rec = ctx_a.sketch_bytes // 2
    for off in range(0, n_rec, 1 << 28):
        c = min(1 << 28, n_rec - off)
        assert np.array_equal(ra.export(off, c), rb.export(off, c)), off
    assert set(lb[0].tolist()) <= set(la[0].tolist())
    assert len(lb[0]) > 10

    p = oracle.params(prm, oracle.VERIFY_H0)
    thr, _ = oracle.threshold(p.eta, p.theta)
    rng = np.random.default_rng(5)
    hosts = set(T.planted_ips().tolist()) | set(lb[0].tolist()) | set(la[0][:50].tolist())
    hosts |= {T.lib.tg_src_ip(T._h, int(s)) for s in rng.integers(0, W["traffic"]["n_src"], 200)}
    hosts = sorted(hosts)
    cols = {x: oracle.rhfg(p, tabs, x) for x in hosts}
    rows = np.concatenate([np.arange(p.r, dtype=np.uint32) for _ in hosts])
    cc = np.concatenate([cols[x] for x in hosts]).astype(np.uint32)
    extra_c = rng.integers(0, p.C, 64).astype(np.uint32)
    extra_r = rng.integers(0, p.r, 64).astype(np.uint32)
    sampled = oracle.Sampled(p, np.concatenate([rows, extra_r]), np.concatenate([cc, extra_c]))
    for t in range(SLOTS):
        if t:
            sampled.advance()
        sampled.scan(tabs, slots[t])
    # state after the last slot's close = one more advance
    sampled.advance()
    for row, col in list(zip(extra_r.tolist(), extra_c.tolist())) + [(i, int(cols[hosts[0]][i])) for i in range(p.r)]:
        assert np.array_equal(ra.export_estimator(row, col), sampled.get(row, col)), (row, col)
    # membership and R_k of every sampled host in the checked list (pre-advance recorders:
    # recorder < k before the advance is recorder < k + 1 after it, with 65535 staying 65535)
    got = dict(zip(lb[0].tolist(), lb[1].tolist()))
    checked_in = 0
    for x in hosts:
        below = [sampled.get(i, int(cols[x][i])) < p.k + 1 for i in range(p.r)]
        rks = [int(b.sum()) for b in below]
        union = int(np.logical_and.reduce(below).sum())
        member = all(v >= thr for v in rks) and union >= thr
        assert (x in got) == member, hex(x)
        if member:
            assert got[x] == union, hex(x)
            checked_in += 1
    assert checked_in == len(lb[0])   # every listed host was sampled and confirmed
    ctx_a.close()
    ctx_b.close()
