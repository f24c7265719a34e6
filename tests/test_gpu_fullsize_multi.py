"""Parity at the full size of the many-router workloads, in the launch configuration bench.py
times for them (one ssd_scan_batch over every router, then one ssd_close_slot):

- 16 edge routers, lognormal packet counts, 30 % of sources at several routers (17 RSEAs of
  5 GiB with the merged one), under the merge tile the autotuner picked for it (groups of 2) and
  under the defaults;
- 32 routers, 15.6 M packets per slot with ten hot sources (33 RSEAs, 165 GiB).

The oracle cannot hold these sketches, so it follows a sample of estimators of every router
through every packet (Algorithm 2 and the recorder update restricted to them), merges them by the
elementwise minimum (Algorithm 5) and decides, for a sample of hosts, whether each is a sliding
super point: with the RHFG[0] check on, a host is listed exactly when its r merged estimators are
all hot and their union has R_k >= the threshold, which the sampled estimators decide completely.
In the 32-router run the planted hosts gain about 4 peers per slot against a 300-slot window, so
no host reaches the threshold in the slots run here; the test then checks the sketch state and
that neither side lists anything."""
import numpy as np
import pytest

import oracle
import paper_1803_11036_gb300 as ssd
import trafficgen as tg
from gpu_harness import to_dev

pytestmark = pytest.mark.gpu


def advanced(v):
    return np.where(v < 0xFFFF, v + 1, v).astype(np.uint16)


def run_gpu(ctx, routers, glob, slots):
    lst = None
    for pairs in slots:
        devs = [to_dev(x) for x in pairs]
        ctx.scan_batch(routers, devs)
        lst = ctx.close_slot(routers, glob)
        del devs
    return lst


def sampled_oracle(p, tabs, slots, hosts, n_extra=48, seed=5):
    """Per-router sampled estimators after the last slot's scan (before its advance)."""
    rng = np.random.default_rng(seed)
    cols = {x: oracle.rhfg(p, tabs, x) for x in hosts}
    rows = np.concatenate([np.arange(p.r, dtype=np.uint32) for _ in hosts] +
                          [rng.integers(0, p.r, n_extra).astype(np.uint32)])
    cc = np.concatenate([cols[x].astype(np.uint32) for x in hosts] +
                        [rng.integers(0, p.C, n_extra).astype(np.uint32)])
    R = len(slots[0])
    samp = [oracle.Sampled(p, rows, cc) for _ in range(R)]
    for t, pairs in enumerate(slots):
        for j in range(R):
            if t:
                samp[j].advance()
            samp[j].scan(tabs, pairs[j])
    extra = list(zip(rows[-n_extra:].tolist(), cc[-n_extra:].tolist()))
    return samp, cols, extra


def check(p, tabs, samp, cols, extra, hosts, routers, glob, got):
    thr, _ = oracle.threshold(p.eta, p.theta)
    R = len(samp)

    def merged(row, col):
        return np.minimum.reduce([s.get(row, col) for s in samp])

    probe = extra + [(i, int(cols[hosts[0]][i])) for i in range(p.r)]
    for row, col in probe:
        assert np.array_equal(glob.export_estimator(row, col), merged(row, col)), (row, col)
        for j in sorted({0, R // 2, R - 1}):
            assert np.array_equal(routers[j].export_estimator(row, col), advanced(samp[j].get(row, col))), (j, row, col)
    listed = dict(zip(got[0].tolist(), got[1].tolist()))
    members = 0
    for x in hosts:
        below = [merged(i, int(cols[x][i])) < p.k for i in range(p.r)]
        rks = [int(b.sum()) for b in below]
        union = int(np.logical_and.reduce(below).sum())
        member = all(v >= thr for v in rks) and union >= thr
        assert (x in listed) == member, hex(x)
        if member:
            assert listed[x] == union, hex(x)
            members += 1
    return members


def sample_hosts(T, W, got, n_random=150, seed=7):
    rng = np.random.default_rng(seed)
    hosts = set(T.planted_ips().tolist()[:300]) | set(got[0].tolist())
    hosts |= {T.lib.tg_src_ip(T._h, int(s)) for s in rng.integers(0, W["traffic"]["n_src"], n_random)}
    if T.n_hot:
        hosts |= set(T.hot_ips().tolist())
    return sorted(hosts)


@pytest.mark.parametrize("tuning", [dict(merge_group=2), None])
def test_edge16_full_size_sampled(tuning):
    import torch
    W = tg.workload("edge16_c3")
    prm = W["params"]
    tabs = tg.hash_tables(W["hash_seed"])
    T = tg.traffic_for(W)
    R = T.routers
    n_slots = 10
    slots = [T.slot(t) for t in range(n_slots)]
    # A: literal regain (the bench's lists); B: with the RHFG[0] check, so that sampled
    # estimators decide membership
    ctx_a = ssd.Context(ssd.make_params(prm), tabs)
    ctx_b = ssd.Context(ssd.make_params(prm, ssd.SSD_VERIFY_H0), tabs)
    if tuning:
        ctx_a.tuning = tuning
        ctx_b.tuning = tuning
    ra = [ctx_a.sketch() for _ in range(R)]
    ga = ctx_a.sketch()
    rb = [ctx_b.sketch() for _ in range(R)]
    gb = ctx_b.sketch()
    la = run_gpu(ctx_a, ra, ga, slots)
    lb = run_gpu(ctx_b, rb, gb, slots)
    torch.cuda.synchronize()
    assert set(lb[0].tolist()) <= set(la[0].tolist())
    assert len(lb[0]) > 5
    n_rec = ctx_a.sketch_bytes // 2
    for off in range(0, n_rec, 1 << 28):         # the flag changes no recorder
        c = min(1 << 28, n_rec - off)
        assert np.array_equal(ga.export(off, c), gb.export(off, c)), off
    ctx_a.close()
    p = oracle.params(prm, oracle.VERIFY_H0)
    hosts = sample_hosts(T, W, lb)
    samp, cols, extra = sampled_oracle(p, tabs, slots, hosts)
    members = check(p, tabs, samp, cols, extra, hosts, rb, gb, lb)
    assert members == len(lb[0])                   # every listed host was sampled and confirmed
    ctx_b.close()


def test_stress32_full_size_sampled():
    import torch
    W = tg.workload("stress32_c4")
    prm = W["params"]
    tabs = tg.hash_tables(W["hash_seed"])
    T = tg.traffic_for(W)
    R = T.routers
    n_slots = 6
    slots = [T.slot(t) for t in range(n_slots)]
    assert sum(len(x) for x in slots[0]) == 15_600_000
    ctx = ssd.Context(ssd.make_params(prm, ssd.SSD_VERIFY_H0), tabs)
    ctx.tuning = dict(merge_group=4, combine_touches=2)
    routers = [ctx.sketch() for _ in range(R)]
    glob = ctx.sketch()
    got = run_gpu(ctx, routers, glob, slots)
    torch.cuda.synchronize()
    p = oracle.params(prm, oracle.VERIFY_H0)
    hosts = sample_hosts(T, W, got)
    samp, cols, extra = sampled_oracle(p, tabs, slots, hosts)
    assert check(p, tabs, samp, cols, extra, hosts, routers, glob, got) == len(got[0]) == 0
    # the hot sources' estimators were written: the row-0 estimator of each holds recently
    # touched recorders at every router that carried its packets
    hot = T.hot_ips().tolist()
    assert hot
    for x in hot[:3]:
        c0 = int(cols[x][0])
        assert (glob.export_estimator(0, c0) < p.k).sum() > 0
    ctx.close()
