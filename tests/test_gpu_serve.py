"""Served form: every router's lists are the same when it is served alone and when it is served in
a mix of routers whose slices overlap on the device; they equal the oracle's; routers that cannot
be admitted wait for memory and are served once it frees up."""
import numpy as np
import pytest

import oracle
import paper_1803_11036_gb300 as ssd
import trafficgen as tg
from paper_1803_11036_gb300 import serve

pytestmark = pytest.mark.gpu


def make_slices(W, routers, per_router, mean_gap_s, seed=0):
    import torch
    rng = np.random.default_rng(seed)
    out = []
    for r in routers:
        tr = dict(W["traffic"])
        tr["seed"] = tr["seed"] + 101 * r
        T = tg.Traffic(**tr)
        t = 0.0
        for j in range(per_router):
            t += rng.exponential(mean_gap_s)
            pairs = T.fill(j)
            host = torch.from_numpy(np.ascontiguousarray(pairs).reshape(-1).view(np.int32)).pin_memory()
            out.append(serve.Slice(router=r, pairs=host, arrival=t, seq=j))
    return out


def by_slot(results):
    return {(x.router, x.slot): (x.ips, x.rk) for x in results}


def run_server(W, slices, **kw):
    srv = serve.Server(ssd.make_params(W["params"]), tg.hash_tables(W["hash_seed"]), **kw)
    res = srv.run(slices)
    order = list(srv.admitted_order)
    srv.close()
    return res, order


def test_alone_equals_mix_and_oracle():
    W = tg.workload("served_small")
    slices = make_slices(W, range(6), 6, mean_gap_s=0.002)
    # the mix reserves every router's buffers for the largest slice and runs another launch
    # configuration; neither may change a list
    mix, _ = run_server(W, slices, max_inflight=4, max_slice_pairs=W["traffic"]["count_b"],
                        tuning=dict(scan_unroll=2, combine_touches=1, touch_chunk_bytes=4 << 20))
    assert len(mix) == len(slices)
    mixd = by_slot(mix)
    for r in (0, 3, 5):
        alone, _ = run_server(W, [s for s in slices if s.router == r], max_inflight=4)
        for x in alone:
            got = mixd[(r, x.slot)]
            assert np.array_equal(got[0], x.ips) and np.array_equal(got[1], x.rk), (r, x.slot)
    # router 0 against the oracle, slot by slot
    p = oracle.params(W["params"])
    pipe = oracle.Pipeline(p, tg.hash_tables(W["hash_seed"]), 1)
    mine = sorted([s for s in slices if s.router == 0], key=lambda s: s.seq)
    nonempty = 0
    for s in mine:
        want = pipe.step([s.pairs.numpy().view(np.uint32).reshape(-1, 2)], "pruned")
        got = mixd[(0, s.seq)]
        assert np.array_equal(got[0], want["ips"]) and np.array_equal(got[1], want["rk"]), s.seq
        nonempty += len(want["ips"]) > 0
    assert nonempty > 0
    summ = serve.latency_summary(mix)
    assert summ["p99_ms"] >= summ["p50_ms"] > 0


def test_admission_waits_for_memory():
    """With room for two routers, four routers are served two at a time (a router's memory is
    freed when its last slice is done) and every list is still the one it gets alone."""
    W = tg.workload("served_small")
    slices = make_slices(W, range(4), 3, mean_gap_s=0.001, seed=1)
    capped, order = run_server(W, slices, max_inflight=4, max_routers=2, evict_when_done=True)
    assert len(capped) == len(slices) and sorted(order) == [0, 1, 2, 3]
    free, _ = run_server(W, slices, max_inflight=8)
    a, b = by_slot(capped), by_slot(free)
    assert a.keys() == b.keys()
    for key in a:
        assert np.array_equal(a[key][0], b[key][0]) and np.array_equal(a[key][1], b[key][1]), key


def test_served_full_size_sampled():
    """Three routers of the served workload at full size (q = 17, slices of 10k-2M packets) through
    the Server in the bench's configuration (16 in flight, buffers reserved for 2M-packet slices).
    With the RHFG[0] check on, each router's list of every slot is decided by a sample of its
    estimators, which the oracle follows through every packet; the router's sketch after its last
    slice is checked on the same sample."""
    W = tg.workload("served_c5")
    tabs = tg.hash_tables(W["hash_seed"])
    routers = range(3)
    slices = make_slices(W, routers, 5, mean_gap_s=0.001, seed=3)
    params = ssd.make_params(W["params"], ssd.SSD_VERIFY_H0)
    srv = serve.Server(params, tabs, max_inflight=16, max_slice_pairs=W["traffic"]["count_b"])
    res = srv.run(slices)
    got = by_slot(res)
    p = oracle.params(W["params"], oracle.VERIFY_H0)
    thr, _ = oracle.threshold(p.eta, p.theta)
    rng = np.random.default_rng(9)
    members = 0
    for r in routers:
        tr = dict(W["traffic"])
        tr["seed"] = tr["seed"] + 101 * r
        T = tg.Traffic(**tr)
        mine = sorted([s for s in slices if s.router == r], key=lambda s: s.seq)
        hosts = set(T.planted_ips().tolist())
        hosts |= {T.lib.tg_src_ip(T._h, int(x)) for x in rng.integers(0, tr["n_src"], 100)}
        for s in mine:
            hosts |= set(got[(r, s.seq)][0].tolist())
        hosts = sorted(hosts)
        cols = {x: oracle.rhfg(p, tabs, x) for x in hosts}
        rows = np.concatenate([np.arange(p.r, dtype=np.uint32) for _ in hosts])
        cc = np.concatenate([cols[x].astype(np.uint32) for x in hosts])
        samp = oracle.Sampled(p, rows, cc)
        for s in mine:
            if s.seq:
                samp.advance()
            samp.scan(tabs, s.pairs.numpy().view(np.uint32).reshape(-1, 2))
            listed = dict(zip(got[(r, s.seq)][0].tolist(), got[(r, s.seq)][1].tolist()))
            for x in hosts:
                below = [samp.get(i, int(cols[x][i])) < p.k for i in range(p.r)]
                union = int(np.logical_and.reduce(below).sum())
                member = all(int(b.sum()) >= thr for b in below) and union >= thr
                assert (x in listed) == member, (r, s.seq, hex(x))
                if member:
                    assert listed[x] == union
                    members += 1
        samp.advance()
        sk = srv.tenants[r].sketch
        for i in range(p.r):
            c = int(cols[hosts[0]][i])
            assert np.array_equal(sk.export_estimator(i, c), samp.get(i, c)), (r, i)
        samp.close()
    assert members > 0
    srv.close()
