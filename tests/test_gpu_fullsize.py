"""Exact parity at the full size of the benchmark workload, on the routes bench.py times (the
default launch configuration, and the pre-hashed route the autotuner also picks for it).

Workload: one core-link router, 6.25 M packets per slot, eta = 2^11, q = 18, r = 5 (a 5 GiB RSEA),
k = 60, theta = 1024, run for k + 4 slots so the window rolls over.

Route A is bench.py's timed step: one ssd_slot call per slot with flags 0 (Algorithm 4's final
test without the RHFG[0] check, as the paper prints it), no global sketch, and the default launch
configuration, which ssd_autotune keeps on this workload. In that call the pairs are pre-hashed once,
one launch collects chunk 0's touch bits, and ten chunk launches run as programmatic dependents,
each applying its chunk's bits and collecting the next chunk's.

Route B is the same traffic through ssd_scan + ssd_close_slot with the RHFG[0] check and the merged
sketch written every slot.

The oracle holds the whole RSEA in host memory and runs Algorithm 2 and the distance recorder
update on every slot. The checks are exact, not sampled:
- both lists and their R_k, entry by entry, at slots inside and after the first window;
- a block of recorders of every router and of the merged sketch at every slot;
- every recorder of both routers and of the merged sketch after the last slot."""
import numpy as np
import pytest

import oracle
import paper_1803_11036_gb300 as ssd
import trafficgen as tg
from gpu_harness import to_dev

pytestmark = pytest.mark.gpu

BLOCK = 1 << 22   # recorders compared at every slot (8 MiB, at a slot-dependent offset)


def _assert_list(got, want, where):
    gi, gr = got
    assert len(gi) == len(want["ips"]), f"{where}: {len(gi)} hosts, oracle {len(want['ips'])}"
    assert np.array_equal(gi, want["ips"]), f"{where}: hosts differ"
    assert np.array_equal(gr, want["rk"]), f"{where}: R_k differs"


def test_corelink_full_size_bench_route_exact():
    import torch
    W = tg.workload("corelink_c2")
    prm = W["params"]
    k = prm["k"]
    slots = k + 4
    checkpoints = {9, k - 1, k, slots - 1}
    tabs = tg.hash_tables(W["hash_seed"])
    T = tg.traffic_for(W)
    assert T.routers == 1

    ctx_a = ssd.Context(ssd.make_params(prm), tabs)
    ctx_b = ssd.Context(ssd.make_params(prm, ssd.SSD_VERIFY_H0), tabs)
    ra, rb, gb = ctx_a.sketch(), ctx_b.sketch(), ctx_b.sketch()
    n_rec = ctx_a.sketch_bytes // 2
    p_lit = oracle.params(prm)
    p_chk = oracle.params(prm, oracle.VERIFY_H0)
    sk = oracle.new_sketch(p_lit)
    assert sk.size == n_rec
    rng = np.random.default_rng(7)
    listed = {"literal": 0, "checked": 0}
    for t in range(slots):
        pairs = T.slot(t)[0]
        # oracle: advance at the start of every slot after the first, then Algorithm 2
        if t:
            oracle.advance(p_lit, sk)
            # both routers after slot t-1's close hold the advanced recorders
            off = int(rng.integers(0, n_rec - BLOCK))
            assert np.array_equal(ra.export(off, BLOCK), sk[off:off + BLOCK]), (t, off)
            assert np.array_equal(rb.export(off, BLOCK), sk[off:off + BLOCK]), (t, off)
        oracle.scan(p_lit, tabs, sk, pairs)
        dev = to_dev(pairs)
        got_a = ctx_a.slot([ra], [dev])
        ctx_b.scan(rb, dev)
        got_b = ctx_b.close_slot([rb], gb)
        del dev
        # the merged sketch of slot t is the state before the close's advance
        off = int(rng.integers(0, n_rec - BLOCK))
        assert np.array_equal(gb.export(off, BLOCK), sk[off:off + BLOCK]), (t, off)
        if t in checkpoints:
            want_lit = oracle.regain(p_lit, tabs, sk, "pruned")
            want_chk = oracle.regain(p_chk, tabs, sk, "pruned")
            _assert_list(got_a, want_lit, f"slot {t}, ssd_slot, literal list")
            _assert_list(got_b, want_chk, f"slot {t}, ssd_close_slot, checked list")
            assert ctx_b.stats()["hot"] == [int(oracle.hse(p_chk, sk, i).size) for i in range(p_chk.r)]
            listed["literal"] += len(want_lit["ips"])
            listed["checked"] += len(want_chk["ips"])
    torch.cuda.synchronize()
    assert listed["checked"] > 10 and listed["literal"] >= listed["checked"]

    # every recorder: the merged sketch of the last slot, then both routers one advance further
    step = 1 << 28
    for off in range(0, n_rec, step):
        c = min(step, n_rec - off)
        assert np.array_equal(gb.export(off, c), sk[off:off + c]), ("global", off)
    oracle.advance(p_lit, sk)
    for off in range(0, n_rec, step):
        c = min(step, n_rec - off)
        assert np.array_equal(ra.export(off, c), sk[off:off + c]), ("ssd_slot router", off)
        assert np.array_equal(rb.export(off, c), sk[off:off + c]), ("ssd_close_slot router", off)
    assert ra.slot == rb.slot == slots
    ctx_a.close()
    ctx_b.close()


def test_corelink_full_size_prehashed_route_exact():
    """The same workload at full size on the other route the autotuner picks for it: pre-hashed
    pairs re-read by every chunk launch (collect_touches 1) with 64 MiB touch chunks, five chunk
    launches per slot, scan unroll 8. Six slots (the window not yet full, so every slot's list is
    that of slots 0..t): every recorder of the router after each slot's close in blocks, the list
    and its R_k at the last slot entry by entry, and every recorder at the end."""
    import torch
    W = tg.workload("corelink_c2")
    prm = W["params"]
    slots = 6
    tabs = tg.hash_tables(W["hash_seed"])
    T = tg.traffic_for(W)
    ctx = ssd.Context(ssd.make_params(prm), tabs)
    ctx.tuning = dict(touch_chunk_bytes=64 << 20, collect_touches=1, scan_unroll=8)
    router = ctx.sketch()
    n_rec = ctx.sketch_bytes // 2
    p_lit = oracle.params(prm)
    sk = oracle.new_sketch(p_lit)
    rng = np.random.default_rng(11)
    got = None
    for t in range(slots):
        pairs = T.slot(t)[0]
        if t:
            oracle.advance(p_lit, sk)
            off = int(rng.integers(0, n_rec - BLOCK))
            assert np.array_equal(router.export(off, BLOCK), sk[off:off + BLOCK]), (t, off)
        oracle.scan(p_lit, tabs, sk, pairs)
        dev = to_dev(pairs)
        got = ctx.slot([router], [dev])
        del dev
    torch.cuda.synchronize()
    want = oracle.regain(p_lit, tabs, sk, "pruned")
    _assert_list(got, want, f"slot {slots - 1}, pre-hashed route, literal list")
    assert len(want["ips"]) > 0
    oracle.advance(p_lit, sk)
    step = 1 << 28
    for off in range(0, n_rec, step):
        c = min(step, n_rec - off)
        assert np.array_equal(router.export(off, c), sk[off:off + c]), ("router", off)
    ctx.close()
