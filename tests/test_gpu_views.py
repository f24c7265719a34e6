"""Sketch views (Sec. 3.1: the ONet side by exchanging the roles of the two networks; Sec. 6:
several RSEAs, each regaining one group of hosts split by their IP addresses). Every view gives
the oracle's sketch and list on the pairs that view takes (oracle.view_pairs; a group's list holds
only its hosts, oracle.in_group), on every route: one ssd_scan_batch launch scanning the same
pairs for both sides or for every group, ssd_close_slot, and the routes of ssd_slot. Combining
sketches of different views is refused."""
import numpy as np
import pytest

import oracle
import paper_1803_11036_gb300 as ssd
import trafficgen as tg
from gpu_harness import to_dev

pytestmark = pytest.mark.gpu
CN, ON = ssd.SSD_SIDE_CNET, ssd.SSD_SIDE_ONET


def swapped_stream(W, t):
    """Slot t of the workload with the fields exchanged: its ONet side holds the planted hosts."""
    return np.ascontiguousarray(tg.traffic_for(W).slot(t)[0][:, ::-1])


def expect(p, tabs, pipe, pairs, gb=0, g=0):
    want = pipe.step([pairs], "pruned")
    keep = oracle.in_group(want["ips"], gb, g)
    return want["ips"][keep], want["rk"][keep]


def test_both_sides_in_one_scan():
    """ssd_scan_batch over a CNet and an ONet sketch of the same pair buffer (one launch), then one
    close per side: each side equals the oracle on its view of the pairs, slot after slot."""
    W = tg.workload("paper_c1")
    p = oracle.params(W["params"])
    tabs = tg.hash_tables(W["hash_seed"])
    ctx = ssd.Context(ssd.make_params(W["params"]), tabs)
    cn, on = ctx.sketch().set_view(CN), ctx.sketch().set_view(ON)
    gcn, gon = ctx.sketch(), ctx.sketch()
    pipes = {CN: oracle.Pipeline(p, tabs, 1), ON: oracle.Pipeline(p, tabs, 1)}
    found = 0
    for t in range(6):
        pairs = swapped_stream(W, t)
        dev = to_dev(pairs)
        l0 = ctx.launch_count
        ctx.scan_batch([cn, on], [dev, dev])
        assert ctx.launch_count - l0 == 1
        for side, sk, gl in ((CN, cn, gcn), (ON, on, gon)):
            got = ctx.close_slot([sk], gl)
            want = expect(p, tabs, pipes[side], oracle.view_pairs(pairs, side))
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), (side, t)
            assert np.array_equal(gl.export(), pipes[side].global_sk), (side, t)
            assert gl.view == (side, 0, 0)
            found += len(got[0]) if side == ON else 0
    assert found > 0
    ctx.close()


@pytest.mark.parametrize("chunk,flags", [(0, 0), (2 << 20, 0), (2 << 20, ssd.SSD_SLOT_CHUNKED), (64 << 10, 0)])
def test_onet_side_through_ssd_slot(chunk, flags):
    """The ONet side through each route of ssd_slot (one router: pre-hashed pairs with the next
    chunk's touches collected in the chunk kernel; side stream; scan + close fallback)."""
    W = tg.workload("paper_c1")
    p = oracle.params(W["params"])
    tabs = tg.hash_tables(W["hash_seed"])
    ctx = ssd.Context(ssd.make_params(W["params"], flags, touch_chunk_bytes=chunk), tabs)
    sk, gl = ctx.sketch().set_view(ON), ctx.sketch()
    pipe = oracle.Pipeline(p, tabs, 1)
    found = 0
    for t in range(5):
        pairs = swapped_stream(W, t)
        got = ctx.slot([sk], [to_dev(pairs)], gl)
        want = expect(p, tabs, pipe, oracle.view_pairs(pairs, ON))
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), t
        assert np.array_equal(gl.export(), pipe.global_sk), t
        found += len(got[0])
    assert found > 0
    nxt = pipe.routers[0].copy()
    oracle.advance(p, nxt)
    assert np.array_equal(sk.export(), nxt)
    ctx.close()


@pytest.mark.parametrize("how", ["batch", "slot", "slot_small_chunks"])
def test_ip_groups(how):
    """Four groups (the top two bits of the host): one sketch per group over the same pairs; each
    sketch and list equal the oracle's on that group's pairs, and every listed host is in its group."""
    W = tg.workload("paper_c1")
    p = oracle.params(W["params"])
    tabs = tg.hash_tables(W["hash_seed"])
    gb = 2
    chunk = 2 << 20 if how == "slot_small_chunks" else 0
    ctx = ssd.Context(ssd.make_params(W["params"], touch_chunk_bytes=chunk), tabs)
    sks = [ctx.sketch().set_view(CN, gb, g) for g in range(1 << gb)]
    gls = [ctx.sketch() for _ in sks]
    pipes = [oracle.Pipeline(p, tabs, 1) for _ in sks]
    T = tg.traffic_for(W)
    found = 0
    for t in range(5):
        pairs = T.slot(t)[0]
        dev = to_dev(pairs)
        if how == "batch":
            ctx.scan_batch(sks, [dev] * len(sks))
        for g, (sk, gl) in enumerate(zip(sks, gls)):
            got = ctx.close_slot([sk], gl) if how == "batch" else ctx.slot([sk], [dev], gl)
            want = expect(p, tabs, pipes[g], oracle.view_pairs(pairs, CN, gb, g), gb, g)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), (g, t)
            assert np.array_equal(gl.export(), pipes[g].global_sk), (g, t)
            assert oracle.in_group(got[0], gb, g).all()
            found += len(got[0])
    assert found > 0
    ctx.close()


def test_view_rules():
    W = tg.workload("tiny")
    ctx = ssd.Context(ssd.make_params(W["params"]), tg.hash_tables(W["hash_seed"]))
    a, b, gl = ctx.sketch(), ctx.sketch(), ctx.sketch()
    assert a.view == (CN, 0, 0)
    for bad in ((2, 0, 0), (CN, 17, 0), (CN, 2, 4)):
        with pytest.raises(ssd.SSDError) as e:
            a.set_view(*bad)
        assert e.value.code == ssd._abi.SSD_EINVAL
    a.set_view(CN, 3, 5)
    assert a.view == (CN, 3, 5)
    b.set_view(ON)
    dev = to_dev(tg.traffic_for(W).slot(0)[0])
    for call in (lambda: ctx.merge([a, b], gl), lambda: ctx.close_slot([a, b], gl),
                 lambda: ctx.slot([a, b], [dev, dev], gl)):
        with pytest.raises(ssd.SSDError) as e:
            call()
        assert e.value.code == ssd._abi.SSD_EINVAL
    ctx.close_slot([b], gl)
    assert gl.view == (ON, 0, 0)
    with pytest.raises(ssd.SSDError) as e:
        b.set_view(CN)             # b has advanced a slot
    assert e.value.code == ssd._abi.SSD_ESTATE
    ctx.close()
