"""A slot captured once as a CUDA graph (SlotGraph over ssd_slot) and replayed on new pairs gives
exactly what direct ssd_slot calls give: the same list every slot, the same routers, the same
merged sketch and the same slot counters."""
import numpy as np
import pytest

import paper_1803_11036_gb300 as ssd
import trafficgen as tg
from gpu_harness import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("wl,flags,with_global", [
    ("paper_c1", 0, False),                     # one router: pre-hash, touch, chunk kernels
    ("paper_c1", ssd.SSD_SLOT_CHUNKED, True),   # side stream forked and joined inside the capture
    ("stress_small", 0, True),                  # eight routers, fixed per-router counts
])
def test_captured_slot_equals_direct_calls(wl, flags, with_global):
    W = tg.workload(wl)
    tabs = tg.hash_tables(W["hash_seed"])
    T = tg.traffic_for(W)
    R = T.routers
    counts = [T.count(0, r) for r in range(R)]
    assert all(T.count(t, r) == counts[r] for t in range(4) for r in range(R))
    ctx_a = ssd.Context(ssd.make_params(W["params"], flags, touch_chunk_bytes=4 << 20), tabs)
    ctx_b = ssd.Context(ssd.make_params(W["params"], flags, touch_chunk_bytes=4 << 20), tabs)
    ra = [ctx_a.sketch() for _ in range(R)]
    rb = [ctx_b.sketch() for _ in range(R)]
    ga = ctx_a.sketch() if with_global else None
    gb = ctx_b.sketch() if with_global else None
    graph = ssd.SlotGraph(ctx_b, rb, counts, gb)
    nonempty = 0
    for t in range(W["slots"]):
        pairs = [to_dev(x) for x in T.slot(t)]
        want = ctx_a.slot(ra, pairs, ga)
        for dst, src in zip(graph.inputs, pairs):
            dst.copy_(src)
        graph.replay()
        got = graph.result()
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), t
        nonempty += len(want[0]) > 0
        if with_global:
            assert np.array_equal(ga.export(), gb.export()) and ga.slot == gb.slot
    assert nonempty > 0
    for x, y in zip(ra, rb):
        assert np.array_equal(x.export(), y.export()) and x.slot == y.slot == W["slots"]
    ctx_a.close()
    ctx_b.close()


def test_replay_refused_after_buffers_replaced():
    """A graph holds the context's touch buffers: once ssd_tuning_set replaces them (a new touch
    chunk size), ssd_buffer_epoch has moved and SlotGraph.replay refuses instead of running on
    freed memory."""
    W = tg.workload("paper_c1")
    tabs = tg.hash_tables(W["hash_seed"])
    T = tg.traffic_for(W)
    ctx = ssd.Context(ssd.make_params(W["params"]), tabs)
    routers = [ctx.sketch()]
    graph = ssd.SlotGraph(ctx, routers, [T.count(0, 0)])
    graph.inputs[0].copy_(to_dev(T.slot(0)[0]))
    graph.replay()
    graph.result()
    e0 = int(ctx.L.ssd_buffer_epoch(ctx._h))
    ctx.tuning = dict(touch_chunk_bytes=16 << 20)
    assert int(ctx.L.ssd_buffer_epoch(ctx._h)) == e0 + 1
    with pytest.raises(RuntimeError):
        graph.replay()
    ctx.close()
