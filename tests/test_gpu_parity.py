"""GPU parity: the CUDA library through its C ABI against the CPU oracle on the
same seeded inputs, element by element. Everything here is integer work, so the
bar is bit-exact: every recorder of every sketch, every host and every R_k."""
import numpy as np
import pytest

import oracle
import paper_1803_11036_gb300 as ssd
import trafficgen as tg
from gpu_harness import Run, assert_list_equal, setup, to_dev

pytestmark = pytest.mark.gpu


# ------------------------------------------------------------------ scan

@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 31, 32, 33, 1000, (1 << 18) + 5])
def test_scan_ragged_sizes(n):
    """Algorithm 2 on pair counts that hit the vector body, the odd tail and the empty case."""
    W = tg.workload("paper_c1")
    p, tabs, ctx = setup(W)
    pairs = tg.traffic_for(W).fill(0, n=max(n, 1))[:n]
    sk = ctx.sketch()
    ctx.scan(sk, to_dev(pairs))
    want = oracle.new_sketch(p)
    oracle.scan(p, tabs, want, pairs)
    assert np.array_equal(sk.export(), want)
    ctx.close()


@pytest.mark.parametrize("offset", [1, 3])
def test_scan_unaligned_start(offset):
    """A pair buffer that starts 8 bytes past a 16-byte boundary (a head packet outside the body)."""
    W = tg.workload("paper_c1")
    p, tabs, ctx = setup(W)
    pairs = tg.traffic_for(W).fill(1, n=4099)
    dev = to_dev(pairs)
    sub = dev[2 * offset:]          # drops `offset` packets; odd offsets start at 8 mod 16
    assert (sub.data_ptr() % 16 == 8) == (offset % 2 == 1)
    sk = ctx.sketch()
    ctx.scan(sk, sub)
    want = oracle.new_sketch(p)
    oracle.scan(p, tabs, want, pairs[offset:])
    assert np.array_equal(sk.export(), want)
    ctx.close()


def test_scan_batch_equals_separate_scans():
    """One launch over uneven routers (empty, odd, unaligned) = one scan per router."""
    W = tg.workload("edge_small")
    p, tabs, ctx = setup(W)
    T = tg.traffic_for(W)
    base = T.slot(0)
    pieces = [base[0][:0], base[1][:1], base[2][:4097], base[3], base[0][:77]]
    devs = [to_dev(x) for x in pieces]
    devs[4] = to_dev(np.concatenate([base[0][:1], base[0][:77]]))[2:]  # starts at 8 mod 16
    a = [ctx.sketch() for _ in pieces]
    ctx.scan_batch(a, devs)
    for sk, pr in zip(a, pieces):
        want = oracle.new_sketch(p)
        oracle.scan(p, tabs, want, pr)
        assert np.array_equal(sk.export(), want)
    ctx.close()


def test_scan_small_and_large_eta_and_r3():
    """eta = 32 (a quarter-warp estimator), eta = 2^15 (the largest) and r = 3."""
    for prm in (dict(log2_eta=5, q=9, r=5, delta=8, k=3, theta=20),
                dict(log2_eta=15, q=9, r=5, delta=8, k=3, theta=20000),
                dict(log2_eta=5, q=17, r=3, delta=15, k=2, theta=20)):
        W = tg.workload("tiny")
        W["params"] = prm
        p, tabs, ctx = setup(W)
        pairs = tg.traffic_for(W).fill(0, n=3000)
        sk = ctx.sketch()
        ctx.scan(sk, to_dev(pairs))
        want = oracle.new_sketch(p)
        oracle.scan(p, tabs, want, pairs)
        assert np.array_equal(sk.export(), want), prm
        ctx.close()


# ---------------------------------------------------------- advance / merge

def test_advance_saturates_and_counts_slots():
    """Sec. 3.2: recorders below 65535 grow by one; 65534 -> 65535 -> 65535."""
    W = tg.workload("tiny")
    p, tabs, ctx = setup(W)
    rng = np.random.default_rng(1)
    n = ctx.sketch_bytes // 2
    state = rng.integers(0, 65536, n).astype(np.uint16)
    state[:64] = [65535, 65534, 65533, 0, 1, 2, 3, 4] * 8
    sk = ctx.sketch()
    sk.load(state, slot=7)
    ctx.advance([sk])
    want = state.copy()
    oracle.advance(p, want)
    assert np.array_equal(sk.export(), want) and sk.slot == 8
    ctx.advance([sk])
    oracle.advance(p, want)
    assert np.array_equal(sk.export(), want) and sk.export(0, 2).tolist() == [65535, 65535]
    ctx.close()


@pytest.mark.parametrize("nr", [1, 2, 5, 17])
def test_merge_is_elementwise_min(nr):
    W = tg.workload("tiny")
    p, tabs, ctx = setup(W)
    rng = np.random.default_rng(nr)
    n = ctx.sketch_bytes // 2
    states = [rng.integers(0, 65536, n).astype(np.uint16) for _ in range(nr)]
    rs = [ctx.sketch() for _ in range(nr)]
    for sk, st in zip(rs, states):
        sk.load(st, slot=3)
    g = ctx.sketch()
    ctx.merge(rs, g)
    assert np.array_equal(g.export(), oracle.merge(p, states)) and g.slot == 3
    ctx.close()


def test_merge_rejects_slot_mismatch():
    W = tg.workload("tiny")
    _, _, ctx = setup(W)
    a, b, g = ctx.sketch(), ctx.sketch(), ctx.sketch()
    ctx.advance([a])
    with pytest.raises(ssd.SSDError) as e:
        ctx.merge([a, b], g)
    assert e.value.code == -6
    with pytest.raises(ssd.SSDError):
        ctx.merge([a, g], g)
    ctx.close()


# ------------------------------------------------------------------ regain

def _dense_tiny():
    W = tg.workload("tiny")
    W["traffic"].update(n_planted=12, count_a=400)
    return W


@pytest.mark.parametrize("flags", [0, ssd.SSD_VERIFY_H0, ssd.SSD_NO_PRUNE, ssd.SSD_NO_PRUNE | ssd.SSD_VERIFY_H0])
@pytest.mark.parametrize("wl", ["tiny", "dense_tiny"])
def test_slots_unfused_tiny(wl, flags):
    """Every slot: the merged sketch bit-exact, the list and R_k equal the oracle's, and the
    candidate count of every row equals the oracle's literal (no prune) or pruned level count."""
    W = _dense_tiny() if wl == "dense_tiny" else tg.workload(wl)
    run = Run(W, flags)
    method = "levelwise" if flags & ssd.SSD_NO_PRUNE else "pruned"
    for _ in range(W["slots"]):
        got, want = run.step_unfused(method)
        assert np.array_equal(run.glob.export(), run.pipe.global_sk)
        assert_list_equal(got, want, f"slot {run.t}")
        st = run.ctx.stats()
        hot = [len(oracle.hse(run.p, run.pipe.global_sk, i)) for i in range(run.p.r)]
        assert st["hot"] == hot
        assert st["level"] == [int(x) for x in want["levels"]]
        assert st["raw"] == want["raw"]
    run.close()


@pytest.mark.parametrize("wl,slots", [("paper_c1", 12), ("corelink_small", 14)])
def test_slots_unfused_single_router(wl, slots):
    run = Run(wl)
    for _ in range(slots):
        got, want = run.step_unfused("pruned", batch=False)
        assert np.array_equal(run.glob.export(), run.pipe.global_sk)
        for r_gpu, r_or in zip(run.routers, run.pipe.routers):
            assert np.array_equal(r_gpu.export(), r_or)
        assert_list_equal(got, want, f"{wl} slot {run.t}")
    run.close()


@pytest.mark.parametrize("wl,slots", [("edge_small", 10), ("stress_small", 10)])
def test_slots_unfused_many_routers(wl, slots):
    run = Run(wl)
    for _ in range(slots):
        got, want = run.step_unfused("pruned")
        assert np.array_equal(run.glob.export(), run.pipe.global_sk)
        assert_list_equal(got, want, f"{wl} slot {run.t}")
        st = run.ctx.stats()
        assert st["level"] == [int(x) for x in want["levels"]]
    for r_gpu, r_or in zip(run.routers, run.pipe.routers):
        assert np.array_equal(r_gpu.export(), r_or)
    run.close()


@pytest.mark.parametrize("wl,with_global", [("tiny", True), ("paper_c1", False), ("edge_small", True),
                                            ("stress_small", False)])
def test_slots_fused_close(wl, with_global):
    """close_slot (one pass: merge + hot extraction + advance, then the candidate levels) gives
    the oracle's list every slot; the merged sketch it writes is the oracle's merged sketch; the
    routers it leaves are the oracle's routers advanced by one slot."""
    run = Run(wl)
    slots = run.W["slots"]
    for _ in range(slots):
        got, want = run.step_fused("pruned", with_global=with_global)
        assert_list_equal(got, want, f"{wl} slot {run.t}")
        if with_global:
            assert np.array_equal(run.glob.export(), run.pipe.global_sk)
        assert all(r.slot == run.t + 1 for r in run.routers)
    for r_gpu, r_or in zip(run.routers, run.pipe.routers):
        nxt = r_or.copy()
        oracle.advance(run.p, nxt)
        assert np.array_equal(r_gpu.export(), nxt)
    run.close()


CH = ssd.SSD_SLOT_CHUNKED


@pytest.mark.parametrize("wl,chunk,flags,with_global", [
    ("tiny", 0, 0, True),                   # one chunk, eta = 64 (small-estimator kernel)
    ("tiny", 4096, 0, True),                # five chunks of one row
    ("tiny", 1024, 0, False),               # too many chunks: scan_batch + close_slot
    ("paper_c1", 0, 0, False),              # one router: one chunk, no next-chunk collection
    ("paper_c1", 2 << 20, 0, True),         # one router: ten chunks, each collecting the next
    ("paper_c1", 10 << 20, 0, False),       # one router: three chunks, the last one partial
    ("corelink_small", 4 << 20, 0, False),
    ("paper_c1", 0, CH, False),             # chunked: one chunk holding all rows
    ("paper_c1", 2 << 20, CH, True),        # ten chunks, two per row
    ("paper_c1", 10 << 20, CH, False),      # three chunks of two rows, the last one partial
    ("edge_small", 0, 0, True),             # four routers
    ("stress_small", 16 << 20, 0, False),   # eight routers, hot sources, ten chunks
    ("stress_small", 64 << 10, 0, False),   # eight routers, fallback
])
def test_fused_slot(wl, chunk, flags, with_global):
    """ssd_slot (the scan's touches applied by the streaming pass, from L2 bits or from binned
    records) gives the oracle's list and merged sketch every slot, and leaves the routers the
    oracle holds advanced by one."""
    run = Run(wl, flags, touch_chunk_bytes=chunk)
    for _ in range(run.W["slots"]):
        got, want = run.step_slot("pruned", with_global=with_global)
        assert_list_equal(got, want, f"{wl} slot {run.t}")
        if with_global:
            assert np.array_equal(run.glob.export(), run.pipe.global_sk)
    for r_gpu, r_or in zip(run.routers, run.pipe.routers):
        nxt = r_or.copy()
        oracle.advance(run.p, nxt)
        assert np.array_equal(r_gpu.export(), nxt)
    run.close()


@pytest.mark.parametrize("flags", [0, CH])
@pytest.mark.parametrize("n", [0, 1, 3, 4097, (1 << 18) + 5])
@pytest.mark.parametrize("offset", [0, 1])
def test_slot_ragged(n, offset, flags):
    """The one-router routes (chunks collecting the next chunk's bits; bits collected on the side
    stream) on empty, odd and unaligned pair buffers: the router they leave is the oracle's after
    scan + advance, and the list is the oracle's."""
    W = tg.workload("paper_c1")
    p, tabs, ctx = setup(W, flags, touch_chunk_bytes=2 << 20)
    pairs = tg.traffic_for(W).fill(0, n=n + 2)
    dev = to_dev(pairs)[2 * offset: 2 * (offset + n)]
    sk = ctx.sketch()
    got = ctx.slot([sk], [dev])
    want_sk = oracle.new_sketch(p)
    oracle.scan(p, tabs, want_sk, pairs[offset:offset + n])
    want = oracle.regain(p, tabs, want_sk, "pruned")
    assert np.array_equal(got[0], want["ips"]) and np.array_equal(got[1], want["rk"])
    oracle.advance(p, want_sk)
    assert np.array_equal(sk.export(), want_sk)
    ctx.close()


@pytest.mark.parametrize("wl,pinned", [("edge_small", False), ("paper_c1", True)])
def test_slot_from_host_memory(wl, pinned):
    """ssd_slot_host (pairs copied from host memory into double-buffered staging that grows with
    the slot size) gives the oracle's list every slot and leaves the oracle's routers."""
    import torch
    run = Run(wl)
    for _ in range(run.W["slots"]):
        run.t += 1
        pairs = run.slot_pairs(run.t)
        want = run.pipe.step(pairs, "pruned")
        if pinned:
            host = [torch.from_numpy(np.ascontiguousarray(x).reshape(-1).view(np.int32)).pin_memory() for x in pairs]
        else:
            host = pairs
        got = run.ctx.slot_host(run.routers, host)
        assert_list_equal(got, want, f"{wl} slot {run.t}")
    for r_gpu, r_or in zip(run.routers, run.pipe.routers):
        nxt = r_or.copy()
        oracle.advance(run.p, nxt)
        assert np.array_equal(r_gpu.export(), nxt)
    run.close()


def test_list_capacity_reports_required_size():
    run = Run("paper_c1")
    for _ in range(4):
        run.step_unfused(None)
    full_ips, _ = run.ctx.regain(run.glob)
    assert len(full_ips) > 3
    with pytest.raises(ssd.SSDError) as e:
        run.ctx.regain(run.glob, cap=3)
    assert e.value.code == ssd.SSD_ECAPACITY
    assert run.ctx.stats()["n_out"] == len(full_ips)
    run.close()


def test_candidate_buffer_overflow_is_an_error():
    W = _dense_tiny()
    run = Run(W, ssd.SSD_NO_PRUNE, ctb_capacity=16)
    for _ in range(4):
        run.step_unfused(None)
    with pytest.raises(ssd.SSDError) as e:
        run.ctx.regain(run.glob)
    assert e.value.code == ssd.SSD_ECAPACITY
    assert run.ctx.stats()["status"] & ssd.SSD_STATUS_CTB_OVERFLOW
    run.close()


def test_checkpoint_resume_is_bit_identical():
    """Export every router and the slot counter mid-run, import into a fresh context, continue:
    identical to the uninterrupted run."""
    W = tg.workload("edge_small")
    a = Run(W)
    for _ in range(4):
        a.step_fused(None, with_global=False)
    saved = [(r.export(), r.slot) for r in a.routers]
    b = Run(W)
    for sk, (rec, slot) in zip(b.routers, saved):
        sk.load(rec, slot)
    b.t = a.t
    for _ in range(3):
        pairs = a.T.slot(a.t + 1)
        a.t += 1
        devs = [to_dev(x) for x in pairs]
        a.ctx.scan_batch(a.routers, devs)
        b.ctx.scan_batch(b.routers, devs)
        la = a.ctx.close_slot(a.routers)
        lb = b.ctx.close_slot(b.routers)
        assert np.array_equal(la[0], lb[0]) and np.array_equal(la[1], lb[1])
    for x, y in zip(a.routers, b.routers):
        assert np.array_equal(x.export(), y.export()) and x.slot == y.slot
    a.close()
    b.close()


@pytest.mark.parametrize("step", ["slot", "fused", "unfused"])
def test_discrete_window_k1(step):
    """k = 1, the discrete-window case of the sliding estimator: a recorder counts only in the slot
    that touched it, so each slot's list depends on that slot's pairs alone. The planted hosts send
    all their peers in every slot (pacing D/k with k = 1)."""
    W = tg.workload("paper_c1")
    W["params"]["k"] = 1
    W["traffic"]["k"] = 1
    run = Run(W)
    nonempty = 0
    for _ in range(5):
        if step == "slot":
            got, want = run.step_slot("pruned", with_global=True)
        elif step == "fused":
            got, want = run.step_fused("pruned")
        else:
            got, want = run.step_unfused("pruned")
        assert_list_equal(got, want, f"slot {run.t}")
        assert np.array_equal(run.glob.export(), run.pipe.global_sk), run.t
        nonempty += len(want["ips"]) > 0
    assert nonempty == 5
    run.close()


@pytest.mark.parametrize("wl", ["tiny", "paper_c1"])
@pytest.mark.parametrize("step", ["slot", "fused", "unfused"])
def test_rhfg_literal_variant(wl, step):
    """Eq. 2 as printed (SSD_RHFG_LITERAL: windows at i*delta, bits 0..delta-1 completed by the
    RHFG[0] check) on every path: the merged sketch, the list and R_k equal the oracle's under the
    same reading; on the separate calls so do the candidate counts and the staged completions."""
    run = Run(wl, ssd.SSD_RHFG_LITERAL)
    nonempty = 0
    for _ in range(min(run.W["slots"], 6)):
        if step == "slot":
            got, want = run.step_slot("pruned", with_global=True)
        elif step == "fused":
            got, want = run.step_fused("pruned")
        else:
            got, want = run.step_unfused("pruned")
            st = run.ctx.stats()
            assert st["level"] == [int(x) for x in want["levels"]]
            assert st["raw"] == want["raw"]
        assert_list_equal(got, want, f"{wl} slot {run.t}")
        assert np.array_equal(run.glob.export(), run.pipe.global_sk), run.t
        nonempty += len(want["ips"]) > 0
    assert nonempty > 0
    run.close()


@pytest.mark.parametrize("wl", ["tiny", "paper_c1"])
def test_occupancy_equals_oracle_rk_sums(wl):
    """ssd_sketch_occupancy: per row, the sum of R_k over the row's estimators, for the merged
    sketch and every router, equal to the oracle's rows of R_k summed."""
    run = Run(wl)
    for _ in range(3):
        run.step_unfused("pruned")
    rows = range(run.p.r)
    assert run.glob.occupancy() == [int(oracle.rk_row(run.p, run.pipe.global_sk, i).sum()) for i in rows]
    for r_gpu, r_or in zip(run.routers, run.pipe.routers):
        assert r_gpu.occupancy() == [int(oracle.rk_row(run.p, r_or, i).sum()) for i in rows]
    run.close()
