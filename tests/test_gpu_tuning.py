"""The launch configuration (ssd_tuning) spreads the same work differently and changes no
result: slots run under non-default configurations give the oracle's lists, merged sketch and
routers every slot, on every route of ssd_slot (one router with the next chunk's touches
collected in the chunk kernel, several routers with touches on the side stream, and the
scan + close fallback) and on the separate calls. ssd_autotune returns the sketches to their
initial state, keeps a configuration it measured, and refuses sketches that already ran a slot."""
import numpy as np
import pytest

import oracle
import paper_1803_11036_gb300 as ssd
import trafficgen as tg
from gpu_harness import Run, assert_list_equal, to_dev

pytestmark = pytest.mark.gpu

TUNINGS = [
    dict(touch_chunk_bytes=2 << 20, stream_blocks_per_sm=1, scan_blocks_per_sm=2, scan_unroll=1, merge_group=2,
         combine_touches=1, collect_touches=0, pair_level=1),
    dict(touch_chunk_bytes=4 << 20, stream_blocks_per_sm=2, scan_blocks_per_sm=32, scan_unroll=8, merge_group=4,
         combine_touches=1, collect_touches=1, pair_level=0),
    dict(touch_chunk_bytes=16 << 20, stream_blocks_per_sm=0, scan_blocks_per_sm=1, scan_unroll=2, merge_group=8,
         combine_touches=0, collect_touches=1, pair_level=1),
    dict(touch_chunk_bytes=8 << 20, stream_blocks_per_sm=3, scan_blocks_per_sm=4, scan_unroll=4, merge_group=8,
         combine_touches=2, collect_touches=0, pair_level=0),
    dict(touch_chunk_bytes=2 << 20, stream_blocks_per_sm=0, scan_blocks_per_sm=8, scan_unroll=4, merge_group=8,
         combine_touches=2, collect_touches=1, pair_level=0),
]


def hot_one_router():
    """The stress recipe (ten sources each sending 5 % of the packets over 256 peers) on one
    router, so the one-router chunk route sees many same-word touches in a warp."""
    W = tg.workload("stress_small")
    W["traffic"]["routers"] = 1
    W["traffic"]["count"] = "fixed"
    W["traffic"]["count_a"] = 300_000
    return W


def check_run(run, steps, step):
    for _ in range(steps):
        got, want = step()
        assert_list_equal(got, want, f"slot {run.t}")
        assert np.array_equal(run.glob.export(), run.pipe.global_sk), run.t


@pytest.mark.parametrize("ti", range(len(TUNINGS)))
@pytest.mark.parametrize("wl", ["paper_c1", "hot1", "edge_small", "stress_small"])
def test_tuned_slots_match_oracle(wl, ti):
    run = Run(hot_one_router() if wl == "hot1" else wl)
    run.ctx.tuning = TUNINGS[ti]
    assert run.ctx.tuning == TUNINGS[ti]
    check_run(run, run.W["slots"], lambda: run.step_slot("pruned", with_global=True))
    for r_gpu, r_or in zip(run.routers, run.pipe.routers):
        nxt = r_or.copy()
        oracle.advance(run.p, nxt)
        assert np.array_equal(r_gpu.export(), nxt)
    run.close()


@pytest.mark.parametrize("ti", range(len(TUNINGS)))
def test_tuned_separate_calls_match_oracle(ti):
    """scan_batch + close_slot and scan_batch + merge + regain + advance under each configuration."""
    for mode in ("fused", "unfused"):    # separate runs: the two paths advance at different points
        run = Run("stress_small")
        run.ctx.tuning = TUNINGS[ti]
        check_run(run, 4, (lambda: run.step_fused("pruned")) if mode == "fused" else
                  (lambda: run.step_unfused("pruned")))
        run.close()


def test_tuning_rejects_bad_values():
    W = tg.workload("tiny")
    ctx = ssd.Context(ssd.make_params(W["params"]), tg.hash_tables(W["hash_seed"]))
    before = ctx.tuning
    assert before == dict(touch_chunk_bytes=32 << 20, stream_blocks_per_sm=0, scan_blocks_per_sm=8, scan_unroll=4,
                          merge_group=8, combine_touches=0, collect_touches=0, pair_level=0)
    for bad in (dict(scan_unroll=3), dict(merge_group=1), dict(scan_blocks_per_sm=0), dict(scan_blocks_per_sm=33),
                dict(stream_blocks_per_sm=9), dict(combine_touches=3), dict(collect_touches=2), dict(pair_level=2),
                dict(touch_chunk_bytes=1 << 10),
                dict(touch_chunk_bytes=2 << 30)):
        with pytest.raises(ssd.SSDError) as e:
            ctx.tuning = bad
        assert e.value.code == ssd._abi.SSD_EINVAL
        assert ctx.tuning == before
    with pytest.raises(ValueError):
        ctx.tuning = dict(blocks=2)
    ctx.close()


@pytest.mark.parametrize("wl", ["paper_c1", "stress_small"])
def test_autotune_resets_and_keeps_results(wl):
    """After ssd_autotune the sketches hold 65535 everywhere at slot 0; slots then run under the
    chosen configuration give the oracle's results from the start."""
    run = Run(wl)
    pairs0 = [to_dev(p) for p in run.T.slot(0)]
    chosen = run.ctx.autotune(run.routers, pairs0, run.glob, reps=1)
    assert chosen == run.ctx.tuning
    assert set(chosen) == set(ssd._abi.TUNING_FIELDS)
    for sk in run.routers + [run.glob]:
        assert sk.slot == 0
        assert (sk.export() == 0xFFFF).all()
    check_run(run, 5, lambda: run.step_slot("pruned", with_global=True))
    # sketches that ran a slot are refused, and nothing changes
    with pytest.raises(ssd.SSDError) as e:
        run.ctx.autotune(run.routers, pairs0, run.glob, reps=1)
    assert e.value.code == ssd._abi.SSD_ESTATE
    assert run.routers[0].slot == 5
    run.close()


def test_tuning_cache_round_trip(tmp_path):
    """tuning.tuned: the first call tunes and stores, the second takes the stored configuration."""
    from paper_1803_11036_gb300 import tuning
    W = tg.workload("paper_c1")
    tabs = tg.hash_tables(W["hash_seed"])
    pairs = [to_dev(tg.traffic_for(W).slot(0)[0])]
    path = str(tmp_path / "tuning.json")
    ctx = ssd.Context(ssd.make_params(W["params"]), tabs)
    sk = [ctx.sketch()]
    first = tuning.tuned(ctx, sk, pairs, path=path, reps=1)
    assert len(tuning.load(path)) == 1
    ctx2 = ssd.Context(ssd.make_params(W["params"]), tabs)
    sk2 = [ctx2.sketch()]
    ctx2.tuning = dict(scan_unroll=1)
    second = tuning.tuned(ctx2, sk2, pairs, path=path, reps=1)
    assert second == first == ctx2.tuning
    ctx.close()
    ctx2.close()
