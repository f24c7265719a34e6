"""The library stores each distance recorder as a stamp (the slot of its last touch modulo 65535,
0xFFFF for distance 65535) next to a per-sketch clock. These tests pin that form against the
distances of Sec. 3.2 as the paper defines them:

- every one of the 65536 distance values, at clocks on both sides of every wrap (clock 0, the last
  clock 65534, the clocks where the window [tm - k + 1, tm] wraps past 65534), for k = 1, 2, 60,
  65533 and 65534, on estimators of 32 and 2048 recorders: an import reads back unchanged; the
  recorders inside the window (R_k summed per row) equal numpy's count of distances below k; an
  advance gives min(d + 1, 65535) for every recorder;
- whole slots of seeded traffic while the clock wraps from 65534 to 0, from a state that holds
  recorders at distances 65533 and 65534 (they reach 65535 during the run): every route's lists
  and every recorder equal the oracle's at every slot."""
import numpy as np
import pytest

import oracle
import paper_1803_11036_gb300 as ssd
import trafficgen as tg
from gpu_harness import assert_list_equal, to_dev

pytestmark = pytest.mark.gpu


def _every_distance(n: int, seed: int) -> np.ndarray:
    """n recorders holding each of the 65536 distances n / 65536 times, in a seeded order."""
    assert n % 65536 == 0
    a = np.tile(np.arange(65536, dtype=np.uint32), n // 65536).astype(np.uint16)
    np.random.default_rng(seed).shuffle(a)
    return a


def _row_counts(dist: np.ndarray, r: int, k: int) -> list[int]:
    return [int(x) for x in (dist.reshape(r, -1) < k).sum(axis=1)]


@pytest.mark.parametrize("dims", [dict(log2_eta=5, q=14, r=5, delta=6, theta=20),
                                  dict(log2_eta=11, q=11, r=5, delta=7, theta=1024)])
@pytest.mark.parametrize("k", [1, 2, 60, 65533, 65534])
def test_every_distance_at_every_clock_edge(dims, k):
    prm = dict(dims, k=k)
    ctx = ssd.Context(ssd.make_params(prm), tg.hash_tables(5))
    sk = ctx.sketch()
    n = ctx.sketch_bytes // 2
    dist = _every_distance(n, seed=k)
    advanced = np.minimum(dist.astype(np.uint32) + 1, 65535).astype(np.uint16)
    clocks = sorted({0, 1, max(k - 2, 0), k - 1, k, 65533, 65534})
    for tm in clocks:
        for slot in (tm, tm + 65535 * 3):          # the clock is the slot counter modulo 65535
            sk.load(dist, slot)
            assert np.array_equal(sk.export(), dist), (k, slot)
            assert sk.occupancy() == _row_counts(dist, prm["r"], k), (k, slot)
            ctx.advance([sk])
            assert sk.slot == slot + 1
            assert np.array_equal(sk.export(), advanced), (k, slot)
            assert sk.occupancy() == _row_counts(advanced, prm["r"], k), (k, slot)
    # a part read back at an offset that is not a multiple of 8 recorders
    sk.load(dist, 65534)
    assert np.array_equal(sk.export(13, 1001), dist[13:1014])
    ctx.close()


def _near_expiry(p, sk: np.ndarray, seed: int) -> None:
    """Sets some recorders of a distance array to 65533 and 65534 (they reach 65535 within two
    advances) and some to k - 1 (they leave the window at the next advance)."""
    rng = np.random.default_rng(seed)
    for v in (65533, 65534, p.k - 1):
        idx = rng.choice(sk.size, size=sk.size // 50, replace=False)
        sk[idx] = v


@pytest.mark.parametrize("route", ["slot", "close", "separate"])
@pytest.mark.parametrize("wl", ["paper_c1", "corelink_small"])
def test_slots_across_the_clock_wrap(wl, route):
    W = tg.workload(wl)
    W["traffic"]["count_a"] = min(W["traffic"]["count_a"], 1 << 17)
    prm = W["params"]
    p = oracle.params(prm)
    tabs = tg.hash_tables(W["hash_seed"])
    T = tg.Traffic(**W["traffic"])
    # chunked one-router slot: 8192 estimators per chunk, ten chunk launches at q = 14
    ctx = ssd.Context(ssd.make_params(prm, touch_chunk_bytes=2 << 20), tabs)
    router, glob = ctx.sketch(), ctx.sketch()
    sk = oracle.new_sketch(p)
    for t in range(3):                      # a state with recent traffic
        if t:
            oracle.advance(p, sk)
        oracle.scan(p, tabs, sk, T.slot(t)[0])
    oracle.advance(p, sk)
    _near_expiry(p, sk, seed=len(wl))
    start = 65535 - 3                       # the clock reaches 65534 and wraps to 0 during the run
    router.load(sk, start)
    listed = 0
    for i in range(p.k + 6):
        t = 3 + i
        pairs = T.slot(t)[0]
        if i:
            oracle.advance(p, sk)
        oracle.scan(p, tabs, sk, pairs)
        want = oracle.regain(p, tabs, sk, "pruned")
        dev = to_dev(pairs)
        if route == "slot":
            got = ctx.slot([router], [dev])
        elif route == "close":
            ctx.scan(router, dev)
            got = ctx.close_slot([router], glob)
            assert np.array_equal(glob.export(), sk), (wl, i)
        else:
            if i:
                ctx.advance([router])
            ctx.scan(router, dev)
            ctx.merge([router], glob)
            assert np.array_equal(glob.export(), sk), (wl, i)
            got = ctx.regain(glob)
        assert_list_equal(got, want, f"{wl} {route} slot {start + i}")
        listed += len(want["ips"])
        if route != "separate":            # the close advanced the router: compare one advance on
            adv = sk.copy()
            oracle.advance(p, adv)
            assert np.array_equal(router.export(), adv), (wl, route, i)
        else:
            assert np.array_equal(router.export(), sk), (wl, route, i)
    assert router.slot == start + p.k + 6 - (1 if route == "separate" else 0)
    assert listed > 0
    ctx.close()
