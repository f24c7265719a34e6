"""The seeded input generator: determinism and the workload shapes it promises."""
import numpy as np

import oracle
import trafficgen as tg


def test_deterministic_and_slot_distinct():
    T = tg.traffic_for("paper_c1")
    a, b = T.fill(3), T.fill(3)
    assert a.dtype == np.uint32 and a.shape == (1 << 18, 2)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, T.fill(4))
    many = T.fill_many([(3, 0), (4, 0)])
    assert np.array_equal(many[0], a)
    assert np.array_equal(tg.hash_tables(5), tg.hash_tables(5))
    assert not np.array_equal(tg.hash_tables(5), tg.hash_tables(6))


def test_planted_window_degree_is_exact():
    """Planted hosts cycle a list of D peers at ceil(D/k) per slot, so once the window is full
    their exact opposite number is D."""
    W = tg.workload("paper_c1")
    T = tg.traffic_for(W)
    k = W["params"]["k"]
    ex = oracle.Exact(k, W["params"]["theta"])
    for t in range(k + 1):
        ex.add_slot(T.slot(t)[0])
    ips, deg = ex.report()
    got = dict(zip(ips.tolist(), deg.tolist()))
    for ip, d in zip(T.planted_ips().tolist(), T.planted_degrees().tolist()):
        assert got[ip] == d


def test_repeat_fraction_and_hot_sources():
    W = tg.workload("stress_small")
    T = tg.traffic_for(W)
    pr = T.fill(0, 0)
    hot = set(T.hot_ips().tolist())
    frac_hot = np.isin(pr[:, 0], list(hot)).mean()
    assert abs(frac_hot - 10 * 0.05) < 0.02
    keys = pr[:, 0].astype(np.uint64) << np.uint64(32) | pr[:, 1].astype(np.uint64)
    dup = 1 - len(np.unique(keys)) / len(keys)
    assert dup > 0.5   # 60% repeats plus hot-source collisions


def test_router_counts_and_sharing():
    W = tg.workload("edge_small")
    T = tg.traffic_for(W)
    counts = [T.count(0, r) for r in range(T.routers)]
    assert len(set(counts)) == T.routers and min(counts) > 0
    srcs = [set(T.fill(0, r)[:, 0].tolist()) for r in range(T.routers)]
    inter = len(srcs[0] & srcs[1])
    assert inter > 0
    W4 = tg.workload("stress_small")
    T4 = tg.traffic_for(W4)
    assert sum(T4.count(0, r) for r in range(T4.routers)) == W4["traffic"]["count_a"]
