"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Each test ties one oracle function to something other than itself: a worked
example the paper prints, a closed form, an invariant, a special case that
reduces to a known function, or brute force. None of these needs a GPU.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
import trafficgen as tg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def P(log2_eta, q, r, delta, k, theta, flags=0):
    return oracle.Params(log2_eta, q, r, delta, k, theta, flags)


def identity_tables():
    """Tables with T_j[b] = b << 8j in both sets: the tabulation hash is then x itself."""
    t = np.zeros(2048, np.uint32)
    for s in (0, 1024):
        for j in range(4):
            t[s + 256 * j: s + 256 * (j + 1)] = (np.arange(256, dtype=np.uint64) << np.uint64(8 * j)).astype(np.uint32)
    return t


# ------------------------------------------------------------------ hashes

def test_tabulation_reduces_to_identity():
    """Special case: with T_j[b] = b<<8j, H1(oip) = oip mod eta and RHFG[0](cip) = cip mod 2^q.
    A wrong byte order, shift or table offset breaks this."""
    p = P(11, 14, 5, 6, 4, 1024)
    t = identity_tables()
    rng = np.random.default_rng(1)
    for x in list(rng.integers(0, 2**32, 300, dtype=np.uint64)) + [0, 1, 255, 256, 2**24, 2**32 - 1]:
        x = int(x)
        assert oracle.h1(p, t, x) == x % 2048
        assert int(oracle.rhfg(p, t, x)[0]) == x % (1 << 14)


def test_rhfg_row_i_only_depends_on_row0_and_window():
    """Eq. 2-3: RHFG[i](cip) XOR RHFG[0](cip) = B(i) does not depend on the random tables."""
    p = P(11, 14, 5, 6, 4, 1024)
    rng = np.random.default_rng(2)
    ta, tb = tg.hash_tables(5), tg.hash_tables(6)
    for x in rng.integers(0, 2**32, 200, dtype=np.uint64):
        ca, cb = oracle.rhfg(p, ta, int(x)), oracle.rhfg(p, tb, int(x))
        assert np.array_equal(ca[1:] ^ ca[0], cb[1:] ^ cb[0])


PARAM_SETS = [
    P(11, 14, 5, 6, 4, 1024),   # the paper's dimensions: (r-2)*delta+q = 32
    P(11, 18, 5, 5, 60, 1024),  # q=18: 33 bits of windows
    P(6, 9, 5, 8, 3, 40),       # tiny: 33 bits, 1-bit overlap
    P(11, 24, 3, 8, 4, 1024),   # r=3
    P(11, 16, 4, 8, 4, 1024),   # r=4
    P(11, 12, 6, 5, 4, 1024),   # r=6
]


@pytest.mark.parametrize("p", PARAM_SETS, ids=lambda p: f"q{p.q}r{p.r}d{p.delta}")
def test_rhfg_roundtrip_sampled(p):
    """Every bit of cip appears in some B(i) when (r-2)*delta+q >= 32 (Sec. 3.3): regaining a
    host from its own tuple gives it back, on 2^22 random values and the edge values."""
    t = tg.hash_tables(99)
    rng = np.random.default_rng(p.q * 131 + p.r)
    xs = rng.integers(0, 2**32, 1 << 22, dtype=np.uint64).astype(np.uint32)
    edges = np.array([0, 1, 2**31, 2**32 - 1, 0x80000001, 0x7FFFFFFF] + [1 << b for b in range(32)],
                     dtype=np.uint64).astype(np.uint32)
    assert oracle.roundtrip_failures(p, t, xs) == 0
    assert oracle.roundtrip_failures(p, t, edges) == 0


@pytest.mark.parametrize("p", PARAM_SETS, ids=lambda p: f"q{p.q}r{p.r}d{p.delta}")
def test_overlap_property_of_true_tuples(p):
    """Sec. 3.3: the high q-delta bits of B(i) equal the low q-delta bits of B(i+1)."""
    t = tg.hash_tables(3)
    rng = np.random.default_rng(7)
    w = p.q - p.delta
    for x in rng.integers(0, 2**32, 500, dtype=np.uint64):
        c = oracle.rhfg(p, t, int(x)).astype(np.int64)
        B = c ^ c[0]
        for i in range(2, p.r):
            assert (B[i - 1] >> p.delta) == (B[i] & ((1 << w) - 1))


def test_extract_rejects_window_bits_beyond_32():
    """Tiny dims cover 33 bits: a tuple whose last window has bit 32 set names no IPv4 host."""
    p = P(6, 9, 5, 8, 3, 40)
    t = tg.hash_tables(4)
    x = 0xDEADBEEF
    c = oracle.rhfg(p, t, x).astype(np.uint32)
    assert oracle.extract(p, c) == x
    bad = c.copy()
    bad[4] ^= np.uint32(1 << 8)   # B(4) covers bits 24..32; bit 8 of B(4) is bit 32 of cip
    assert oracle.extract(p, bad) is None
    worse = c.copy()
    worse[2] ^= np.uint32(1)      # breaks the B(1)/B(2) overlap
    assert oracle.extract(p, worse) is None


def test_bit_coverage_condition_is_needed():
    """With (r-2)*delta+q < 32 some bit of cip is in no window, and check_params refuses it."""
    assert oracle.check_params(P(11, 14, 5, 6, 4, 1024))
    assert not oracle.check_params(P(11, 13, 5, 6, 4, 1024))
    assert not oracle.check_params(P(11, 14, 5, 14, 4, 1024))  # delta < q
    assert not oracle.check_params(P(11, 14, 5, 6, 65535, 1024))
    assert oracle.check_params(P(11, 14, 5, 6, 65534, 1024))


# ---------------------------------------------------------------- threshold

@pytest.mark.parametrize("eta,theta", [(2048, 1024), (64, 40), (2048, 1), (2048, 5000), (32768, 1024),
                                       (256, 1024), (4096, 333)])
def test_threshold_is_eq1_inverse(eta, theta):
    """Sec. 3.3 defines R^_k so that Eq. 1 with z0 = eta - R^_k estimates exactly theta; the
    integer threshold is the first R_k whose Eq. 1 estimate reaches theta."""
    thr, rhat = oracle.threshold(eta, theta)
    assert math.isclose(-eta * math.log((eta - rhat) / eta), theta, rel_tol=1e-12)
    assert thr - 1 < rhat <= thr
    assert oracle.estimate(eta, thr) >= theta
    assert oracle.estimate(eta, thr - 1) < theta


def test_paper_parameters(golden):
    g = golden["experiment_parameters"]
    p = P(int(math.log2(g["eta"])), g["q"], g["r"], g["delta"], 4, g["theta"])
    assert 1 << p.log2_eta == g["eta"]
    assert oracle.check_params(p)
    assert (p.r - 2) * p.delta + p.q == 32
    b = golden["pair_buffer"]
    assert b["alpha"] == g["alpha"] and b["alpha"] * b["bytes_per_pair"] == b["kilobytes"] * 1024
    lw = golden["longest_window"]
    assert oracle.check_params(P(11, 14, 5, 6, lw["k_max"], 1024))
    assert not oracle.check_params(P(11, 14, 5, 6, lw["k_max"] + 1, 1024))
    assert round(lw["k_max"] / 3600, 1) == lw["hours_at_one_second_slots"]


def test_linear_counting_estimate_tracks_distinct_count():
    """Eq. 1 on one estimator fed m distinct opposite hosts estimates m (linear counting)."""
    p = P(11, 14, 5, 6, 1, 1024)
    t = tg.hash_tables(21)
    rng = np.random.default_rng(5)
    for m in (200, 1000, 3000):
        sk = oracle.new_sketch(p)
        oips = rng.choice(2**32, size=m, replace=False).astype(np.uint32)
        pairs = np.stack([np.full(m, 0x0A000001, np.uint32), oips], axis=1)
        oracle.scan(p, t, sk, pairs)
        col = int(oracle.rhfg(p, t, 0x0A000001)[0])
        rk = int(oracle.rk_row(p, sk, 0)[col])
        est = oracle.estimate(p.eta, rk)
        assert abs(est - m) < 0.1 * m, (m, rk, est)


# ------------------------------------------------------------------ sketch

def _recorder_index(p, t, cip, oip):
    cols = oracle.rhfg(p, t, cip)
    d = oracle.h1(p, t, oip)
    return [((i << p.q) + int(cols[i])) * p.eta + d for i in range(p.r)]


def _random_slots(rng, nslots, n, nsrc, peers):
    srcs = rng.integers(0, 2**32, nsrc, dtype=np.uint64).astype(np.uint32)
    out = []
    for _ in range(nslots):
        cnt = int(rng.integers(0, n + 1))
        s = srcs[rng.integers(0, nsrc, cnt)]
        o = rng.integers(0, peers, cnt).astype(np.uint32) * np.uint32(2654435761)
        out.append(np.stack([s, o], axis=1).astype(np.uint32))
    return out


def test_sketch_matches_closed_form():
    """Sec. 3.2: after slot t every recorder equals min(65535, t - s), s being the last slot in
    which some pair set it to 0 (65535 if never). Checked at every slot of a random stream."""
    p = P(5, 9, 5, 8, 3, 10)
    t = tg.hash_tables(8)
    rng = np.random.default_rng(11)
    slots = _random_slots(rng, 12, 300, 40, 5000)
    sk = oracle.new_sketch(p)
    last = np.full(sk.size, -1, dtype=np.int64)
    for ts, pairs in enumerate(slots):
        if ts:
            oracle.advance(p, sk)
        oracle.scan(p, t, sk, pairs)
        for cip, oip in pairs:
            for idx in _recorder_index(p, t, int(cip), int(oip)):
                last[idx] = ts
        expect = np.where(last < 0, 65535, np.minimum(65535, ts - last)).astype(np.uint16)
        assert np.array_equal(sk, expect), ts


def test_saturation_and_longest_window():
    """Recorders never pass 65535 (Sec. 3.2): after 65535 advances a recorder set at slot 0 reads
    65535 and stays there; one set at slot 1 reads 65534 = k_max, which is outside the window."""
    p = P(1, 6, 8, 5, 65534, 1)
    t = tg.hash_tables(9)
    sk = oracle.new_sketch(p)
    pa = np.array([[0x01020304, 77]], np.uint32)
    pb = np.array([[0x0A0B0C0D, 99]], np.uint32)
    oracle.scan(p, t, sk, pa)
    ia = _recorder_index(p, t, 0x01020304, 77)
    ib = _recorder_index(p, t, 0x0A0B0C0D, 99)
    oracle.advance(p, sk)
    oracle.scan(p, t, sk, pb)
    for _ in range(65534):
        oracle.advance(p, sk)
    assert all(sk[i] == 65535 for i in ia if i not in ib)
    assert all(sk[i] == 65534 for i in ib)
    assert all(oracle.rk_row(p, sk, r).sum() == 0 for r in range(p.r))  # 65534 is not < k
    for _ in range(3):
        oracle.advance(p, sk)
    assert sk.max() == 65535 and sk.min() == 65535


def test_scan_is_order_free():
    """Setting a recorder to 0 is idempotent (Sec. 4.1): any permutation of the pairs gives the
    same RSEA."""
    p = P(11, 14, 5, 6, 4, 1024)
    t = tg.hash_tables(12)
    pairs = tg.traffic_for("paper_c1").fill(0, n=20000)
    a, b = oracle.new_sketch(p), oracle.new_sketch(p)
    oracle.scan(p, t, a, pairs)
    oracle.scan(p, t, b, pairs[np.random.default_rng(0).permutation(len(pairs))])
    assert np.array_equal(a, b)


def test_slice_leaving_window_stops_counting():
    """A slot's pairs count for exactly k slots: k-1 advances later they are in R_k, k later not."""
    p = P(11, 14, 5, 6, 4, 1024)
    t = tg.hash_tables(13)
    sk = oracle.new_sketch(p)
    pairs = tg.traffic_for("paper_c1").fill(0, n=5000)
    oracle.scan(p, t, sk, pairs)
    for _ in range(p.k - 1):
        oracle.advance(p, sk)
    assert sum(int(oracle.rk_row(p, sk, r).sum()) for r in range(p.r)) > 0
    oracle.advance(p, sk)
    assert sum(int(oracle.rk_row(p, sk, r).sum()) for r in range(p.r)) == 0


def test_min_merge_equals_single_sketch_of_all_pairs():
    """Distributed equivalence (Sec. 4, Algorithm 5 with the min reading): n routers' sketches,
    each advanced every slot, merge into the sketch one router would hold had it seen every pair.
    Min commutes with the saturating +1. The literal max merge keeps only recorders seen by every
    router and does not."""
    p = P(8, 12, 6, 5, 3, 100)
    t = tg.hash_tables(14)
    rng = np.random.default_rng(3)
    R = 4
    routers = [oracle.new_sketch(p) for _ in range(R)]
    single = oracle.new_sketch(p)
    for ts in range(7):
        if ts:
            for sk in routers + [single]:
                oracle.advance(p, sk)
        for sk in routers:
            pr = _random_slots(rng, 1, 2000, 200, 100000)[0]
            oracle.scan(p, t, sk, pr)
            oracle.scan(p, t, single, pr)
        assert np.array_equal(oracle.merge(p, routers), single)
    pmax = P(8, 12, 6, 5, 3, 100, oracle.MAX_MERGE)
    assert not np.array_equal(oracle.merge(pmax, routers), single)


# ------------------------------------------------------------------ regain

def _pipeline_states(name, nslots):
    W = tg.workload(name)
    p = oracle.params(W["params"])
    tabs = tg.hash_tables(W["hash_seed"])
    T = tg.traffic_for(W)
    pipe = oracle.Pipeline(p, tabs, T.routers)
    for ts in range(nslots):
        pipe.step(T.slot(ts), regain_method=None)
        yield p, tabs, pipe.global_sk, T


@pytest.mark.parametrize("name,nslots", [("tiny", 8), ("paper_c1", 5)])
def test_recursive_and_levelwise_regain_agree(name, nslots):
    """Algorithms 3-4 (recursive) and 6-7 (level by level) are written separately; they must give
    the same list, the same R_k and the same candidate count at every row. The pruned form must
    give the same list."""
    for p, tabs, gsk, _ in _pipeline_states(name, nslots):
        for flags in (0, oracle.VERIFY_H0):
            pp = oracle.Params(*[getattr(p, f) for f in ("log2_eta", "q", "r", "delta", "k", "theta")], flags)
            a = oracle.regain(pp, tabs, gsk, "recursive")
            b = oracle.regain(pp, tabs, gsk, "levelwise")
            c = oracle.regain(pp, tabs, gsk, "pruned")
            assert np.array_equal(a["ips"], b["ips"]) and np.array_equal(a["rk"], b["rk"])
            assert np.array_equal(a["levels"], b["levels"])
            assert np.array_equal(b["ips"], c["ips"]) and np.array_equal(b["rk"], c["rk"])
            assert np.all(np.diff(b["ips"].astype(np.int64)) > 0)


_BF = None


def _bruteforce_lib():
    global _BF
    if _BF is None:
        out = os.path.join(ROOT, "tests", "_build", "libbrute.so")
        src = os.path.join(ROOT, "tests", "brute_force.c")
        os.makedirs(os.path.dirname(out), exist_ok=True)
        if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", out + ".tmp", src])
            os.replace(out + ".tmp", out)
        _BF = ctypes.CDLL(out)
        _BF.bf_enumerate.restype = ctypes.c_uint64
    return _BF


class _BfIn(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("log2_eta", "q", "r", "delta", "k", "thr")] + \
               [("tables", ctypes.c_void_p), ("hot", ctypes.c_void_p), ("bitmaps", ctypes.c_void_p),
                ("sh0", ctypes.c_uint32)]


def bruteforce(p, tabs, sk, verify, sh0=0):
    """All hosts in [0, 2^32) the definitions list, computed forward (see brute_force.c). sh0 is
    the bit where window B(1) starts: 0 for the (i-1)*delta windows, delta for Eq. 2 as printed."""
    thr, _ = oracle.threshold(p.eta, p.theta)
    below = (sk.reshape(p.r, p.C, p.eta) < p.k)
    rk = below.sum(axis=2)
    hot = (rk >= thr).astype(np.uint8)
    bm = np.packbits(below, axis=2, bitorder="little").view(np.uint32)
    bm = np.ascontiguousarray(bm)
    h0 = np.nonzero(hot[0])[0].astype(np.uint32)
    tabs = np.ascontiguousarray(tabs, np.uint32)
    cap = 1 << 20
    xs = np.empty(cap, np.uint32)
    rks = np.empty(cap, np.uint32)
    bi = _BfIn(p.log2_eta, p.q, p.r, p.delta, p.k, thr, tabs.ctypes.data, hot.ctypes.data, bm.ctypes.data, sh0)
    n = _bruteforce_lib().bf_enumerate(ctypes.byref(bi), int(verify), ctypes.c_void_p(h0.ctypes.data),
                                       ctypes.c_uint32(h0.size), ctypes.c_void_p(xs.ctypes.data),
                                       ctypes.c_void_p(rks.ctypes.data), ctypes.c_uint64(cap))
    assert n <= cap
    order = np.argsort(xs[:n])
    return xs[:n][order], rks[:n][order]


def _dense_tiny():
    """tiny dimensions with twelve planted hosts: many hot estimators, so with the 1-bit overlap
    the candidate tuples include many hosts' columns."""
    W = tg.workload("tiny")
    W["traffic"].update(n_planted=12, count_a=400)
    return W


@pytest.mark.slow
def test_regain_equals_bruteforce_over_all_ipv4():
    """Exhaustive pin: over every IPv4 value, the regained list equals the forward definition,
    with and without the RHFG[0] check."""
    for W in (tg.workload("tiny"), _dense_tiny()):
        p0 = oracle.params(W["params"])
        tabs = tg.hash_tables(W["hash_seed"])
        T = tg.Traffic(**W["traffic"])
        pipe = oracle.Pipeline(p0, tabs, T.routers)
        for ts in range(4):
            pipe.step(T.slot(ts), regain_method=None)
        for verify in (True, False):
            p = oracle.params(W["params"], oracle.VERIFY_H0 if verify else 0)
            got = oracle.regain(p, tabs, pipe.global_sk, "levelwise")
            bx, brk = bruteforce(p, tabs, pipe.global_sk, verify)
            assert np.array_equal(got["ips"], bx)
            assert np.array_equal(got["rk"], brk)
            assert len(bx) > 0


@pytest.mark.slow
def test_literal_shift_regain_equals_bruteforce_over_all_ipv4():
    """Completeness of Eq. 2 as printed (windows at i*delta): the sketch is scanned with the
    printed shift, and over every IPv4 value the regained list equals the forward definition -
    x is listed iff its own r estimators RHFG[i](x) are hot with union R_k >= threshold. A
    completion of bits 0..delta-1 that the regain wrongly dropped, or a host it made up, fails
    here; the soundness pins alone would pass both."""
    for W in (tg.workload("tiny"), _dense_tiny()):
        p = oracle.params(W["params"], oracle.RHFG_LITERAL)
        tabs = tg.hash_tables(W["hash_seed"])
        T = tg.Traffic(**W["traffic"])
        pipe = oracle.Pipeline(p, tabs, T.routers)
        total = 0
        for ts in range(4):
            pipe.step(T.slot(ts), regain_method=None)
            got = oracle.regain(p, tabs, pipe.global_sk, "levelwise")
            bx, brk = bruteforce(p, tabs, pipe.global_sk, True, sh0=p.delta)
            assert np.array_equal(got["ips"], bx), ts
            assert np.array_equal(got["rk"], brk), ts
            total += len(bx)
        assert total > 0


# ---------------------------------------------------------- precise algorithm

def test_precise_algorithm_paper_example(golden):
    g = golden["precise_algorithm_example"]
    names = {}
    ids = lambda s: names.setdefault(s, len(names) + 1)  # noqa: E731
    pairs = np.array([[ids(a), ids(b)] for a, b in g["pairs"]], np.uint32)
    ex = oracle.Exact(k=1, theta=1)
    ex.add_slot(pairs)
    ips, deg = ex.report()
    assert list(ips) == [ids("cip")] and list(deg) == [g["opposite_number"]]
    # the unsynchronised count the example warns about is the number of pairs inserted blindly
    assert len(g["pairs"]) == g["unsynchronised_parallel_count"]


def test_sliding_window_paper_example(golden):
    """Sec. 3.1: theta peers only in S5, k = 5 -> reported in SSP(1,5)..SSP(5,5) and, under
    discrete windows of the same length starting at S0, only in the second window."""
    g = golden["sliding_window_example"]
    k, theta, s5 = g["k"], 8, g["active_slot"]
    host = 0x0A000001
    ex = oracle.Exact(k=k, theta=theta)
    reported = []
    for ts in range(15):
        pr = np.array([[host, 1000 + j] for j in range(theta)], np.uint32) if ts == s5 else \
            np.array([[0x0B000000 + ts, 7]], np.uint32)
        ex.add_slot(pr)
        ips, _ = ex.report()
        if host in ips:
            reported.append(ts - k + 1)   # window SW(i, k) ends at slot i+k-1
    assert reported == g["sliding_windows_reporting"]
    dis = oracle.Exact(k=1, theta=theta)  # discrete window of k slots: one merged slot per window
    rep = []
    for w in range(3):
        slots = [np.array([[host, 1000 + j] for j in range(theta)], np.uint32) if ts == s5 else
                 np.zeros((0, 2), np.uint32) for ts in range(w * k, (w + 1) * k)]
        dis.add_slot(np.concatenate(slots))
        if host in dis.report()[0]:
            rep.append(w)
    assert rep == g["discrete_window_reporting"]


def test_sliding_example_through_the_sketch(golden):
    """The same example through the sliding estimator array: the host is regained at the end of
    S5..S9 and not before or after (2*theta peers keep the estimate clear of the threshold)."""
    g = golden["sliding_window_example"]
    k = g["k"]
    p = P(11, 14, 5, 6, k, 1024)
    tabs = tg.hash_tables(31)
    host = 0xC0A80101
    pipe = oracle.Pipeline(p, tabs, 1)
    seen = []
    for ts in range(13):
        pr = np.array([[host, 0x50000000 + j] for j in range(2 * p.theta)], np.uint32) if ts == g["active_slot"] \
            else np.zeros((0, 2), np.uint32)
        res = pipe.step([pr])
        if host in res["ips"]:
            seen.append(ts - k + 1)
    assert seen == g["sliding_windows_reporting"]


def test_precise_counter_bruteforce():
    """Exact counter against recomputing each window's distinct pairs from scratch."""
    rng = np.random.default_rng(17)
    k, theta = 3, 5
    slots = _random_slots(rng, 10, 120, 6, 40)
    ex = oracle.Exact(k=k, theta=theta)
    for ts in range(len(slots)):
        ex.add_slot(slots[ts])
        ips, deg = ex.report()
        window = set()
        for s in range(max(0, ts - k + 1), ts + 1):
            window |= {(int(a), int(b)) for a, b in slots[s]}
        counts = {}
        for a, _ in window:
            counts[a] = counts.get(a, 0) + 1
        expect = sorted((a, c) for a, c in counts.items() if c >= theta)
        assert list(zip(ips.tolist(), deg.tolist())) == expect
        for a, c in counts.items():
            assert ex.degree(a) == c


def test_views_swap_and_partition():
    """Sec. 3.1 / Sec. 6 views: the ONet view of a swapped stream is the CNet view of the original,
    sketch for sketch; the groups of one group_bits split the pairs into disjoint parts that
    together hold every pair, and each part holds only its group's hosts."""
    W = tg.workload("tiny")
    p = oracle.params(W["params"])
    tabs = tg.hash_tables(W["hash_seed"])
    pairs = tg.traffic_for(W).slot(0)[0]
    swapped = np.ascontiguousarray(pairs[:, ::-1])
    a, b = oracle.new_sketch(p), oracle.new_sketch(p)
    oracle.scan(p, tabs, a, oracle.view_pairs(pairs))
    oracle.scan(p, tabs, b, oracle.view_pairs(swapped, side=1))
    assert np.array_equal(a, b)
    assert np.array_equal(oracle.view_pairs(pairs), pairs)
    for gb in (1, 3):
        parts = [oracle.view_pairs(pairs, 0, gb, g) for g in range(1 << gb)]
        assert sum(len(x) for x in parts) == len(pairs)
        for g, part in enumerate(parts):
            assert oracle.in_group(part[:, 0], gb, g).all()
        both = np.concatenate(parts)
        key = lambda a_: a_[:, 0].astype(np.uint64) << np.uint64(32) | a_[:, 1]
        assert np.array_equal(np.sort(key(both)), np.sort(key(pairs)))


@pytest.mark.parametrize("p", PARAM_SETS[:3], ids=lambda p: f"q{p.q}r{p.r}d{p.delta}")
def test_literal_shift_loses_low_bits_and_completion_recovers_them(p):
    """Eq. 2 as printed (windows at i*delta): hosts that differ only in bits 0..delta-1 share
    every window B(1..r-1), so no tuple can tell them apart; the extraction fixes bits
    delta..31 and, among the 2^delta completions, the host is one whose RHFG[0] is he_0."""
    lit = oracle.Params(*[getattr(p, f) for f in ("log2_eta", "q", "r", "delta", "k", "theta")],
                        oracle.RHFG_LITERAL)
    t = tg.hash_tables(77)
    rng = np.random.default_rng(p.q)
    low = (1 << p.delta) - 1
    extra = 0
    for x in rng.integers(0, 2**32, 300, dtype=np.uint64).astype(np.uint32).tolist():
        cols = oracle.rhfg(lit, t, x)
        y = x ^ 1                     # differs in bit 0 only
        cy = oracle.rhfg(lit, t, y)
        assert np.array_equal(cols[1:] ^ cols[0], cy[1:] ^ cy[0])
        prefix = oracle.extract(lit, cols)
        assert prefix == x & ~low & 0xFFFFFFFF
        hits = [prefix | v for v in range(1 << p.delta) if oracle.rhfg(lit, t, prefix | v)[0] == cols[0]]
        assert x in hits
        extra += len(hits) - 1
    expected = 300 * ((1 << p.delta) - 1) / (1 << p.q)   # each wrong completion passes with odds 2^-q
    assert extra < 2 * expected + 30


@pytest.mark.parametrize("name,nslots", [("tiny", 6), ("paper_c1", 4)])
def test_literal_shift_regain_forms_agree(name, nslots):
    """Under Eq. 2 as printed the recursive, level-wise and pruned regains still agree, and every
    listed host's tuple of columns (from its own RHFG) has all r estimators hot."""
    W = tg.workload(name)
    p = oracle.params(W["params"], oracle.RHFG_LITERAL)
    tabs = tg.hash_tables(W["hash_seed"])
    T = tg.traffic_for(W)
    pipe = oracle.Pipeline(p, tabs, T.routers)
    thr, _ = oracle.threshold(p.eta, p.theta)
    listed = 0
    for ts in range(nslots):
        pipe.step(T.slot(ts), regain_method=None)
        gsk = pipe.global_sk
        a = oracle.regain(p, tabs, gsk, "recursive")
        b = oracle.regain(p, tabs, gsk, "levelwise")
        c = oracle.regain(p, tabs, gsk, "pruned")
        assert np.array_equal(a["ips"], b["ips"]) and np.array_equal(a["rk"], b["rk"])
        assert np.array_equal(a["levels"], b["levels"])
        assert np.array_equal(b["ips"], c["ips"]) and np.array_equal(b["rk"], c["rk"])
        for x in b["ips"].tolist():
            cols = oracle.rhfg(p, tabs, x)
            assert all(oracle.rk_row(p, gsk, i)[cols[i]] >= thr for i in range(p.r))
        listed += len(b["ips"])
    assert listed > 0


@pytest.mark.parametrize("name", ["paper_c1", "edge_small"])
def test_sampled_estimators_follow_the_full_sketch(name):
    """oracle.Sampled (Algorithm 2 and the recorder update restricted to chosen estimators, the
    oracle of the full-size tests) equals the full RSEA of the oracle's pipeline on every chosen
    estimator of every router after every slot: two separate routines (a hashed subset against the
    whole array) agree."""
    W = tg.workload(name)
    p = oracle.params(W["params"])
    tabs = tg.hash_tables(W["hash_seed"])
    T = tg.traffic_for(W)
    rng = np.random.default_rng(3)
    hosts = T.planted_ips()[:5].tolist()
    rows = [i for _ in hosts for i in range(p.r)] + rng.integers(0, p.r, 60).tolist()
    cols = [int(c) for x in hosts for c in oracle.rhfg(p, tabs, x)] + rng.integers(0, p.C, 60).tolist()
    rows = np.array(rows, dtype=np.uint32)
    cols = np.array(cols, dtype=np.uint32)
    pipe = oracle.Pipeline(p, tabs, T.routers)
    samp = [oracle.Sampled(p, rows, cols) for _ in range(T.routers)]
    touched = 0
    for t in range(4):
        pairs = T.slot(t)
        pipe.step(pairs, regain_method=None)
        for j in range(T.routers):
            if t:
                samp[j].advance()
            samp[j].scan(tabs, pairs[j])
            full = pipe.routers[j].reshape(p.r, p.C, p.eta)
            for r_, c_ in zip(rows.tolist(), cols.tolist()):
                got = samp[j].get(r_, c_)
                assert np.array_equal(got, full[r_, c_]), (t, j, r_, c_)
                touched += int((got < p.k).sum())
    assert touched > 0


def test_oracle_lists_match_the_committed_fixture():
    """The oracle's lists, R_k, level counts and staged tuples for two seeded workloads equal those
    written by tests/golden/make_oracle_lists.py when the fixture was made: a change to the oracle's
    arithmetic shows here and must come with a regenerated fixture."""
    import json
    import importlib.util
    here = os.path.join(ROOT, "tests", "golden")
    spec = importlib.util.spec_from_file_location("make_oracle_lists", os.path.join(here, "make_oracle_lists.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(os.path.join(here, "oracle_lists.json")) as f:
        want = json.load(f)
    assert mod.compute() == want
