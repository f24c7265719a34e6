"""Named workloads: a traffic recipe plus the detector parameters it is run with.

Numbers only. ``params`` holds the sliding-estimator array dimensions and the
window/threshold (eta = 2**log2_eta distance recorders per estimator, 2**q
columns, r rows, shift step delta, window k slots, threshold theta);
``hash_seed`` seeds the two tabulation-hash table sets (``hash_tables``);
``traffic`` is the keyword set of ``trafficgen.Traffic``; ``slots`` is the run
length the parity tests use.

The full-size entries follow the five workload shapes of the detector's
evaluation plan (one core link, 16 and 32 edge routers, 64 served routers) on
synthetic traffic; the ``*_small`` entries keep each recipe's structure at a
size the single-threaded oracle finishes in seconds.
"""
from __future__ import annotations

import copy


def _p(log2_eta, q, r, delta, k, theta):
    return dict(log2_eta=log2_eta, q=q, r=r, delta=delta, k=k, theta=theta)


WORKLOADS = {
    # eta=64, q=9, r=5, delta=8: (r-2)*delta+q = 33 >= 32 with a 1-bit overlap; k=3, theta=40.
    "tiny": dict(
        params=_p(6, 9, 5, 8, 3, 40), hash_seed=7, slots=8,
        traffic=dict(seed=1000, n_src=48, zipf_s=1.2, deg_cap=24, rho=0.3, n_planted=4,
                     planted_lo=45, planted_hi=70, k=3, count="fixed", count_a=160)),
    # The paper's own dimensions (Sec. 5): eta=2^11, q=14, r=5, delta=6, theta=1024; window of 4 slots.
    "paper_c1": dict(
        params=_p(11, 14, 5, 6, 4, 1024), hash_seed=11, slots=12,
        traffic=dict(seed=1001, n_src=50_000, zipf_s=1.2, deg_cap=512, rho=0.3, n_planted=20,
                     planted_lo=2000, planted_hi=8000, k=4, count="fixed", count_a=1 << 18)),
    # One core-link router: 6.25M packets per one-second slot (40 Gb/s at 800 B), window of 60 slots.
    "corelink_c2": dict(
        params=_p(11, 18, 5, 5, 60, 1024), hash_seed=12, slots=68,
        traffic=dict(seed=1002, n_src=1_000_000, zipf_s=1.1, deg_cap=512, rho=0.3, n_planted=200,
                     planted_lo=1500, planted_hi=50_000, k=60, planted_mode=1, count="fixed",
                     count_a=6_250_000)),
    # 16 edge routers, lognormal(13, 1) packets per router-slot, 30% of sources at >= 2 routers.
    "edge16_c3": dict(
        params=_p(11, 18, 5, 5, 60, 1024), hash_seed=13, slots=68,
        traffic=dict(seed=1003, routers=16, n_src=1_000_000, zipf_s=1.1, deg_cap=512, rho=0.3,
                     shared_frac=0.3, n_planted=200, planted_lo=1500, planted_hi=50_000, k=60,
                     planted_mode=1, count="lognormal", ln_mu=13.0, ln_sigma=1.0)),
    # 32 routers, 15.6M packets per slot, 5000 hosts straddling the threshold, 10 hot sources.
    "stress32_c4": dict(
        params=_p(11, 18, 5, 5, 300, 1024), hash_seed=14, slots=304,
        traffic=dict(seed=1004, routers=32, n_src=4_000_000, zipf_s=1.1, deg_cap=64, rho=0.6,
                     n_planted=5000, planted_lo=900, planted_hi=1150, k=300, n_hot=10, hot_frac=0.05,
                     hot_peers=256, count="split", count_a=15_600_000)),
    # Per-tenant recipe of the served form: router-slots of uniform [10k, 2M] packets.
    "served_c5": dict(
        params=_p(11, 17, 5, 5, 60, 1024), hash_seed=15, slots=68,
        traffic=dict(seed=1005, n_src=1_000_000, zipf_s=1.1, deg_cap=512, rho=0.3, n_planted=20,
                     planted_lo=1500, planted_hi=50_000, k=60, planted_mode=1, count="uniform",
                     count_a=10_000, count_b=2_000_000)),
    # The core-link recipe at q=16 (a 1.25 GiB RSEA, still ten times L2) for profiler captures.
    "corelink_prof": dict(
        params=_p(11, 16, 5, 6, 60, 1024), hash_seed=12, slots=12,
        traffic=dict(seed=1012, n_src=250_000, zipf_s=1.1, deg_cap=512, rho=0.3, n_planted=50,
                     planted_lo=1500, planted_hi=50_000, k=60, planted_mode=1, count="fixed",
                     count_a=1_562_500)),
    # The core-link recipe at 1/16 scale (packets, sources, planted hosts; q=14 keeps the column
    # load near the full size's) for three windows of 60 slots: the long sliding-window accuracy
    # run against the exact counts (the precise algorithm is too slow for full-size windows).
    "corelink_acc": dict(
        params=_p(11, 14, 5, 6, 60, 1024), hash_seed=32, slots=180,
        traffic=dict(seed=3002, n_src=62_500, zipf_s=1.1, deg_cap=512, rho=0.3, n_planted=50,
                     planted_lo=1500, planted_hi=50_000, k=60, planted_mode=1, count="fixed",
                     count_a=390_625)),
    # ---- reduced sizes of the same recipes (element-by-element parity) ----
    "corelink_small": dict(
        params=_p(11, 14, 5, 6, 8, 1024), hash_seed=22, slots=14,
        traffic=dict(seed=2002, n_src=100_000, zipf_s=1.1, deg_cap=512, rho=0.3, n_planted=40,
                     planted_lo=1500, planted_hi=20_000, k=8, planted_mode=1, count="fixed",
                     count_a=400_000)),
    "edge_small": dict(
        params=_p(11, 14, 5, 6, 6, 1024), hash_seed=23, slots=10,
        traffic=dict(seed=2003, routers=4, n_src=100_000, zipf_s=1.1, deg_cap=512, rho=0.3,
                     shared_frac=0.3, n_planted=30, planted_lo=1500, planted_hi=12_000, k=6,
                     planted_mode=1, count="lognormal", ln_mu=11.5, ln_sigma=1.0)),
    "stress_small": dict(
        params=_p(11, 14, 5, 6, 8, 1024), hash_seed=24, slots=10,
        traffic=dict(seed=2004, routers=8, n_src=200_000, zipf_s=1.1, deg_cap=64, rho=0.6,
                     n_planted=300, planted_lo=900, planted_hi=1150, k=8, n_hot=10, hot_frac=0.05,
                     hot_peers=256, count="split", count_a=1_000_000)),
    "served_small": dict(
        params=_p(11, 14, 5, 6, 6, 1024), hash_seed=25, slots=10,
        traffic=dict(seed=2005, n_src=50_000, zipf_s=1.1, deg_cap=512, rho=0.3, n_planted=10,
                     planted_lo=1500, planted_hi=8000, k=6, planted_mode=1, count="uniform",
                     count_a=1_000, count_b=200_000)),
}


def workload(name: str) -> dict:
    """A deep copy of a named workload (callers may edit it)."""
    return copy.deepcopy(WORKLOADS[name])
