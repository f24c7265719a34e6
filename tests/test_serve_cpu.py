"""Host logic of the served form (no GPU): the latency summary over finished slices, the device
memory a router is admitted against, and admission refused once the router cap is reached (before
any device query)."""
import numpy as np
import pytest

import paper_1803_11036_gb300 as ssd
from paper_1803_11036_gb300 import serve

P = dict(log2_eta=11, q=17, r=5, delta=5, k=60, theta=1024)


def result(arrival, done, packets, router=0, slot=0):
    return serve.Result(router, slot, np.zeros(0, np.uint32), np.zeros(0, np.uint32), arrival, done, packets)


def test_latency_summary():
    res = [result(0.000, 0.001, 1000), result(0.010, 0.012, 3000), result(0.020, 0.030, 6000)]
    s = serve.latency_summary(res)
    assert s["slices"] == 3 and s["packets"] == 10000
    assert s["p50_ms"] == pytest.approx(2.0) and s["mean_ms"] == pytest.approx(13.0 / 3, abs=1e-3)
    assert s["p99_ms"] == pytest.approx(np.percentile([1.0, 2.0, 10.0], 99), abs=1e-3)
    assert s["span_s"] == pytest.approx(0.030) and s["mpps"] == pytest.approx(10000 / 0.030 / 1e6, abs=0.05)


def test_memory_a_router_is_admitted_against():
    tabs = np.zeros(2048, np.uint32)
    plain = serve.Server(ssd.make_params(P), tabs)
    reserved = serve.Server(ssd.make_params(P), tabs, max_slice_pairs=2_000_000)
    rsea = 5 << (17 + 11 + 1)                        # r * 2^q * eta * 2 bytes
    assert plain.bytes_per_router() >= rsea
    assert reserved.bytes_per_router() - plain.bytes_per_router() == 24 * 2_000_000


def test_router_cap_refuses_before_touching_the_device():
    srv = serve.Server(ssd.make_params(P), np.zeros(2048, np.uint32), max_routers=0)
    assert srv.try_admit(7) is False and srv.tenants == {} and srv.admitted_order == []
