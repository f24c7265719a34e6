"""Failure detection on the host, with the GPU path real: four edge routers deliver slices to a
SlotCollector; one router's slice of slot 1 is withheld until after the deadline (then it arrives
late and is dropped), so slot 1 closes partial with that router scanned as an empty slice. Every
slot's list and merged sketch equal the oracle's on exactly the pairs that were scanned, and the
routers stay aligned: later slots close complete and still match."""
import numpy as np
import pytest

import paper_1803_11036_gb300 as ssd
import trafficgen as tg
from gpu_harness import Run, to_dev
from paper_1803_11036_gb300.collector import SlotCollector

pytestmark = pytest.mark.gpu


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def test_withheld_slice_closes_partial_and_matches_oracle():
    run = Run("edge_small")
    assert run.n == 4
    clock = Clock()
    col = SlotCollector(run.ctx, run.routers, run.glob, deadline_s=1.0, clock=clock)
    withheld = (1, 2)   # (slot, router)
    results = []
    for t in range(5):
        pairs = run.T.slot(t)
        scanned = []
        for r in range(run.n):
            if (t, r) == withheld:
                scanned.append(np.zeros((0, 2), dtype=np.uint32))
                continue
            assert col.submit(r, t, to_dev(pairs[r])) == "accepted"
            scanned.append(pairs[r])
        if t == withheld[0]:
            assert col.poll() == []          # not complete, deadline not reached
            clock.t += 1.0
        res = col.poll()
        assert len(res) == 1
        got = res[0]
        if t == withheld[0]:
            assert got.partial and got.missing == [withheld[1]] and got.closed_by == "deadline"
            assert col.submit(withheld[1], t, to_dev(pairs[withheld[1]])) == "late"
        else:
            assert not got.partial and got.closed_by == "complete"
        want = run.pipe.step(scanned, "pruned")
        assert np.array_equal(got.ips, want["ips"]) and np.array_equal(got.rk, want["rk"]), t
        assert np.array_equal(run.glob.export(), run.pipe.global_sk), t
        results.append(got)
    assert col.late == 1
    assert all(r.slot == 5 for r in run.routers)
    assert sum(len(r.ips) for r in results) > 0
    run.close()
