"""The slot collector's host logic (no GPU): slots close when every router has delivered or at the
deadline, in order; missing routers are scanned as empty slices and named; late slices are dropped
and counted, duplicates kept once, slices for later slots held until their slot opens."""
import numpy as np

from paper_1803_11036_gb300.collector import SlotCollector


class FakeSketch:
    def __init__(self):
        self.slot = 0


class FakeCtx:
    """Records every ssd_slot call: the slot number and each router's pair count."""

    def __init__(self, routers):
        self.routers = routers
        self.calls = []

    def slot(self, routers, pairs, glob, cap):
        self.calls.append([len(p) for p in pairs])
        for r in routers:
            r.slot += 1
        return np.array([len(self.calls)], dtype=np.uint32), np.array([1], dtype=np.uint32)


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def make(n=3, deadline=1.0):
    routers = [FakeSketch() for _ in range(n)]
    ctx, clock = FakeCtx(routers), Clock()
    col = SlotCollector(ctx, routers, deadline_s=deadline, clock=clock, empty=lambda: [])
    return col, ctx, clock


def test_closes_when_complete():
    col, ctx, clock = make()
    assert col.submit(0, 0, [1, 2]) == "accepted"
    assert col.submit(1, 0, [3]) == "accepted"
    assert col.poll() == []
    col.submit(2, 0, [4, 5, 6])
    (res,) = col.poll()
    assert res.slot == 0 and not res.partial and res.closed_by == "complete"
    assert ctx.calls == [[2, 1, 3]] and col.slot == 1


def test_deadline_scans_missing_routers_empty():
    col, ctx, clock = make(deadline=0.5)
    col.submit(0, 0, [1])
    col.submit(2, 0, [1, 1])
    clock.t = 0.49
    assert col.poll() == []
    clock.t = 0.5
    (res,) = col.poll()
    assert res.partial and res.missing == [1] and res.closed_by == "deadline"
    assert ctx.calls == [[1, 0, 2]]
    assert [r.slot for r in ctx.routers] == [1, 1, 1]   # the missing router advanced too


def test_late_duplicate_and_held_slices():
    col, ctx, clock = make(n=2)
    assert col.submit(0, 1, [9]) == "held"               # slot 1 is not open yet
    col.submit(0, 0, [1])
    assert col.submit(0, 0, [2, 2]) == "duplicate"
    col.submit(1, 0, [1])
    (r0,) = col.poll()
    assert ctx.calls[-1] == [1, 1]                       # the first slice of router 0 was kept
    assert col.submit(1, 0, [5]) == "late"               # slot 0 has closed
    assert col.late == 1 and col.duplicates == 1
    col.submit(1, 1, [7, 7])
    (r1,) = col.poll()                                   # the held slice completes slot 1
    assert r1.slot == 1 and ctx.calls[-1] == [1, 2] and not r1.partial


def test_held_slices_can_close_several_slots():
    col, ctx, clock = make(n=2)
    for s in (1, 2):
        col.submit(0, s, [s])
        col.submit(1, s, [s, s])
    col.submit(0, 0, [0])
    col.submit(1, 0, [0])
    res = col.poll()
    assert [r.slot for r in res] == [0, 1, 2] and col.slot == 3
    assert ctx.calls == [[1, 1], [1, 2], [1, 2]]


def test_deadline_restarts_when_a_slot_closes():
    col, ctx, clock = make(n=2, deadline=1.0)
    col.submit(0, 0, [1])
    clock.t = 1.0
    (a,) = col.poll()
    assert a.missing == [1]
    clock.t = 1.5                                        # slot 1 opened at 1.0
    assert col.poll() == []
    clock.t = 2.0
    (b,) = col.poll()
    assert b.slot == 1 and b.missing == [0, 1]
