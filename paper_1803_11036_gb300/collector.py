"""Assembling a slot from distributed edge routers, with a deadline.

The paper's routers each scan their own traffic and ship their RSEAs to one monitor server, which
merges them at the end of every slot (Sec. 4, Algorithm 5); how routers fail or fall behind is left
open ("nodes communication, load balance": future work, Sec. 6). Here every router's slice of slot t
is submitted as it arrives. The slot is closed - one ssd_slot call over all routers - as soon as
every router has delivered or when the slot's deadline passes, whichever comes first. A router that
has not delivered by then is scanned as an empty slice: its sketch still advances one slot, so the
window stays aligned across routers, and the result names it and is marked partial (its packets of
that slot are missing from the list). A slice for a slot already closed is late: it is dropped and
counted. A slice for a later slot waits until that slot opens.

All decisions are made on the host from the clock and the submissions; nothing waits on the GPU
except reading a closed slot's list.
"""
from __future__ import annotations

import dataclasses
import time
from collections import defaultdict


@dataclasses.dataclass
class SlotResult:
    slot: int
    ips: object               # numpy uint32 array of sliding super points
    rk: object                # their R_k
    missing: list             # routers scanned as empty slices
    closed_by: str            # "complete" or "deadline"

    @property
    def partial(self) -> bool:
        return bool(self.missing)


class SlotCollector:
    """Collects one slice per router per slot and closes slots in order.

    ctx, routers, global_sketch: the detector context, one sketch per router (all at the same slot),
        and an optional merged sketch (as for Context.slot);
    deadline_s: how long a slot may stay open after it opened (the previous slot closed, or the
        first call for slot 0);
    clock: a function returning seconds (time.monotonic by default; tests pass their own);
    empty: a function returning an empty pair tensor on the context's device.
    """

    def __init__(self, ctx, routers, global_sketch=None, deadline_s: float = 1.0, clock=time.monotonic,
                 empty=None, cap: int = 1 << 16):
        self.ctx, self.routers, self.global_sketch = ctx, list(routers), global_sketch
        self.deadline_s = float(deadline_s)
        self.clock = clock
        self.cap = cap
        if empty is None:
            def empty():
                import torch
                return torch.empty(0, dtype=torch.int32, device=ctx.device)
        self._empty = empty
        self.slot = int(self.routers[0].slot) if hasattr(self.routers[0], "slot") else 0
        self._have: dict[int, object] = {}
        self._future: dict[int, dict[int, object]] = defaultdict(dict)
        self._opened: float | None = None
        self.late = 0             # slices dropped because their slot had closed
        self.duplicates = 0       # second slices of one router for one slot (the first is kept)

    # ---- submissions
    def submit(self, router: int, slot: int, pairs) -> str:
        """Hand over router's slice of `slot`: a device tensor of (cip, oip) pairs, as for
        Context.slot (it is read when the slot closes). Returns "accepted", "held" (a later slot),
        "late" or "duplicate"."""
        if not 0 <= router < len(self.routers):
            raise ValueError(f"no router {router}")
        if self._opened is None:
            self._opened = self.clock()
        if slot < self.slot:
            self.late += 1
            return "late"
        box = self._have if slot == self.slot else self._future[slot]
        if router in box:
            self.duplicates += 1
            return "duplicate"
        box[router] = pairs
        return "accepted" if slot == self.slot else "held"

    # ---- closing
    def due(self) -> str | None:
        """Why the open slot should close now ("complete", "deadline"), or None."""
        if len(self._have) == len(self.routers):
            return "complete"
        if self._opened is not None and self.clock() - self._opened >= self.deadline_s:
            return "deadline"
        return None

    def poll(self) -> list[SlotResult]:
        """Close every slot that is due (one, or several when held slices complete the next ones)."""
        out = []
        while True:
            why = self.due()
            if why is None:
                return out
            out.append(self._close(why))

    def close_now(self) -> SlotResult:
        """Close the open slot whatever has arrived (for example at shutdown)."""
        return self._close("deadline")

    def _close(self, why: str) -> SlotResult:
        missing = [r for r in range(len(self.routers)) if r not in self._have]
        pairs = [self._have[r] if r in self._have else self._empty() for r in range(len(self.routers))]
        ips, rk = self.ctx.slot(self.routers, pairs, self.global_sketch, cap=self.cap)
        res = SlotResult(self.slot, ips, rk, missing, why)
        self.slot += 1
        self._have = self._future.pop(self.slot, {})
        self._opened = self.clock()
        return res
