"""Served form: many routers stream slices; each router's RSEA and window stay
resident on the device, routers are admitted by device memory, and slices are
processed as they arrive with continuous batching.

Each admitted router (tenant) owns a detector context, its RSEA and a CUDA
stream. A slice is one slot of that router's packets: scan + merge/regain/
advance in one ``ssd_slot_host`` call (Sec. 4), followed by the device-to-host
copy of the router's sliding super point list. Slices of different routers run
concurrently on their own streams; a router's slices run in arrival order on
its stream, so its window state is exactly what it would be alone. At most
``max_inflight`` slices are on the device at once; a slice that arrives while
the device is full waits in the ready queue and is admitted as soon as one
finishes. Latency is measured from a slice's arrival time to the moment its
list is on the host.
"""
from __future__ import annotations

import collections
import dataclasses
import heapq
import time

import numpy as np

from . import Context, SSDError, _abi


@dataclasses.dataclass
class Slice:
    router: int
    pairs: object            # pinned CPU tensor (or numpy array) of (cip, oip) pairs
    arrival: float           # seconds on the server clock
    seq: int = 0


@dataclasses.dataclass
class Result:
    router: int
    slot: int
    ips: np.ndarray
    rk: np.ndarray
    arrival: float
    done: float
    packets: int

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def device_free_bytes(device: int) -> int:
    import torch
    free, _ = torch.cuda.mem_get_info(device)
    return int(free)


class _Tenant:
    def __init__(self, params, tables, device, list_cap, max_slice_pairs=None, tuning=None):
        import torch
        self.ctx = Context(params, tables, device)
        if tuning:
            self.ctx.tuning = tuning
        if max_slice_pairs:
            # the pre-hash and staging buffers a slice of this size needs, allocated now: a later
            # slice never grows them, so no cudaFree / cudaMalloc stalls the other tenants' work
            self.ctx.reserve(max_slice_pairs)
        self.sketch = self.ctx.sketch()
        self.stream = torch.cuda.Stream(torch.device("cuda", device))
        self.slot = 0
        self.list_cap = list_cap

    def close(self):
        self.ctx.close()


class Server:
    """Request loop over many routers on one GPU."""

    def __init__(self, params, tables, device: int = 0, max_inflight: int = 16, list_cap: int = 4096,
                 reserve_bytes: int = 2 << 30, max_routers: int | None = None, evict_when_done: bool = False,
                 max_slice_pairs: int | None = None, tuning: dict | None = None):
        """max_slice_pairs: the largest slice a router sends; each admitted router reserves its
        buffers for it (see Context.reserve). tuning: a launch configuration for every router's
        context (for instance one picked by Context.autotune on a representative slice)."""
        import torch
        self.params, self.tables, self.device = params, tables, device
        self.max_inflight = max_inflight
        self.list_cap = list_cap
        self.reserve = reserve_bytes
        self.tenants: dict[int, _Tenant] = {}
        self.waiting_admission: collections.deque = collections.deque()
        self.ready: collections.deque = collections.deque()
        self.inflight: list = []
        self.results: list[Result] = []
        self.dev = torch.device("cuda", device)
        self._pool = []   # reusable (device ips, rk, n_out, pinned ips, rk, n_out) sets
        self.t0 = None
        self.admitted_order: list[int] = []
        self.max_routers = max_routers
        self.evict_when_done = evict_when_done
        self.max_slice_pairs = max_slice_pairs
        self.tuning = tuning
        self._left: collections.Counter = collections.Counter()   # scheduled slices not yet finished

    # ---- admission by device memory
    def bytes_per_router(self) -> int:
        p = self.params
        sketch = p.r << (p.q + p.log2_eta + 1)
        staged = 24 * (self.max_slice_pairs or 0)   # pre-hashed pairs + two host staging areas
        return int(sketch * 1.1) + (256 << 20) + staged   # RSEA + context scratch (pools, candidate buffers)

    def try_admit(self, router: int) -> bool:
        if router in self.tenants:
            return True
        if self.max_routers is not None and len(self.tenants) >= self.max_routers:
            return False
        if device_free_bytes(self.device) < self.bytes_per_router() + self.reserve:
            return False
        try:
            self.tenants[router] = _Tenant(self.params, self.tables, self.device, self.list_cap,
                                           self.max_slice_pairs, self.tuning)
        except SSDError as e:
            if e.code == _abi.SSD_ENOMEM:
                return False
            raise
        self.admitted_order.append(router)
        return True

    def evict(self, router: int) -> None:
        t = self.tenants.pop(router, None)
        if t is not None:
            t.stream.synchronize()
            t.close()

    # ---- buffers
    def _buffers(self):
        import torch
        if self._pool:
            return self._pool.pop()
        c = self.list_cap
        return (torch.empty(c, dtype=torch.int32, device=self.dev), torch.empty(c, dtype=torch.int32, device=self.dev),
                torch.zeros(1, dtype=torch.int64, device=self.dev),
                torch.empty(c, dtype=torch.int32).pin_memory(), torch.empty(c, dtype=torch.int32).pin_memory(),
                torch.zeros(1, dtype=torch.int64).pin_memory())

    def now(self) -> float:
        return time.perf_counter() - self.t0

    # ---- the loop
    def _launch(self, s: Slice):
        import torch
        ten = self.tenants[s.router]
        buf = self._buffers()
        dips, drk, dn, hips, hrk, hn = buf
        with torch.cuda.stream(ten.stream):
            ten.ctx.slot_host([ten.sketch], [s.pairs], None, out=(dips, drk, dn), stream=ten.stream, sync=False)
            hn.copy_(dn, non_blocking=True)
            hips.copy_(dips, non_blocking=True)
            hrk.copy_(drk, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(ten.stream)
        slot = ten.slot
        ten.slot += 1
        n = s.pairs.numel() // 2 if hasattr(s.pairs, "numel") else len(s.pairs)
        self.inflight.append((ev, s, slot, buf, n))

    def _reap(self):
        still = []
        for item in self.inflight:
            ev, s, slot, buf, n = item
            if ev.query():
                done = self.now()
                m = int(buf[5].item())
                if m > self.list_cap:
                    raise SSDError(_abi.SSD_ECAPACITY, f"router {s.router}: list of {m} > {self.list_cap}")
                ips = buf[3][:m].numpy().view(np.uint32).copy()
                rk = buf[4][:m].numpy().view(np.uint32).copy()
                self.results.append(Result(s.router, slot, ips, rk, s.arrival, done, n))
                self._pool.append(buf)
                self._left[s.router] -= 1
                if self.evict_when_done and self._left[s.router] == 0:
                    self.evict(s.router)   # its window ends here: free the memory for waiting routers
            else:
                still.append(item)
        self.inflight = still

    def run(self, slices, realtime: bool = True, poll_s: float = 20e-6) -> list[Result]:
        """Serve `slices` (Slice objects with arrival times). With realtime=True a slice becomes
        ready at its arrival time on the server clock; otherwise all are ready at once."""
        order = sorted(range(len(slices)), key=lambda i: (slices[i].arrival, i))
        pending = [(slices[i].arrival if realtime else 0.0, k, slices[i]) for k, i in enumerate(order)]
        heapq.heapify(pending)
        for s in slices:
            self._left[s.router] += 1
        self.t0 = time.perf_counter()
        while pending or self.ready or self.inflight or self.waiting_admission:
            now = self.now()
            while pending and pending[0][0] <= now:
                _, _, s = heapq.heappop(pending)
                if not realtime:
                    s.arrival = now
                self.waiting_admission.append(s)
            # admission: a router's first slice waits until its memory can be had
            nxt = collections.deque()
            while self.waiting_admission:
                s = self.waiting_admission.popleft()
                if s.router in self.tenants or self.try_admit(s.router):
                    self.ready.append(s)
                else:
                    nxt.append(s)
            self.waiting_admission = nxt
            # continuous batching: fill the device up to max_inflight
            while self.ready and len(self.inflight) < self.max_inflight:
                self._launch(self.ready.popleft())
            self._reap()
            if self.waiting_admission and not self.inflight and not self.ready and not pending:
                raise RuntimeError("routers waiting for device memory with nothing in flight to free it")
            if pending and not self.ready and not self.inflight:
                time.sleep(max(0.0, min(pending[0][0] - self.now(), 1e-3)))
            elif self.inflight:
                time.sleep(poll_s)
        return self.results

    def close(self):
        for r in list(self.tenants):
            self.evict(r)


def latency_summary(results) -> dict:
    lat = np.array([r.latency for r in results]) * 1e3
    pk = sum(r.packets for r in results)
    span = max(r.done for r in results) - min(r.arrival for r in results)
    return {"slices": len(results), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
            "mpps": round(pk / span / 1e6, 1), "packets": int(pk), "span_s": round(span, 4)}
