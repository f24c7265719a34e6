"""GB300 sliding super point detector (arXiv 1803.11036), Python binding.

Every step runs in the CUDA library behind ``include/ssd.h``; this module only
marshals arguments. PyTorch provides device memory (pair buffers and list
outputs are CUDA tensors) and streams. Names follow the paper: a router's
sketch is its RSEA, ``scan`` is Algorithm 2, ``advance`` the distance recorder
update, ``merge`` Algorithm 5, ``regain`` the reconstruction of sliding super
points, ``close_slot`` all end-of-slot work fused.

Typical slot loop on n routers::

    ctx = Context(params, tables)          # tables: 2048 uint32 (H1 then RHFG[0])
    routers = [ctx.sketch() for _ in range(n)]
    for each slot:
        ctx.scan_batch(routers, pair_tensors)          # or ctx.scan per router
        ips, rk = ctx.close_slot(routers)               # merge + regain + advance
"""
from __future__ import annotations

import ctypes
import weakref

import numpy as np

from ._abi import (SSD_ECAPACITY, SSD_MAX_GROUP_BITS, SSD_MAX_R, SSD_MAX_ROUTERS, SSD_NO_PRUNE, SSD_SIDE_CNET,  # noqa: F401
                   SSD_RHFG_LITERAL, SSD_SIDE_ONET, SSD_SLOT_CHUNKED,
                   SSD_STATUS_CTB_OVERFLOW,
                   SSD_STATUS_HSE_OVERFLOW, SSD_STATUS_LIST_OVERFLOW, SSD_STATUS_OUT_OVERFLOW, SSD_VERIFY_H0,
                   TUNING_FIELDS, Params, SSDError, Stats, Tuning, check, load)

__all__ = ["Context", "Sketch", "SlotGraph", "SSDError", "SSD_VERIFY_H0", "SSD_NO_PRUNE", "make_params",
           "threshold", "params_ok", "library_path"]


def library_path() -> str:
    from . import _abi
    return _abi.lib_path()


def make_params(d: dict, flags: int = 0, hse_capacity: int = 0, ctb_capacity: int = 0,
                out_capacity: int = 0, touch_chunk_bytes: int = 0) -> Params:
    """Params from a dict with log2_eta, q, r, delta, k, theta (and optional flags)."""
    return Params(d["log2_eta"], d["q"], d["r"], d["delta"], d["k"], d["theta"], d.get("flags", 0) | flags,
                  hse_capacity, ctb_capacity, out_capacity, touch_chunk_bytes)


def params_ok(p: Params) -> bool:
    return load().ssd_params_check(ctypes.byref(p)) == 0


def threshold(p: Params) -> int:
    thr = ctypes.c_uint32()
    check(load().ssd_threshold(ctypes.byref(p), ctypes.byref(thr)), "ssd_threshold")
    return thr.value


def _torch():
    import torch
    return torch


def _stream_handle(stream, device) -> ctypes.c_void_p:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _pairs_ptr(t, device):
    """Device pointer and packet count of a pair tensor: 4-byte integers, (n, 2) or (2n,), contiguous."""
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError("pairs must be a CUDA tensor")
    if t.device != device:
        raise ValueError(f"pairs on {t.device}, context on {device}")
    if t.element_size() != 4 or not t.is_contiguous():
        raise ValueError("pairs must be a contiguous tensor of 4-byte integers")
    n = t.numel()
    if n % 2:
        raise ValueError("pairs hold (cip, oip) couples: even element count")
    return ctypes.c_void_p(t.data_ptr() if n else 0), n // 2


class Sketch:
    """One RSEA on the device (a router's or the global one)."""

    def __init__(self, ctx: "Context"):
        self.ctx = ctx
        self._h = ctypes.c_void_p()
        check(ctx.L.ssd_sketch_create(ctx._h, ctypes.byref(self._h)), "ssd_sketch_create")
        ctx._sketches.add(self)

    @property
    def slot(self) -> int:
        v = ctypes.c_uint64()
        check(self.ctx.L.ssd_sketch_slot(self._h, ctypes.byref(v)), "ssd_sketch_slot")
        return v.value

    @slot.setter
    def slot(self, value: int) -> None:
        check(self.ctx.L.ssd_sketch_set_slot(self._h, value), "ssd_sketch_set_slot")

    @property
    def view(self) -> tuple[int, int, int]:
        """(side, group_bits, group): which hosts the sketch counts (see ssd_sketch_set_view)."""
        a, b, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        check(self.ctx.L.ssd_sketch_view(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
              "ssd_sketch_view")
        return a.value, b.value, c.value

    def set_view(self, side: int = SSD_SIDE_CNET, group_bits: int = 0, group: int = 0) -> "Sketch":
        """Count the hosts of `side` (SSD_SIDE_CNET: first field of a pair; SSD_SIDE_ONET: second)
        whose top group_bits bits are `group`. Before the sketch's first scan."""
        check(self.ctx.L.ssd_sketch_set_view(self._h, side, group_bits, group), "ssd_sketch_set_view")
        return self

    def occupancy(self, stream=None) -> list[int]:
        """Per row, the sum over its estimators of R_k (recorders below k); see ssd_sketch_occupancy."""
        out = (ctypes.c_uint64 * SSD_MAX_R)()
        check(self.ctx.L.ssd_sketch_occupancy(self._h, out, _stream_handle(stream, self.ctx.device)),
              "ssd_sketch_occupancy")
        return [int(x) for x in out[: self.ctx.params.r]]

    def device_view(self):
        """The sketch's stored recorders as a CUDA int16 tensor sharing the library's memory (no
        copy): the library's stamp form (the slot of a recorder's last touch modulo 65535, or 0xFFFF
        for distance 65535), not the distances; export() and export_device() give distances.
        Valid while the sketch lives; the caller orders its use against the context's stream."""
        torch = _torch()
        ptr = ctypes.c_void_p()
        check(self.ctx.L.ssd_sketch_data(self._h, ctypes.byref(ptr)), "ssd_sketch_data")
        n = self.ctx.sketch_bytes // 2

        class _Recorders:
            __cuda_array_interface__ = {"shape": (n,), "typestr": "<i2", "data": (ptr.value, False),
                                        "version": 2, "strides": None}

        return torch.as_tensor(_Recorders(), device=self.ctx.device)

    def export_device(self, out=None, first: int = 0, count: int | None = None, stream=None):
        """Distance recorders [first, first+count) written to a CUDA int16 tensor (`out`, or a new
        one) on the sketch's device; waits for the stream."""
        torch = _torch()
        n = self.ctx.sketch_bytes // 2
        count = n - first if count is None else count
        if out is None:
            out = torch.empty(count, dtype=torch.int16, device=self.ctx.device)
        if out.numel() != count or out.element_size() != 2 or not out.is_contiguous() or out.device != self.ctx.device:
            raise ValueError("out must be a contiguous 16-bit tensor of `count` elements on the sketch's device")
        check(self.ctx.L.ssd_sketch_export(self._h, first, count, ctypes.c_void_p(out.data_ptr()),
                                           _stream_handle(stream, self.ctx.device)), "ssd_sketch_export")
        return out

    def load_device(self, recorders, slot: int, stream=None) -> None:
        """Overwrite every recorder from a CUDA 16-bit tensor of distances and set the slot counter."""
        if recorders.numel() * recorders.element_size() != self.ctx.sketch_bytes or not recorders.is_contiguous():
            raise ValueError("recorder tensor has the wrong size")
        if recorders.device != self.ctx.device:
            raise ValueError("recorder tensor is on another device")
        check(self.ctx.L.ssd_sketch_import(self._h, ctypes.c_void_p(recorders.data_ptr()), slot,
                                           _stream_handle(stream, self.ctx.device)), "ssd_sketch_import")

    def export(self, first: int = 0, count: int | None = None, stream=None) -> np.ndarray:
        """Distance recorders [first, first+count) copied to a host uint16 array (waits for the
        stream)."""
        n = self.ctx.sketch_bytes // 2
        count = n - first if count is None else count
        out = np.empty(count, dtype=np.uint16)
        check(self.ctx.L.ssd_sketch_export(self._h, first, count, out.ctypes.data,
                                           _stream_handle(stream, self.ctx.device)), "ssd_sketch_export")
        return out

    def export_estimator(self, row: int, col: int, stream=None) -> np.ndarray:
        eta = 1 << self.ctx.params.log2_eta
        return self.export(((row << self.ctx.params.q) + col) * eta, eta, stream)

    def load(self, recorders: np.ndarray, slot: int, stream=None) -> None:
        """Overwrite every recorder from a host uint16 array of distances and set the slot counter."""
        a = np.ascontiguousarray(recorders, dtype=np.uint16)
        if a.nbytes != self.ctx.sketch_bytes:
            raise ValueError("recorder array has the wrong size")
        check(self.ctx.L.ssd_sketch_import(self._h, a.ctypes.data, slot,
                                           _stream_handle(stream, self.ctx.device)), "ssd_sketch_import")

    def close(self) -> None:
        if self._h:
            self.ctx.L.ssd_sketch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def _handles(sketches):
    arr = (ctypes.c_void_p * len(sketches))(*[s._h.value for s in sketches])
    return arr


class Context:
    """Detector parameters, hash tables and scratch on one CUDA device."""

    def __init__(self, params, tables, device: int = 0):
        self.L = load()
        self.params = params if isinstance(params, Params) else make_params(params)
        tab = np.ascontiguousarray(tables, dtype=np.uint32)
        if tab.size != 2048:
            raise ValueError("tables must hold 2048 uint32 words")
        torch = _torch()
        self.device = torch.device("cuda", device)
        self._h = ctypes.c_void_p()
        self._sketches = weakref.WeakSet()
        check(self.L.ssd_create(ctypes.byref(self.params), tab.ctypes.data, device, ctypes.byref(self._h)),
              "ssd_create")
        self.sketch_bytes = int(self.L.ssd_sketch_bytes(self._h))
        self.threshold = threshold(self.params)
        self._n_out = torch.zeros(1, dtype=torch.int64, device=self.device)

    def sketch(self) -> Sketch:
        return Sketch(self)

    # -- Algorithm 2 --
    def scan(self, sketch: Sketch, pairs, stream=None) -> None:
        ptr, n = _pairs_ptr(pairs, self.device)
        check(self.L.ssd_scan(sketch._h, ptr, n, _stream_handle(stream, self.device)), "ssd_scan")

    def scan_host(self, sketch: Sketch, pairs, stream=None) -> None:
        """Algorithm 2 on pairs in host memory: a (n, 2) uint32 numpy array or a CPU tensor
        (pinned for overlap). With pinned memory keep the buffer unchanged until the stream
        has passed this call."""
        torch = _torch()
        if isinstance(pairs, torch.Tensor):
            if pairs.is_cuda or pairs.element_size() != 4 or not pairs.is_contiguous():
                raise ValueError("host pairs: contiguous CPU tensor of 4-byte integers")
            ptr, n = pairs.data_ptr(), pairs.numel() // 2
        else:
            a = np.ascontiguousarray(pairs, dtype=np.uint32)
            ptr, n = a.ctypes.data, a.size // 2
            self._host_keep = a
        check(self.L.ssd_scan_host(sketch._h, ctypes.c_void_p(ptr), n, _stream_handle(stream, self.device)),
              "ssd_scan_host")

    def set_trace(self, ev_start=None, ev_pass=None, ev_end=None) -> None:
        """torch.cuda.Event objects recorded at the start, after the streaming pass and at the
        end of each close_slot / regain; all None switches tracing off."""
        h = [ctypes.c_void_p(e.cuda_event) if e is not None else None for e in (ev_start, ev_pass, ev_end)]
        check(self.L.ssd_set_trace(self._h, *h), "ssd_set_trace")

    def scan_batch(self, sketches, pairs_list, stream=None) -> None:
        if len(sketches) != len(pairs_list):
            raise ValueError("one pair tensor per sketch")
        ptrs, counts = [], []
        for t in pairs_list:
            p, n = _pairs_ptr(t, self.device)
            ptrs.append(p.value or 0)
            counts.append(n)
        P = (ctypes.c_void_p * len(ptrs))(*ptrs)
        N = (ctypes.c_uint64 * len(counts))(*counts)
        check(self.L.ssd_scan_batch(_handles(sketches), P, N, len(sketches), _stream_handle(stream, self.device)),
              "ssd_scan_batch")

    # -- Sec. 4.3 --
    def advance(self, sketches, stream=None) -> None:
        check(self.L.ssd_advance(_handles(sketches), len(sketches), _stream_handle(stream, self.device)),
              "ssd_advance")

    # -- Algorithm 5 --
    def merge(self, routers, global_sketch: Sketch, stream=None) -> None:
        check(self.L.ssd_merge(_handles(routers), len(routers), global_sketch._h,
                               _stream_handle(stream, self.device)), "ssd_merge")

    def _outputs(self, cap):
        torch = _torch()
        return (torch.empty(max(cap, 1), dtype=torch.int32, device=self.device),
                torch.empty(max(cap, 1), dtype=torch.int32, device=self.device))

    def min_merge(self, out, inputs, stream=None) -> None:
        """out[x] = min over the inputs of input[x] (ssd_min_merge): CUDA tensors of 16-bit
        recorders on this context's device, 16-byte aligned, all as long as `out`. The reduction of
        a merge whose routers are spread over GPUs (see shard.py)."""
        torch = _torch()
        for t in [out, *inputs]:
            if not isinstance(t, torch.Tensor) or t.device != self.device or t.element_size() != 2 or \
                    not t.is_contiguous():
                raise ValueError("min_merge takes contiguous 16-bit CUDA tensors on the context's device")
            if t.numel() != out.numel():
                raise ValueError("min_merge inputs and output differ in length")
        P = (ctypes.c_void_p * len(inputs))(*[t.data_ptr() for t in inputs])
        check(self.L.ssd_min_merge(self._h, ctypes.c_void_p(out.data_ptr()), P, len(inputs), out.numel(),
                                   _stream_handle(stream, self.device)), "ssd_min_merge")

    # -- Sec. 3.3 / 4.2 --
    def regain(self, global_sketch: Sketch, cap: int = 1 << 16, stream=None):
        """(ips, rk) as int64 CPU tensors of the unsigned values; raises SSDError on overflow."""
        ips, rk = self._outputs(cap)
        n = ctypes.c_uint64()
        rc = self.L.ssd_regain(self._h, global_sketch._h, ctypes.c_void_p(ips.data_ptr()),
                               ctypes.c_void_p(rk.data_ptr()), cap, ctypes.byref(n),
                               _stream_handle(stream, self.device))
        check(rc, "ssd_regain")
        m = n.value
        return ips[:m].cpu().numpy().view(np.uint32).copy(), rk[:m].cpu().numpy().view(np.uint32).copy()

    def close_slot(self, routers, global_sketch: Sketch | None = None, cap: int = 1 << 16, out=None,
                   stream=None, sync: bool = True):
        """Merge, regain and advance in one call. With sync=False returns the device
        tensors (ips, rk, n_out) without waiting; with sync=True returns host arrays."""
        if out is None:
            ips, rk = self._outputs(cap)
            n_out = self._n_out
        else:
            ips, rk, n_out = out
            cap = min(ips.numel(), rk.numel())
        st = _stream_handle(stream, self.device)
        check(self.L.ssd_close_slot(self._h, _handles(routers), len(routers),
                                    global_sketch._h if global_sketch is not None else None,
                                    ctypes.c_void_p(ips.data_ptr()), ctypes.c_void_p(rk.data_ptr()), cap,
                                    ctypes.c_void_p(n_out.data_ptr()), st), "ssd_close_slot")
        if not sync:
            return ips, rk, n_out
        s = self.stats(stream)
        if s["status"]:
            raise SSDError(SSD_ECAPACITY, f"ssd_close_slot (status {s['status']})")
        m = int(n_out.item())
        return ips[:m].cpu().numpy().view(np.uint32).copy(), rk[:m].cpu().numpy().view(np.uint32).copy()

    def slot(self, routers, pairs_list, global_sketch: Sketch | None = None, cap: int = 1 << 16, out=None,
             stream=None, sync: bool = True):
        """A whole slot: scan every router's pairs, then merge, regain and advance (one call,
        touches kept in L2). Same result and return convention as scan_batch + close_slot."""
        if len(routers) != len(pairs_list):
            raise ValueError("one pair tensor per router")
        ptrs, counts = [], []
        for t in pairs_list:
            p, n = _pairs_ptr(t, self.device)
            ptrs.append(p.value or 0)
            counts.append(n)
        P = (ctypes.c_void_p * len(ptrs))(*ptrs)
        N = (ctypes.c_uint64 * len(counts))(*counts)
        if out is None:
            ips, rk = self._outputs(cap)
            n_out = self._n_out
        else:
            ips, rk, n_out = out
            cap = min(ips.numel(), rk.numel())
        st = _stream_handle(stream, self.device)
        check(self.L.ssd_slot(self._h, _handles(routers), P, N, len(routers),
                              global_sketch._h if global_sketch is not None else None,
                              ctypes.c_void_p(ips.data_ptr()), ctypes.c_void_p(rk.data_ptr()), cap,
                              ctypes.c_void_p(n_out.data_ptr()), st), "ssd_slot")
        if not sync:
            return ips, rk, n_out
        s = self.stats(stream)
        if s["status"]:
            raise SSDError(SSD_ECAPACITY, f"ssd_slot (status {s['status']})")
        m = int(n_out.item())
        return ips[:m].cpu().numpy().view(np.uint32).copy(), rk[:m].cpu().numpy().view(np.uint32).copy()

    def slot_host(self, routers, host_pairs, global_sketch: Sketch | None = None, cap: int = 1 << 16, out=None,
                  stream=None, sync: bool = True):
        """slot() on pairs in host memory: (n, 2) uint32 numpy arrays or CPU tensors (pinned for
        overlap; keep them unchanged until the stream has passed this call)."""
        torch = _torch()
        if len(routers) != len(host_pairs):
            raise ValueError("one pair buffer per router")
        ptrs, counts, keep = [], [], []
        for h in host_pairs:
            if isinstance(h, torch.Tensor):
                if h.is_cuda or h.element_size() != 4 or not h.is_contiguous():
                    raise ValueError("host pairs: contiguous CPU tensor of 4-byte integers")
                ptrs.append(h.data_ptr() if h.numel() else 0)
                counts.append(h.numel() // 2)
            else:
                a = np.ascontiguousarray(h, dtype=np.uint32)
                keep.append(a)
                ptrs.append(a.ctypes.data if a.size else 0)
                counts.append(a.size // 2)
        self._host_keep = keep
        P = (ctypes.c_void_p * len(ptrs))(*ptrs)
        N = (ctypes.c_uint64 * len(counts))(*counts)
        if out is None:
            ips, rk = self._outputs(cap)
            n_out = self._n_out
        else:
            ips, rk, n_out = out
            cap = min(ips.numel(), rk.numel())
        st = _stream_handle(stream, self.device)
        check(self.L.ssd_slot_host(self._h, _handles(routers), P, N, len(routers),
                                   global_sketch._h if global_sketch is not None else None,
                                   ctypes.c_void_p(ips.data_ptr()), ctypes.c_void_p(rk.data_ptr()), cap,
                                   ctypes.c_void_p(n_out.data_ptr()), st), "ssd_slot_host")
        if not sync:
            return ips, rk, n_out
        s = self.stats(stream)
        if s["status"]:
            raise SSDError(SSD_ECAPACITY, f"ssd_slot_host (status {s['status']})")
        m = int(n_out.item())
        return ips[:m].cpu().numpy().view(np.uint32).copy(), rk[:m].cpu().numpy().view(np.uint32).copy()

    def reserve(self, max_pairs: int) -> None:
        """Allocate what slot()/slot_host() allocate on a first call with up to max_pairs pairs."""
        check(self.L.ssd_reserve(self._h, max_pairs), "ssd_reserve")

    @property
    def tuning(self) -> dict:
        """The launch configuration (ssd_tuning fields); no field changes a result."""
        t = Tuning()
        check(self.L.ssd_tuning_get(self._h, ctypes.byref(t)), "ssd_tuning_get")
        return {f: int(getattr(t, f)) for f in TUNING_FIELDS}

    @tuning.setter
    def tuning(self, value: dict) -> None:
        cur = self.tuning
        unknown = set(value) - set(TUNING_FIELDS)
        if unknown:
            raise ValueError(f"unknown tuning fields {sorted(unknown)}")
        cur.update({k: int(v) for k, v in value.items()})
        t = Tuning(**cur)
        check(self.L.ssd_tuning_set(self._h, ctypes.byref(t)), "ssd_tuning_set")

    def autotune(self, routers, pairs_list, global_sketch: Sketch | None = None, reps: int = 3,
                 stream=None) -> dict:
        """Pick the launch configuration by timing ssd_slot on one representative slot of pairs
        (device tensors, one per router). The sketches must not have run a slot yet and come back
        in their initial state. Returns the chosen configuration, which the context keeps."""
        if len(routers) != len(pairs_list):
            raise ValueError("one pair tensor per router")
        ptrs, counts = [], []
        for t in pairs_list:
            p, n = _pairs_ptr(t, self.device)
            ptrs.append(p.value or 0)
            counts.append(n)
        P = (ctypes.c_void_p * len(ptrs))(*ptrs)
        N = (ctypes.c_uint64 * len(counts))(*counts)
        out = Tuning()
        check(self.L.ssd_autotune(self._h, _handles(routers), P, N, len(routers),
                                  global_sketch._h if global_sketch is not None else None, reps,
                                  ctypes.byref(out), _stream_handle(stream, self.device)), "ssd_autotune")
        return {f: int(getattr(out, f)) for f in TUNING_FIELDS}

    def stats(self, stream=None) -> dict:
        st = Stats()
        check(self.L.ssd_stats_get(self._h, ctypes.byref(st), _stream_handle(stream, self.device)),
              "ssd_stats_get")
        r = self.params.r
        return dict(status=st.status, threshold=st.threshold, hot=list(st.hot)[:r], level=list(st.level)[:r],
                    raw=st.raw, n_out=st.n_out)

    @property
    def launch_count(self) -> int:
        return int(self.L.ssd_launch_count(self._h))

    def close(self) -> None:
        if self._h:
            for sk in list(self._sketches):
                sk.close()
            self.L.ssd_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class SlotGraph:
    """A whole slot (scan + merge + regain + advance, ``Context.slot``) captured once as a CUDA
    graph on fixed device buffers. Each replay processes the pairs currently in ``inputs``
    (router j's buffer holds exactly ``counts[j]`` pairs every slot), writes the list to
    ``ips``/``rk``/``n_out`` and advances the routers' slot counters as the call would have."""

    def __init__(self, ctx: Context, routers, counts, global_sketch: Sketch | None = None, cap: int = 1 << 16):
        torch = _torch()
        self.ctx, self.routers, self.global_sketch = ctx, list(routers), global_sketch
        self.inputs = [torch.zeros(2 * int(n), dtype=torch.int32, device=ctx.device) for n in counts]
        self.ips, self.rk = ctx._outputs(cap)
        self.n_out = torch.zeros(1, dtype=torch.int64, device=ctx.device)
        ctx.reserve(int(sum(counts)))
        slots = [r.slot for r in self.routers]
        gslot = global_sketch.slot if global_sketch is not None else None
        self.stream = torch.cuda.Stream(ctx.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            ctx.slot(self.routers, self.inputs, global_sketch, out=(self.ips, self.rk, self.n_out),
                     stream=torch.cuda.current_stream(), sync=False)
        # capture ran no kernels: put the host counters back
        for r, v in zip(self.routers, slots):
            r.slot = v
        if global_sketch is not None:
            global_sketch.slot = gslot
        self._epoch = int(ctx.L.ssd_buffer_epoch(ctx._h))

    def replay(self) -> None:
        """Run the captured slot on the current contents of `inputs` (asynchronous). Refuses when
        the context has replaced a buffer the graph holds since the capture (ssd_buffer_epoch)."""
        if not self.ctx._h or any(not r._h for r in self.routers) or \
                (self.global_sketch is not None and not self.global_sketch._h):
            raise RuntimeError("the context or a sketch of this graph has been closed")
        if int(self.ctx.L.ssd_buffer_epoch(self.ctx._h)) != self._epoch:
            raise RuntimeError("the context replaced buffers this graph holds (a new touch chunk size, "
                               "ssd_reserve or a larger slot); capture the slot again")
        merged = self.routers[0].slot
        self.graph.replay()
        for r in self.routers:
            r.slot = r.slot + 1
        if self.global_sketch is not None:
            self.global_sketch.slot = merged

    def result(self):
        """The list of the last replay as host arrays (waits for it)."""
        m = int(self.n_out.item())
        return (self.ips[:m].cpu().numpy().view(np.uint32).copy(),
                self.rk[:m].cpu().numpy().view(np.uint32).copy())
