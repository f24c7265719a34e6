#!/usr/bin/env python
"""Benchmark of the sliding super point detector's hot path on one GB300 per rank.

One step = one time slot of the whole path on the workload's routers: scan the
slot's packets (Algorithm 2), then close the slot - merge, hot-estimator
extraction and window advance in one streaming pass, candidate levels, final
test and the sorted list. Inputs are resident in HBM before timing; every step
scans a distinct slice, and the 5 GiB RSEA streamed every step is far larger
than L2. `e2e` repeats the steps through the C ABI from pinned host buffers
(host->device pair copies and the device->host list read inside the timed
region).

    python bench.py [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Under torchrun each rank runs an independent replica (its own traffic seed) on
its own GPU; rank 0 prints one JSON line with the whole-job throughput.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "scan Mpps (Gb/s @800B) + reconstruct ms/slice, batched vs plain, 1 GB300"
DEFAULT_WORKLOAD = "corelink_c2"
PAPER_PACKET_BYTES = 800


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--fill", type=int, default=-1, help="untimed slots before warm-up (default: k)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-stress", action="store_true", help="skip the 32-router batched-vs-plain leg")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-c1", action="store_true", help="skip the leg at the paper's own dimensions")
    ap.add_argument("--touch-chunk-mib", type=int, default=0, help="touch bits per chunk of the fused slot")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch configuration")
    ap.add_argument("--tuning", default="", help="launch configuration as JSON (ssd_tuning fields), "
                    "set instead of running the autotuner, e.g. to profile the configuration a run chose")
    return ap.parse_args()


# ------------------------------------------------------------ distributed

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, local):
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x: float, world: int, op: str) -> float:
    """Max or sum of a float over the ranks (CUDA tensors under NCCL, CPU tensors under gloo)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(x: float, world: int) -> float:
    return _reduce(x, world, "max")


def sum_over_ranks(x: float, world: int) -> float:
    return _reduce(x, world, "sum")


def replica_workload(name: str, rank: int) -> dict:
    """The workload a rank runs: the same parameters, an independent traffic seed per rank."""
    import trafficgen as tg
    W = tg.workload(name)
    W["_name"] = name
    if rank:
        W["traffic"]["seed"] += 7919 * rank
    return W


# ------------------------------------------------------------------ clocks

class Clocks:
    """nvidia-smi samples during the timed region (every 50 ms)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------- misc

def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _code_tokens(text: str) -> str:
    """C/CUDA source without comments and whitespace (string literals kept as written), so that a
    comment or layout edit leaves the kernel's hash alone."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if text.startswith("//", i):
            i = text.find("\n", i)
            i = n if i < 0 else i
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        elif c == '"':
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif c.isspace():
            out.append(" ")
            while i < n and text[i].isspace():
                i += 1
        else:
            out.append(c)
            i += 1
    return re.sub(r"\s+", " ", "".join(out)).strip()


def kernel_source_hash() -> str:
    """Hash of the chunk kernel's sources (code only) for matching a committed profile."""
    h = hashlib.sha256()
    for f in ("ssd_stream.cu", "ssd_internal.cuh"):
        h.update(_code_tokens(open(os.path.join(ROOT, "paper_1803_11036_gb300", "csrc", f)).read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, chunk: int, path: str | None = None, collect: int | None = None):
    """DRAM bytes per chunk launch of the streaming pass from the committed ncu summary, if
    the kernel source has not changed since it was captured, the launch covers as many
    estimators as the captured one and, when `collect` is given, the summary was taken on the
    same touch-collection route (ssd_tuning's collect_touches)."""
    path = path or os.path.join(ROOT, "profiles", f"chunk_pass_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    c = re.search(r"chunk_estimators:\s*([0-9]+)", text)
    if not m or not h or not c or h.group(1) != kernel_source_hash() or int(c.group(1)) != chunk:
        return None
    if collect is not None:
        r = re.search(r"collect_touches:\s*([0-9]+)", text)
        if not r or int(r.group(1)) != collect:
            return None
    return float(m.group(1))


def gbps(mpps: float):
    return {"si": round(mpps * PAPER_PACKET_BYTES * 8 / 1000, 2),
            "paper_convention": round(mpps * PAPER_PACKET_BYTES * 8 / 1024, 2)}


def traced(ctx, stream, calls):
    """Run each call (one slot, or one slot close) with trace events at its phase boundaries;
    returns the per-call milliseconds of the streaming pass (start -> pass) and of the candidate
    levels and list (pass -> end)."""
    import torch
    E = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in calls]
    with torch.cuda.stream(stream):
        for e, call in zip(E, calls):
            for ev in e:
                ev.record(stream)   # torch marks them recorded; the library re-records them in place
            ctx.set_trace(e[0], e[1], e[2])
            call()
    stream.synchronize()
    ctx.set_trace()
    return [e[0].elapsed_time(e[1]) for e in E], [e[1].elapsed_time(e[2]) for e in E]


def step_rooflines(pk, scan_ms, scan_pk, slot_pass, slot_tail, close_pass, close_tail, rec_bytes, r, peak):
    """Each step of the slot against its own roofline (algorithmic bytes / time / measured HBM).
    scan: 8 B pair read + r x 2 B recorder writes per packet (Algorithm 2); streaming pass: every
    recorder of every router read once, 2 B (rec_bytes), since with stamp recorders the advance
    writes nothing but the recorders that reach distance 65535; the slot's pass adds the scan's
    bytes; the candidate levels and the list are latency-bound (a few MB of bitmaps in L2 per
    slot), so only their time is given."""
    scan_b = 8 + 2 * r
    sp, cp = statistics.mean(slot_pass), statistics.mean(close_pass)
    marginal = sp - cp
    pass_bytes = rec_bytes + scan_b * pk
    def frac(b, ms):
        return None if ms <= 0 else round(b / (ms / 1e3) / 1e9 / peak, 4)
    def gbs(b, ms):
        return None if ms <= 0 else round(b / (ms / 1e3) / 1e9, 1)
    return {
        "scan_standalone": {
            "what": "ssd_scan_batch alone: Algorithm 2 storing r recorders per packet directly",
            "ms_per_slice": round(scan_ms, 4), "gpps": round(scan_pk / scan_ms / 1e6, 2),
            "algorithmic_bytes_per_packet": scan_b, "achieved_gbs": gbs(scan_b * scan_pk, scan_ms),
            "bound": "hbm (random 32 B sector read-modify-writes)", "frac": frac(scan_b * scan_pk, scan_ms)},
        "scan_in_slot": {
            "what": "the scan's marginal cost inside ssd_slot: streaming pass with the scan's touches "
                    "minus the close-only pass, same slices",
            "ms_per_slice": round(marginal, 4), "gpps": round(pk / marginal / 1e6, 2) if marginal > 0 else None,
            "algorithmic_bytes_per_packet": scan_b, "achieved_gbs": gbs(scan_b * pk, marginal),
            "bound": "l2 atomics (touch bits)", "frac": frac(scan_b * pk, marginal),
            "target_frac": 0.5, "target_met": bool(marginal > 0 and scan_b * pk / (marginal / 1e3) / 1e9 >= 0.5 * peak)},
        "slot_pass": {
            "what": "streaming pass of ssd_slot with the scan inside (touch lists, chunk launches: touches "
                    "applied, hot extraction, advance, next chunk's touches)",
            "ms_per_slice": round(sp, 4), "algorithmic_bytes": pass_bytes,
            "algorithmic_bytes_model": "2 B read per recorder + 18 B per packet (8 B pair read + r x 2 B "
                                       "recorder writes)",
            "achieved_gbs": gbs(pass_bytes, sp), "bound": "hbm", "frac": frac(pass_bytes, sp)},
        "close_pass": {
            "what": "ssd_close_slot's streaming pass with no scan (merge, hot extraction, advance: one launch)",
            "ms_per_slice": round(cp, 4), "algorithmic_bytes": rec_bytes,
            "algorithmic_bytes_model": "2 B read per recorder",
            "achieved_gbs": gbs(rec_bytes, cp), "bound": "hbm", "frac": frac(rec_bytes, cp)},
        "regain_tail": {
            "what": "pair level, row levels, final test and the sorted list (five launches)",
            "ms_per_slice": round(statistics.mean(slot_tail), 4),
            "ms_per_slice_after_close_only": round(statistics.mean(close_tail), 4),
            "bound": "latency (a few MB of bitmaps in L2; SMs mostly idle)"},
        "peak_gbs": peak,
        "measured": "CUDA events on the launching stream (ssd_set_trace) over 10 slots run right after the "
                    "timed region on the same slices, then 10 closes with no scan",
    }


# ---------------------------------------------------------- CPU oracle leg

def oracle_sample(W: dict, scale_log2: int = 0):
    """The workload for the single-threaded oracle: the same recipe, or (scale_log2 = s > 0) with
    2^s fewer columns and 2^s fewer packets per slot, which keeps the recorder bytes per packet
    (the advance and merge passes) equal to the full workload's."""
    import trafficgen as tg
    S = tg.workload(W["_name"]) if "_name" in W else W
    S = json.loads(json.dumps(S))
    name = W.get("_name", "workload")
    if not scale_log2:
        prm = S["params"]
        return S, (f"{name} as timed (q={prm['q']}, {S['traffic'].get('count_a')} packets/slot/router); "
                   f"advance+scan+merge+regain per slot, window starting empty")
    prm = S["params"]
    q = prm["q"] - scale_log2
    r = prm["r"]
    delta = max(1, -(-(32 - q) // (r - 2)))
    prm.update(q=q, delta=delta)
    tr = S["traffic"]
    if tr.get("count") in ("fixed", "split"):
        tr["count_a"] = max(1, tr["count_a"] >> scale_log2)
    tr["n_src"] = max(1, tr["n_src"] >> scale_log2)
    desc = (f"{name} recipe at 1/{1 << scale_log2} scale: q={q}, delta={delta}, "
            f"{tr.get('count_a')} packets/slot/router, {tr['n_src']} sources; advance+scan+merge+regain per slot")
    return S, desc


class OracleSlots:
    def __init__(self, W: dict, scale_log2: int = 0):
        import oracle
        import trafficgen as tg
        S, self.desc = oracle_sample(W, scale_log2)
        self.p = oracle.params(S["params"])
        self.tabs = tg.hash_tables(S["hash_seed"])
        self.T = tg.Traffic(**S["traffic"])
        self.pipe = oracle.Pipeline(self.p, self.tabs, self.T.routers)
        self.t = 0
        self.seconds = {"advance": 0.0, "scan": 0.0, "merge": 0.0, "regain": 0.0}

    def step(self) -> int:
        """One slot of the oracle's pipeline (oracle.Pipeline.step's order: advance when t > 0,
        scan every router, merge, regain), each step timed on its own."""
        import oracle
        pipe, clock = self.pipe, time.perf_counter
        pairs = self.T.slot(self.t)
        self.t += 1
        t0 = clock()
        pipe.t += 1
        if pipe.t > 0:
            for sk in pipe.routers:
                oracle.advance(pipe.p, sk)
        t1 = clock()
        for sk, pr in zip(pipe.routers, pairs):
            oracle.scan(pipe.p, pipe.tables, sk, pr)
        t2 = clock()
        pipe.global_sk = oracle.merge(pipe.p, pipe.routers)
        t3 = clock()
        oracle.regain(pipe.p, pipe.tables, pipe.global_sk, "pruned")
        t4 = clock()
        for k, dt in zip(("advance", "scan", "merge", "regain"), (t1 - t0, t2 - t1, t3 - t2, t4 - t3)):
            self.seconds[k] += dt
        return sum(len(x) for x in pairs)


def cpu_model() -> str:
    """The host CPU's model as /proc/cpuinfo names it (x86: model name; Arm: implementer and part
    numbers), else the machine type."""
    import platform
    try:
        info = open("/proc/cpuinfo").read()
    except OSError:
        return platform.machine()
    m = re.search(r"^model name\s*:\s*(.+)$", info, re.M)
    if m:
        return m.group(1).strip()
    imp = re.search(r"^CPU implementer\s*:\s*(\S+)", info, re.M)
    part = re.search(r"^CPU part\s*:\s*(\S+)", info, re.M)
    if imp and part:
        return f"{platform.machine()} (CPU implementer {imp.group(1)}, part {part.group(1)})"
    return platform.machine()


def oracle_steps(o: OracleSlots, packets: int, slots: int) -> dict:
    """Each oracle step's share of the timed slots: the scan per packet, the others per slot."""
    sec = o.seconds
    return {"scan_ns_per_packet": round(sec["scan"] / max(packets, 1) * 1e9, 2),
            "advance_ms_per_slot": round(sec["advance"] / max(slots, 1) * 1e3, 2),
            "merge_ms_per_slot": round(sec["merge"] / max(slots, 1) * 1e3, 2),
            "regain_ms_per_slot": round(sec["regain"] / max(slots, 1) * 1e3, 2)}


def cpu_baseline(W: dict, budget_s: float = 12.0, min_slots: int = 3) -> dict:
    """The oracle, as it stands, on the bench's own workload: slots until `budget_s` has passed
    (at least min_slots), the window starting empty; also each step's share: the scan in ns per
    packet, the advance, merge and regain in ms per slot."""
    o = OracleSlots(W)
    pk, slots = 0, 0
    t0 = time.perf_counter()
    while slots < min_slots or time.perf_counter() - t0 < budget_s:
        pk += o.step()
        slots += 1
    dt = time.perf_counter() - t0
    return {"value": round(pk / dt / 1e6, 4), "unit": "Mpps", "cores": 1, "kind": "oracle",
            "sample": f"{slots} slots of {o.desc}", "seconds": round(dt, 2),
            "host_cpus": os.cpu_count(), "cpu_model": cpu_model(),
            "steps": dict(oracle_steps(o, pk, slots), note="the first slot has no advance (the window starts empty)")}


def run_reference(args, world, rank):
    """The oracle, as it stands, as the reference arm (rank 0 only), on the same workload and
    metric as our arm: warm-up slots, then `steps` timed slots of the same traffic, the window
    starting empty (the oracle's cost per slot is its advance, merge and hot-estimator passes over
    the whole RSEA plus the scan, whatever the window holds)."""
    if rank != 0:
        return
    import trafficgen as tg
    W = tg.workload(args.workload)
    W["_name"] = args.workload
    o = OracleSlots(W)
    for _ in range(args.warmup):
        o.step()
    o.seconds = dict.fromkeys(o.seconds, 0.0)
    t0 = time.perf_counter()
    pk = 0
    for _ in range(args.steps):
        pk += o.step()
    dt = time.perf_counter() - t0
    v = pk / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "Mpps", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": {"workload": args.workload, "sample": o.desc},
            "cpu_baseline": {"value": round(v, 4), "unit": "Mpps", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} slots of {o.desc}", "cpu_model": cpu_model(),
                             "steps": oracle_steps(o, pk, args.steps)},
            "e2e": {"value": round(v, 4), "unit": "Mpps", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- our arm

def batched_vs_plain(rank: int, local: int, name: str = "edge16_c3", fill: int = 4, warmup: int = 2,
                     steps: int = 5, tune: bool = True, tune_reps: int = 2) -> dict:
    """The same slots of a many-router workload two ways, with identical lists required.
    plain: one ssd_scan per router, then ssd_merge, ssd_regain and ssd_advance;
    batched: one ssd_scan_batch over all routers, then one ssd_close_slot.
    With tune, the autotuner picks the launch configuration once (on the first context's
    fresh sketches) and both ways run under it."""
    import torch

    import paper_1803_11036_gb300 as ssd
    import trafficgen as tg

    dev = torch.device("cuda", local)
    W = replica_workload(name, rank)
    T = tg.Traffic(**W["traffic"])
    R = T.routers
    n = fill + warmup + steps
    slots = []
    for t in range(n):
        slots.append([torch.from_numpy(v.reshape(-1).view(np.int32)).to(dev) for v in T.slot(t)])
    pk = [sum(x.numel() // 2 for x in s) for s in slots]
    stream = torch.cuda.Stream(dev)
    out = {}
    lists = {}
    chosen, tune_s = None, 0.0
    for mode in ("plain", "batched"):
        ctx = ssd.Context(ssd.make_params(W["params"]), tg.hash_tables(W["hash_seed"]), device=local)
        routers = [ctx.sketch() for _ in range(R)]
        glob = ctx.sketch() if mode == "plain" else None
        if tune and chosen is None:
            t0 = time.perf_counter()
            chosen = ctx.autotune(routers, slots[0], None, reps=tune_reps, stream=stream)
            tune_s = time.perf_counter() - t0
        if chosen is not None:
            ctx.tuning = chosen
        got = []
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = 0
        with torch.cuda.stream(stream):
            for t in range(n):
                if t == fill + warmup:
                    stream.synchronize()
                    l0 = ctx.launch_count
                    a.record(stream)
                if mode == "plain":
                    for sk, x in zip(routers, slots[t]):
                        ctx.scan(sk, x, stream=stream)
                    ctx.merge(routers, glob, stream=stream)
                    lst = ctx.regain(glob, stream=stream)
                    ctx.advance(routers, stream=stream)
                else:
                    ctx.scan_batch(routers, slots[t], stream=stream)
                    lst = ctx.close_slot(routers, None, stream=stream)
                if t >= fill + warmup:
                    got.append(lst)
            b.record(stream)
        stream.synchronize()
        ms = a.elapsed_time(b) / steps
        out[mode] = {"ms_per_slot": round(ms, 3), "launches_per_slot": (ctx.launch_count - l0) / steps}
        lists[mode] = got
        del routers, glob
        ctx.close()
        torch.cuda.empty_cache()
    same = all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
               for x, y in zip(lists["plain"], lists["batched"]))
    timed = sum(pk[fill + warmup:])
    return {"workload": name, "routers": R, "packets_per_slot_mean": int(timed / steps),
            "plain": {**out["plain"], "mpps": round(timed / (out["plain"]["ms_per_slot"] * steps) / 1e3, 1)},
            "batched": {**out["batched"], "mpps": round(timed / (out["batched"]["ms_per_slot"] * steps) / 1e3, 1)},
            "speedup": round(out["plain"]["ms_per_slot"] / out["batched"]["ms_per_slot"], 3),
            "identical_lists": bool(same), "window_filled_slots": fill,
            "tuning": chosen, "tune_s": round(tune_s, 2),
            "note": "plain = per-router scans + merge + regain + advance; batched = one scan launch + fused close"}


def paper_c1_leg(rank: int, local: int, warmup: int = 3, steps: int = 30) -> dict:
    """The paper's own dimensions (Sec. 5: eta = 2^11, q = 14, r = 5, delta = 6, theta = 1024; a
    320 MiB RSEA, 2.5x L2) with one router, 2^18 packets per slot and a window of 4 slots, through
    the bench's step (ssd_slot, default configuration): the window is filled first, then `steps`
    slots are timed with nothing else on the stream; the split into steps comes from a traced
    repeat of the first ten."""
    import torch

    import paper_1803_11036_gb300 as ssd
    import trafficgen as tg

    dev = torch.device("cuda", local)
    W = replica_workload("paper_c1", rank)
    prm = W["params"]
    T = tg.Traffic(**W["traffic"])
    fill = prm["k"]
    n = fill + warmup + steps
    slots = [torch.from_numpy(v.reshape(-1).view(np.int32)).to(dev) for v in T.fill_many([(t, 0) for t in range(n)])]
    pk = [x.numel() // 2 for x in slots]
    ctx = ssd.Context(ssd.make_params(prm), tg.hash_tables(W["hash_seed"]), device=local)
    router = ctx.sketch()
    cap = 1 << 16
    out = (torch.empty(cap, dtype=torch.int32, device=dev), torch.empty(cap, dtype=torch.int32, device=dev),
           torch.zeros(1, dtype=torch.int64, device=dev))
    stream = torch.cuda.Stream(dev)

    def step(t):
        ctx.slot([router], [slots[t]], None, out=out, stream=stream, sync=False)

    with torch.cuda.stream(stream):
        for t in range(fill + warmup):
            step(t)
    stream.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = ctx.launch_count
    with torch.cuda.stream(stream):
        a.record(stream)
        for t in range(fill + warmup, n):
            step(t)
        b.record(stream)
    stream.synchronize()
    launches = (ctx.launch_count - l0) / steps
    st = ctx.stats(stream)
    ms = a.elapsed_time(b) / steps
    timed = sum(pk[fill + warmup:])
    tr = list(range(fill + warmup, fill + warmup + min(10, steps)))
    slot_pass, slot_tail = traced(ctx, stream, [lambda t=t: step(t) for t in tr])
    close_pass, close_tail = traced(ctx, stream, [lambda: ctx.close_slot([router], None, out=out, stream=stream,
                                                                         sync=False)] * len(tr))
    eta, C, r = 1 << prm["log2_eta"], 1 << prm["q"], prm["r"]
    peak, _ = measured_peak()
    scratch = ctx.sketch()
    sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ctx.scan(scratch, slots[fill], stream=stream)
        sa.record(stream)
        for t in tr:
            ctx.scan(scratch, slots[t], stream=stream)
        sb.record(stream)
    stream.synchronize()
    scan_ms = sa.elapsed_time(sb) / len(tr)
    steps_ = step_rooflines(pk=statistics.mean(pk[t] for t in tr), scan_ms=scan_ms,
                            scan_pk=statistics.mean(pk[t] for t in tr), slot_pass=slot_pass, slot_tail=slot_tail,
                            close_pass=close_pass, close_tail=close_tail, rec_bytes=eta * C * r * 2, r=r, peak=peak)
    ctx.close()
    torch.cuda.empty_cache()
    mpps = timed / (ms * steps / 1e3) / 1e6
    return {"workload": "paper_c1", "routers": 1, "packets_per_slot": pk[-1], "k": prm["k"], "eta": eta,
            "q": prm["q"], "r": r, "delta": prm["delta"], "theta": prm["theta"], "window_filled_slots": fill,
            "steps": steps, "ms_per_slot": round(ms, 4), "mpps": round(mpps, 1), "gbps_at_800B": gbps(mpps),
            "launches_per_slot": launches, "list_size": st["n_out"], "hot_per_row": st["hot"],
            "split": steps_,
            "l2": "the 320 MiB RSEA (2.5x L2) is streamed every slot and each slot scans a distinct slice"}


def served_leg(rank: int, local: int, name: str = "served_c5", routers: int = 64, per_router: int = 4,
               rates=(500.0, 2000.0, None), max_inflight: int = 16, tuning: dict | None = None) -> dict:
    """Routers stream slices at Poisson times; each slice is scanned and closed on its router's
    resident RSEA as soon as the device has room (continuous batching, at most max_inflight in
    flight). Latency runs from a slice's arrival to its list on the host. Slices arrive in
    pinned buffers that have crossed the host link once before the clock starts, as the
    reused receive buffers of a deployment would have.

    The same slices run at each offered rate of `rates` (None: every slice ready at once, the
    saturated capacity), each time on freshly admitted routers, and then through the plain form:
    one slice at a time, each call waited for before the next (max_inflight 1), at the first rate
    and saturated. The plain lists must equal the served ones, router by router, slot by slot."""
    import torch

    import paper_1803_11036_gb300 as ssd
    import trafficgen as tg
    from paper_1803_11036_gb300 import serve

    W = replica_workload(name, rank)
    dev = torch.device("cuda", local)
    rng = np.random.default_rng(11 + rank)
    base = []   # (router, seq, pinned pairs, unit-rate arrival)
    for r in range(routers):
        tr = dict(W["traffic"])
        tr["seed"] = tr["seed"] + 101 * r
        T = tg.Traffic(**tr)
        views = T.fill_many([(j, 0) for j in range(per_router)])
        t = 0.0
        for j, v in enumerate(views):
            t += rng.exponential(routers)     # one slice per second overall at rate 1
            base.append((r, j, torch.from_numpy(v.reshape(-1).view(np.int32)).pin_memory(), t))
    warm = torch.empty(max(b[2].numel() for b in base), dtype=torch.int32, device=dev)
    for b in base:
        warm[:b[2].numel()].copy_(b[2], non_blocking=True)
    torch.cuda.synchronize(dev)
    del warm

    def run(rate, inflight):
        slices = [serve.Slice(router=r, pairs=pr, arrival=(t / rate if rate else 0.0), seq=j) for r, j, pr, t in base]
        srv = serve.Server(ssd.make_params(W["params"]), tg.hash_tables(W["hash_seed"]), device=local,
                           max_inflight=inflight, max_slice_pairs=int(W["traffic"]["count_b"]), tuning=tuning)
        for r in range(routers):               # admit every router before the clock starts
            if not srv.try_admit(r):
                break
        admitted = len(srv.tenants)
        res = srv.run([s for s in slices if s.router in srv.tenants], realtime=rate is not None)
        srv.close()
        torch.cuda.empty_cache()
        out = serve.latency_summary(res)
        out.update({"offered_slices_per_s": rate if rate else "all at once", "max_inflight": inflight,
                    "routers": admitted})
        return out, {(x.router, x.slot): (x.ips, x.rk) for x in res}

    served, lists = [], None
    for rate in rates:
        o, l = run(rate, max_inflight)
        served.append(o)
        lists = lists or l
    plain = []
    same = True
    for rate in (rates[0], None):
        o, l = run(rate, 1)
        plain.append(o)
        same = same and set(l) == set(lists) and all(
            np.array_equal(l[k][0], lists[k][0]) and np.array_equal(l[k][1], lists[k][1]) for k in lists)
    sat_served = next(x for x in served if x["offered_slices_per_s"] == "all at once")
    sat_plain = plain[-1]
    first = dict(served[0])
    first.update({"workload": name, "q": W["params"]["q"], "slice_packets": "uniform [10k, 2M]",
                  "reserved_slice_pairs": int(W["traffic"]["count_b"]), "tuning": tuning or "default",
                  "by_offered_rate": served, "plain": plain, "identical_lists_plain_vs_served": bool(same),
                  "capacity_mpps": {"served": sat_served["mpps"], "plain": sat_plain["mpps"],
                                    "speedup": round(sat_served["mpps"] / sat_plain["mpps"], 3)},
                  "note": "plain = the same slices one at a time (each ssd_slot_host call waited for before "
                          "the next); capacity = every slice ready at once"})
    return first


def run_ours(args, world, rank, local):
    import torch

    import paper_1803_11036_gb300 as ssd
    import trafficgen as tg

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    W = replica_workload(args.workload, rank)
    prm = W["params"]
    k = prm["k"]
    fill = k if args.fill < 0 else args.fill
    T = tg.Traffic(**W["traffic"])
    R = T.routers
    nslots = fill + args.warmup + args.steps

    # ---- inputs resident in HBM: every slot's packets, generated in chunks
    slot_dev = []
    chunk = 8
    for s0 in range(0, nslots, chunk):
        jobs = [(t, r) for t in range(s0, min(nslots, s0 + chunk)) for r in range(R)]
        views = T.fill_many(jobs)
        for i in range(0, len(views), R):
            slot_dev.append([torch.from_numpy(v.reshape(-1).view(np.int32)).to(dev) for v in views[i:i + R]])
    pk_per_slot = [sum(x.numel() // 2 for x in s) for s in slot_dev]

    ctx = ssd.Context(ssd.make_params(prm, touch_chunk_bytes=args.touch_chunk_mib << 20),
                      tg.hash_tables(W["hash_seed"]), device=local)
    routers = [ctx.sketch() for _ in range(R)]
    stream = torch.cuda.Stream(dev)
    default_tuning = ctx.tuning
    tune_s = 0.0
    if args.tuning:        # a stated configuration (the autotuner does not run)
        ctx.tuning = json.loads(args.tuning)
        args.no_tune = True
    if not args.no_tune:   # launch configuration picked by measurement on the first slot
        t0 = time.perf_counter()
        ctx.autotune(routers, slot_dev[0], None, reps=3, stream=stream)
        tune_s = time.perf_counter() - t0
    cap = 1 << 16
    ips = torch.empty(cap, dtype=torch.int32, device=dev)
    rks = torch.empty(cap, dtype=torch.int32, device=dev)
    n_out = torch.zeros(1, dtype=torch.int64, device=dev)

    def step(t):
        # the whole slot in one call: scan (touches collected in L2) + merge/hot/advance + regain
        ctx.slot(routers, slot_dev[t], None, out=(ips, rks, n_out), stream=stream, sync=False)

    with torch.cuda.stream(stream):
        for t in range(fill + args.warmup):
            step(t)
    stream.synchronize()
    st_fill = ctx.stats(stream)
    if st_fill["status"]:
        raise RuntimeError(f"capacity status {st_fill['status']} during fill")

    # ---- timed region: K slots, nothing but the slot calls on the stream
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = ctx.launch_count
    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks.start()
    with torch.cuda.stream(stream):
        t_start.record(stream)
        for i in range(args.steps):
            step(fill + args.warmup + i)
        t_end.record(stream)
    stream.synchronize()
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    launches = ctx.launch_count - launches0
    st = ctx.stats(stream)
    if st["status"]:
        raise RuntimeError(f"capacity status {st['status']} in the timed region")

    total_ms = t_start.elapsed_time(t_end)
    timed_pk = sum(pk_per_slot[fill + args.warmup:])
    max_ms = max_over_ranks(total_ms, world)
    all_pk = sum_over_ranks(timed_pk, world)
    value = all_pk / (max_ms / 1e3) / 1e6

    # ---- the split of a slot into its steps, outside the timed region: the first timed slices
    # again, with trace events at the phase boundaries (ssd_set_trace), then the same number of
    # slot closes with no scan (ssd_close_slot: the streaming pass without touch bits)
    n_tr = min(args.steps, 10)
    tr_slots = [fill + args.warmup + i for i in range(n_tr)]
    slot_pass, slot_tail = traced(ctx, stream, [lambda t=t: step(t) for t in tr_slots])
    close_pass, close_tail = traced(ctx, stream, [lambda: ctx.close_slot(routers, None, out=(ips, rks, n_out),
                                                                         stream=stream, sync=False)] * n_tr)
    tr_pk = statistics.mean(pk_per_slot[t] for t in tr_slots)

    # ---- realised column load: each row's mean R_k after the last close, through Eq. 1
    occ = routers[0].occupancy(stream)
    C_cols, eta_ = 1 << prm["q"], 1 << prm["log2_eta"]
    mean_rk = [o / C_cols for o in occ]
    load = [round(-eta_ * math.log(1.0 - m / eta_), 1) for m in mean_rk]
    column_load = {"mean_rk_per_row": [round(m, 2) for m in mean_rk], "eq1_distinct_per_column": load,
                   "theta_over_4": prm["theta"] / 4,
                   "note": "router sketch after the last timed slot's close; a column nearing theta/4 turns "
                           "most estimators hot"}

    # ---- the same slots under the default launch configuration, for the tuner's record
    default_leg = None
    tuned = ctx.tuning
    if not args.no_tune:
        n_def = min(args.steps, 10)
        ctx.tuning = default_tuning
        da, db = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            step(fill + args.warmup)         # warm-up
            da.record(stream)
            for i in range(n_def):
                step(fill + args.warmup + i)
            db.record(stream)
        stream.synchronize()
        ctx.tuning = tuned
        def_ms = da.elapsed_time(db) / n_def
        default_leg = {"ms_per_slot": round(def_ms, 4), "tuned_ms_per_slot": round(total_ms / args.steps, 4),
                       "slots": n_def, "configuration": default_tuning}

    # ---- the scan alone (Algorithm 2 writing the recorders directly), on the timed slices
    scratch = [ctx.sketch() for _ in range(R)]
    sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ctx.scan_batch(scratch, slot_dev[fill], stream=stream)   # warm-up
        sa.record(stream)
        for i in range(args.steps):
            ctx.scan_batch(scratch, slot_dev[fill + args.warmup + i], stream=stream)
        sb.record(stream)
    stream.synchronize()
    scan_ms = sa.elapsed_time(sb) / args.steps
    scan_mpps = timed_pk / (scan_ms * args.steps / 1e3) / 1e6
    del scratch

    # ---- the same slots replayed from one captured CUDA graph (fixed-size slots only)
    graph_leg = None
    counts = [x.numel() // 2 for x in slot_dev[0]]
    if not args.no_graph and all([x.numel() // 2 for x in s] == counts for s in slot_dev):
        g = ssd.SlotGraph(ctx, routers, counts, None, cap=cap)
        ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for dst, src in zip(g.inputs, slot_dev[fill]):
                dst.copy_(src)
            g.replay()                       # warm-up
            ga.record(stream)
            for i in range(args.steps):
                for dst, src in zip(g.inputs, slot_dev[fill + args.warmup + i]):
                    dst.copy_(src)
                g.replay()
            gb.record(stream)
        stream.synchronize()
        graph_ms = ga.elapsed_time(gb) / args.steps
        graph_leg = {"replay_ms_per_slot": round(graph_ms, 4), "direct_ms_per_slot": round(total_ms / args.steps, 4),
                     "mpps": round(timed_pk / (graph_ms * args.steps / 1e3) / 1e6, 1),
                     "note": "one captured ssd_slot replayed per slot; the time includes copying the slot's "
                             "pairs into the graph's input buffers"}
        del g

    eta, C, r = 1 << prm["log2_eta"], 1 << prm["q"], prm["r"]
    recorders = eta * C * r
    rec_bytes = recorders * 2 * R               # each router's recorders read once (stamps: no advance writes)
    # the pass runs as chunk launches of `chunk` estimators (the tuned touch bits per chunk)
    n_se = r * C
    chunk = 1
    while chunk * 2 * (eta // 8) * R <= tuned["touch_chunk_bytes"] and chunk * 2 <= 1 << (n_se - 1).bit_length():
        chunk *= 2
    n_chunks = -(-n_se // chunk)
    peak, peak_kind = measured_peak()
    traffic = profiled_traffic(args.workload, chunk, collect=tuned["collect_touches"])
    steps = step_rooflines(pk=tr_pk, scan_ms=scan_ms, scan_pk=timed_pk / args.steps, slot_pass=slot_pass,
                           slot_tail=slot_tail, close_pass=close_pass, close_tail=close_tail,
                           rec_bytes=rec_bytes, r=r, peak=peak)
    achieved = steps["slot_pass"]["achieved_gbs"]

    # ---- end to end through the C ABI from pinned host memory: ssd_slot_host copies each
    # slot's pairs to the device (overlapping the previous slot) and the list of every slot
    # (count + first entries) comes back to pinned host memory; the host reads slot t's list
    # after enqueueing slot t+1.
    e2e = None
    if not args.no_e2e:
        host = [[torch.from_numpy(x.cpu().numpy()).pin_memory() for x in s]
                for s in slot_dev[fill + args.warmup - 1:]]
        head = 1024
        outs = [(torch.empty(cap, dtype=torch.int32, device=dev), torch.empty(cap, dtype=torch.int32, device=dev),
                 torch.zeros(1, dtype=torch.int64, device=dev)) for _ in range(2)]
        hbuf = [(torch.empty(head, dtype=torch.int32).pin_memory(), torch.empty(head, dtype=torch.int32).pin_memory(),
                 torch.zeros(1, dtype=torch.int64).pin_memory()) for _ in range(2)]
        # every pinned buffer crosses the host link once before the clock starts: a DMA through
        # freshly pinned pages can run an order of magnitude slower than through pages already
        # mapped, and a deployment reuses its pinned buffers
        warm = [torch.empty(x.numel(), dtype=x.dtype, device=dev) for x in host[0]]
        with torch.cuda.stream(stream):
            for hs in host:
                for dst, src in zip(warm, hs):
                    dst.copy_(src, non_blocking=True)
        stream.synchronize()
        del warm
        done = [torch.cuda.Event(enable_timing=True) for _ in range(len(host))]
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d2h = 0
        with torch.cuda.stream(stream):
            for j in range(len(host) + 1):      # j = 0 is an untimed warm-up of the host path
                if j < len(host):
                    if j == 1:
                        ea.record(stream)
                    o, hb = outs[j & 1], hbuf[j & 1]
                    ctx.slot_host(routers, host[j], None, out=o, stream=stream, sync=False)
                    hb[2].copy_(o[2], non_blocking=True)
                    hb[0].copy_(o[0][:head], non_blocking=True)
                    hb[1].copy_(o[1][:head], non_blocking=True)
                    done[j].record(stream)
                if j >= 1:
                    done[j - 1].synchronize()
                    hb = hbuf[(j - 1) & 1]
                    m = int(hb[2].item())
                    if m > head:
                        raise RuntimeError("list longer than the read-back head")
                    _ = (hb[0][:m].numpy().copy(), hb[1][:m].numpy().copy())
                    if j - 1 >= 1:
                        d2h += 8 + 2 * 4 * head
            eb.record(stream)
        stream.synchronize()
        # device time between consecutive slot completions (the slot's own pace on the GPU)
        gaps = [done[j - 1].elapsed_time(done[j]) for j in range(2, len(host))]
        # the host link alone: every timed slot's pinned pairs, host -> device, once each
        probe = [torch.empty(x.numel(), dtype=x.dtype, device=dev) for x in host[0]]
        per = []
        with torch.cuda.stream(stream):
            for hs in host[1:]:
                ha, hb_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ha.record(stream)
                for dst, src in zip(probe, hs):
                    dst.copy_(src, non_blocking=True)
                hb_.record(stream)
                per.append((ha, hb_, sum(x.numel() * 4 for x in hs)))
        stream.synchronize()
        rates = [b / (a.elapsed_time(c) / 1e3) / 1e9 for a, c, b in per]
        h2d_gbs = statistics.median(rates)
        del probe
        e2e_ms = max_over_ranks(ea.elapsed_time(eb), world)
        e2e = {"value": round(all_pk / (e2e_ms / 1e3) / 1e6, 2), "unit": "Mpps",
               "h2d_bytes_per_step": int(8 * timed_pk / args.steps),
               "d2h_bytes_per_step": int(d2h / args.steps),
               "path": "ssd_slot_host from pinned buffers, list read back every slot",
               "host_to_device_gbs": round(h2d_gbs, 1), "host_to_device_gbs_min": round(min(rates), 1),
               "slot_completion_ms": {"median": round(statistics.median(gaps), 4), "max": round(max(gaps), 4)}}
        del host

    del slot_dev, routers
    ctx.close()
    torch.cuda.empty_cache()
    c1 = None if args.no_c1 else paper_c1_leg(rank, local)
    bvp = None if args.no_batched else batched_vs_plain(rank, local)
    # 32 routers, 15.6 M packets per slot with ten hot sources (33 RSEAs of 5 GiB); the 300-slot
    # window is not filled, so the regain tail is short and the scan and streaming pass dominate
    stress = None if args.no_stress else batched_vs_plain(rank, local, "stress32_c4", fill=2, warmup=1, steps=3,
                                                                tune_reps=1)
    served = None if args.no_served else served_leg(rank, local)

    if rank != 0:
        return
    cpu = None if args.no_cpu else cpu_baseline(W)
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "Mpps", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(max_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
        "config": {"workload": args.workload, "routers": R, "packets_per_slot": int(pk_per_slot[-1]),
                   "k": k, "eta": eta, "q": prm["q"], "r": r, "delta": prm["delta"], "theta": prm["theta"],
                   "window_filled_slots": fill, "l2": "inputs larger than L2: the 5 GiB RSEA is streamed every "
                   "step and each step scans a distinct slice",
                   "tuning": tuned, "tuned_by": ("--tuning" if args.tuning else "default") if args.no_tune
                   else "ssd_autotune on the first slot",
                   "tune_s": round(tune_s, 2)},
        "default_configuration": default_leg,
        "gbps_at_800B": gbps(value),
        "scan": {"mpps": round(scan_mpps, 2), "gbps_at_800B": gbps(scan_mpps), "ms_per_slice": round(scan_ms, 4),
                 "note": "ssd_scan alone (recorders written directly; steps.scan_standalone has its roofline); in "
                         "the timed slot the scan's touches go to L2 bits applied by the streaming pass "
                         "(steps.scan_in_slot)"},
        "slot_ms": {"streaming_pass_with_scan": steps["slot_pass"]["ms_per_slice"],
                    "candidates_and_list": steps["regain_tail"]["ms_per_slice"],
                    "total": round(max_ms / args.steps, 4)},
        "reconstruct_ms_per_slice": steps["regain_tail"]["ms_per_slice"],
        "steps": steps,
        "paper_c1": c1,
        "cuda_graph": graph_leg,
        "batched_vs_plain": bvp,
        "batched_vs_plain_stress": stress,
        "served": served,
        "roofline": {"kernel": "the streaming pass of ssd_slot: k_lists (every pair hashed once, touch lists "
                               "per chunk) and the k_chunk launches (the scan's touches applied, hot extraction, "
                               "advance; the next chunk's touches set in L2 between estimators)",
                     "launches_per_pass": n_chunks + 1,
                     "algorithmic_bytes_per_chunk_launch": chunk * eta * 2 * R,
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": steps["slot_pass"]["frac"], "peak_source": peak_kind,
                     "algorithmic_bytes_per_pass": steps["slot_pass"]["algorithmic_bytes"],
                     "traffic": traffic,
                     "traffic_source": None if traffic is None else
                     f"profiles/chunk_pass_{args.workload}.md (ncu DRAM bytes of one chunk launch)"},
        "hot_per_row": st["hot"], "candidates_per_level": st["level"], "list_size": st["n_out"],
        "column_load": column_load,
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    dist_init(world, local)
    try:
        run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
