"""Python face of the CPU oracle (``ssd_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers. The product path (the CUDA
library and its binding) never imports this package.

The C core is compiled with gcc into ``oracle/_build/`` on first use (or by
``__graft_entry__.build()``). Arrays are numpy; a sketch (RSEA) is a flat
``uint16`` array laid out ``[row][col][recorder]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "ssd_oracle.c")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

VERIFY_H0 = 1
MAX_MERGE = 2
RHFG_LITERAL = 4   # Eq. 2 as printed: windows at i*delta (R2 takes (i-1)*delta)
MAX_R = 16


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("log2_eta", "q", "r", "delta", "k", "theta", "flags")]

    @property
    def eta(self) -> int:
        return 1 << self.log2_eta

    @property
    def C(self) -> int:
        return 1 << self.q

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


def params(d: dict, flags: int = 0) -> Params:
    return Params(d["log2_eta"], d["q"], d["r"], d["delta"], d["k"], d["theta"], d.get("flags", 0) | flags)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER(Params)
            u32, u64, i64, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p
            sig = {
                "orc_check_params": ([P], ctypes.c_int),
                "orc_threshold": ([u32, u32, vp, vp], ctypes.c_int),
                "orc_estimate": ([u32, u32], ctypes.c_double),
                "orc_h1": ([P, vp, u32], u32),
                "orc_rhfg": ([P, vp, u32, vp], None),
                "orc_extract": ([P, vp, vp], ctypes.c_int),
                "orc_sketch_len": ([P], u64),
                "orc_sketch_init": ([P, vp], None),
                "orc_scan": ([P, vp, vp, vp, u64], None),
                "orc_advance": ([P, vp], None),
                "orc_merge": ([P, vp, ctypes.c_int, vp], None),
                "orc_rk_row": ([P, vp, u32, vp], None),
                "orc_hse": ([P, vp, u32, vp], u32),
                "orc_regain_recursive": ([P, vp, vp, vp, vp, u64, vp], i64),
                "orc_regain_levelwise": ([P, vp, vp, vp, vp, u64, vp, vp], i64),
                "orc_regain_pruned": ([P, vp, vp, vp, vp, u64, vp, vp], i64),
                "orc_sampled_new": ([P, vp, vp, u32], vp),
                "orc_sampled_free": ([vp], None),
                "orc_sampled_scan": ([vp, vp, vp, u64], None),
                "orc_sampled_advance": ([vp], None),
                "orc_sampled_get": ([vp, u32, u32, vp], ctypes.c_int),
                "orc_exact_new": ([u32, u32], vp),
                "orc_exact_free": ([vp], None),
                "orc_exact_add_slot": ([vp, vp, u64], None),
                "orc_exact_report": ([vp, vp, vp, u64], i64),
                "orc_exact_degree": ([vp, u32], u32),
                "orc_roundtrip_failures": ([P, vp, vp, u64], u64),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def check_params(p: Params) -> bool:
    return _load().orc_check_params(ctypes.byref(p)) == 0


def threshold(eta: int, theta: int):
    """(ceil(R^_k), R^_k) with R^_k = eta*(1-exp(-theta/eta)); raises if the rounding is ambiguous."""
    thr = ctypes.c_uint32()
    rhat = ctypes.c_double()
    rc = _load().orc_threshold(eta, theta, ctypes.byref(thr), ctypes.byref(rhat))
    if rc:
        raise ValueError(f"R^_k={rhat.value!r} is within 1e-9 of an integer")
    return thr.value, rhat.value


def estimate(eta: int, rk: int) -> float:
    return _load().orc_estimate(eta, rk)


def h1(p: Params, tables: np.ndarray, oip: int) -> int:
    t = _u32(tables)
    return int(_load().orc_h1(ctypes.byref(p), t.ctypes.data, oip))


def rhfg(p: Params, tables: np.ndarray, cip: int) -> np.ndarray:
    t = _u32(tables)
    cols = np.zeros(MAX_R, dtype=np.uint32)
    _load().orc_rhfg(ctypes.byref(p), t.ctypes.data, cip, cols.ctypes.data)
    return cols[: p.r].copy()


def extract(p: Params, tuple_cols) -> int | None:
    tup = np.zeros(MAX_R, dtype=np.uint32)
    tup[: p.r] = tuple_cols
    out = ctypes.c_uint32()
    rc = _load().orc_extract(ctypes.byref(p), tup.ctypes.data, ctypes.byref(out))
    return None if rc else int(out.value)


def roundtrip_failures(p: Params, tables: np.ndarray, xs) -> int:
    """How many x do not come back from regaining their own tuple RHFG(x)."""
    t = _u32(tables)
    x = _u32(xs)
    return int(_load().orc_roundtrip_failures(ctypes.byref(p), t.ctypes.data, x.ctypes.data, x.size))


def new_sketch(p: Params) -> np.ndarray:
    n = int(_load().orc_sketch_len(ctypes.byref(p)))
    sk = np.empty(n, dtype=np.uint16)
    _load().orc_sketch_init(ctypes.byref(p), sk.ctypes.data)
    return sk


def scan(p: Params, tables: np.ndarray, sk: np.ndarray, pairs: np.ndarray) -> None:
    t = _u32(tables)
    pr = _u32(pairs).reshape(-1)
    assert sk.dtype == np.uint16 and sk.flags.c_contiguous
    _load().orc_scan(ctypes.byref(p), t.ctypes.data, sk.ctypes.data, pr.ctypes.data, pr.size // 2)


def advance(p: Params, sk: np.ndarray) -> None:
    _load().orc_advance(ctypes.byref(p), sk.ctypes.data)


def merge(p: Params, routers) -> np.ndarray:
    out = np.empty_like(routers[0])
    ptrs = (ctypes.c_void_p * len(routers))(*[r.ctypes.data for r in routers])
    _load().orc_merge(ctypes.byref(p), ptrs, len(routers), out.ctypes.data)
    return out


def rk_row(p: Params, sk: np.ndarray, row: int) -> np.ndarray:
    out = np.empty(p.C, dtype=np.uint32)
    _load().orc_rk_row(ctypes.byref(p), sk.ctypes.data, row, out.ctypes.data)
    return out


def hse(p: Params, sk: np.ndarray, row: int) -> np.ndarray:
    out = np.empty(p.C, dtype=np.uint32)
    n = _load().orc_hse(ctypes.byref(p), sk.ctypes.data, row, out.ctypes.data)
    return out[:n].copy()


def regain(p: Params, tables: np.ndarray, sk: np.ndarray, method: str = "levelwise", cap: int = 1 << 20):
    """Sliding super point list from a (global) sketch.

    Returns dict(ips, rk, levels, raw): ascending unique hosts, their R_k, the
    candidate count after each row (levels[0] = |HSE(0)|, levels[1] = pairs,
    levels[i] = tuples over rows 0..i), and the accepted tuples before dedupe
    (raw; None for the recursive form)."""
    L = _load()
    t = _u32(tables)
    ips = np.empty(cap, dtype=np.uint32)
    rks = np.empty(cap, dtype=np.uint32)
    levels = np.zeros(MAX_R, dtype=np.uint64)
    raw = ctypes.c_uint64(0)
    if method == "recursive":
        n = L.orc_regain_recursive(ctypes.byref(p), t.ctypes.data, sk.ctypes.data, ips.ctypes.data,
                                   rks.ctypes.data, cap, levels.ctypes.data)
        rawv = None
    else:
        f = L.orc_regain_levelwise if method == "levelwise" else L.orc_regain_pruned
        n = f(ctypes.byref(p), t.ctypes.data, sk.ctypes.data, ips.ctypes.data, rks.ctypes.data, cap,
              levels.ctypes.data, ctypes.byref(raw))
        rawv = int(raw.value)
    if n < 0:
        raise RuntimeError(f"oracle regain failed ({n})")
    if n > cap:
        raise RuntimeError(f"oracle list has {n} hosts > cap {cap}")
    return dict(ips=ips[:n].copy(), rk=rks[:n].copy(), levels=levels[: p.r].copy(), raw=rawv)


def view_pairs(pairs: np.ndarray, side: int = 0, group_bits: int = 0, group: int = 0) -> np.ndarray:
    """The (host, opposite host) pairs one sketch view counts. Sec. 3.1 defines the detector for
    the hosts of CNet, the first field of each pair, and obtains ONet's by exchanging the roles of
    the two networks (side 1 swaps the fields). Sec. 6 scales to bigger networks with several RSEAs,
    each regaining one group of hosts split by their IP addresses: a group keeps the pairs whose
    host has `group` as its top group_bits bits."""
    a = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
    if side:
        a = a[:, ::-1]
    if group_bits:
        a = a[(a[:, 0] >> np.uint32(32 - group_bits)) == np.uint32(group)]
    return np.ascontiguousarray(a)


def in_group(ips: np.ndarray, group_bits: int, group: int) -> np.ndarray:
    """Mask of the hosts of one IP group (Sec. 6): the regain of a group's RSEA lists only these."""
    ips = np.asarray(ips, dtype=np.uint32)
    if not group_bits:
        return np.ones(ips.shape, dtype=bool)
    return (ips >> np.uint32(32 - group_bits)) == np.uint32(group)


class Sampled:
    """Algorithm 2 and the recorder update restricted to chosen estimators (row, col)."""

    def __init__(self, p: Params, rows, cols):
        self.p = p
        self.L = _load()
        r = _u32(rows)
        c = _u32(cols)
        self._h = self.L.orc_sampled_new(ctypes.byref(p), r.ctypes.data, c.ctypes.data, r.size)
        if not self._h:
            raise MemoryError

    def scan(self, tables, pairs) -> None:
        t = _u32(tables)
        pr = _u32(pairs).reshape(-1)
        self.L.orc_sampled_scan(self._h, t.ctypes.data, pr.ctypes.data, pr.size // 2)

    def advance(self) -> None:
        self.L.orc_sampled_advance(self._h)

    def get(self, row: int, col: int) -> np.ndarray:
        out = np.empty(self.p.eta, dtype=np.uint16)
        if self.L.orc_sampled_get(self._h, row, col, out.ctypes.data):
            raise KeyError((row, col))
        return out

    def close(self) -> None:
        if self._h:
            self.L.orc_sampled_free(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class Exact:
    """Precise algorithm: exact |OP(cip, SW)| per sliding window."""

    def __init__(self, k: int, theta: int):
        self.L = _load()
        self._h = self.L.orc_exact_new(k, theta)

    def add_slot(self, pairs) -> None:
        pr = _u32(pairs).reshape(-1)
        self.L.orc_exact_add_slot(self._h, pr.ctypes.data, pr.size // 2)

    def report(self, cap: int = 1 << 22):
        ips = np.empty(cap, dtype=np.uint32)
        deg = np.empty(cap, dtype=np.uint32)
        n = self.L.orc_exact_report(self._h, ips.ctypes.data, deg.ctypes.data, cap)
        if n > cap:
            raise RuntimeError("exact report overflow")
        return ips[:n].copy(), deg[:n].copy()

    def degree(self, cip: int) -> int:
        return int(self.L.orc_exact_degree(self._h, cip))

    def close(self) -> None:
        if self._h:
            self.L.orc_exact_free(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class Pipeline:
    """The per-slot order on n routers (Sec. 4): at slot t, every router's
    recorders advance (t > 0), each router scans its pairs (Algorithm 2), the
    routers merge into the global RSEA (Algorithm 5), and the global RSEA is
    regained."""

    def __init__(self, p: Params, tables: np.ndarray, routers: int):
        self.p = p
        self.tables = _u32(tables)
        self.routers = [new_sketch(p) for _ in range(routers)]
        self.t = -1
        self.global_sk = None

    def step(self, slot_pairs, regain_method: str | None = "levelwise"):
        self.t += 1
        if self.t > 0:
            for sk in self.routers:
                advance(self.p, sk)
        for sk, pr in zip(self.routers, slot_pairs):
            scan(self.p, self.tables, sk, pr)
        self.global_sk = merge(self.p, self.routers)
        if regain_method is None:
            return None
        return regain(self.p, self.tables, self.global_sk, regain_method)
