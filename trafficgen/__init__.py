"""Seeded synthetic traffic and hash-table draws (inputs only).

Both the CUDA library and the CPU oracle consume what this module produces;
it holds none of the detector's arithmetic. The C core (``trafficgen.c``) is
compiled on first use with gcc into ``trafficgen/_build/``.

A packet is a pair ``(cip, oip)`` of host-order IPv4 values (Sec. 3.1 of the
paper); a router-slot's packets are returned as a ``uint32`` array of shape
``(n, 2)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .workloads import WORKLOADS, workload  # noqa: F401  (re-export)

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libtrafficgen.so")
_SRC = os.path.join(_HERE, "trafficgen.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator's C core; returns the path of the shared object."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Config(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64), ("routers", ctypes.c_uint32), ("n_src", ctypes.c_uint32),
        ("zipf_s", ctypes.c_double), ("deg_cap", ctypes.c_uint32), ("rho", ctypes.c_double),
        ("n_planted", ctypes.c_uint32), ("planted_lo", ctypes.c_uint32), ("planted_hi", ctypes.c_uint32),
        ("k", ctypes.c_uint32), ("planted_mode", ctypes.c_uint32), ("n_hot", ctypes.c_uint32),
        ("hot_frac", ctypes.c_double), ("hot_peers", ctypes.c_uint32), ("shared_frac", ctypes.c_double),
        ("count_mode", ctypes.c_uint32), ("count_a", ctypes.c_uint64), ("count_b", ctypes.c_uint64),
        ("ln_mu", ctypes.c_double), ("ln_sigma", ctypes.c_double),
    ]


_COUNT_MODES = {"fixed": 0, "lognormal": 1, "uniform": 2, "split": 3}


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32, u64, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
            lib.tg_hash_tables.argtypes = [u64, vp]
            lib.tg_hash_tables.restype = None
            lib.tg_setup.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(vp)]
            lib.tg_setup.restype = ctypes.c_int
            lib.tg_free.argtypes = [vp]
            lib.tg_free.restype = None
            for name in ("tg_src_ip", "tg_planted_ip", "tg_hot_ip", "tg_planted_degree", "tg_src_degree"):
                getattr(lib, name).argtypes = [vp, u32]
                getattr(lib, name).restype = u32
            lib.tg_planted_active.argtypes = [vp, u32, u32]
            lib.tg_planted_active.restype = ctypes.c_int
            lib.tg_count.argtypes = [vp, u32, u32]
            lib.tg_count.restype = u64
            lib.tg_fill.argtypes = [vp, u32, u32, vp, u64]
            lib.tg_fill.restype = ctypes.c_int
            lib.tg_fill_batch.argtypes = [vp, vp, vp, vp, vp, u64, ctypes.c_int]
            lib.tg_fill_batch.restype = ctypes.c_int
            _lib = lib
    return _lib


def hash_tables(seed: int) -> np.ndarray:
    """2048 uint32 words from splitmix64(seed): table set 1 (4 x 256) then table set 2 (4 x 256)."""
    out = np.empty(2048, dtype=np.uint32)
    _load().tg_hash_tables(ctypes.c_uint64(seed & (2**64 - 1)), out.ctypes.data)
    return out


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


class Traffic:
    """A seeded stream of router-slots; every packet is a pure function of the recipe and seed."""

    def __init__(self, seed: int, routers: int = 1, n_src: int = 0, zipf_s: float = 1.2,
                 deg_cap: int = 512, rho: float = 0.3, n_planted: int = 0,
                 planted_lo: int = 0, planted_hi: int = 0, k: int = 1, planted_mode: int = 0,
                 n_hot: int = 0, hot_frac: float = 0.0, hot_peers: int = 1, shared_frac: float = 0.0,
                 count: str = "fixed", count_a: int = 0, count_b: int = 0,
                 ln_mu: float = 0.0, ln_sigma: float = 0.0):
        self.lib = _load()
        c = _Config(seed=seed, routers=routers, n_src=n_src, zipf_s=zipf_s, deg_cap=deg_cap, rho=rho,
                     n_planted=n_planted, planted_lo=planted_lo, planted_hi=planted_hi, k=k,
                     planted_mode=planted_mode, n_hot=n_hot, hot_frac=hot_frac, hot_peers=hot_peers,
                     shared_frac=shared_frac, count_mode=_COUNT_MODES[count], count_a=count_a,
                     count_b=count_b, ln_mu=ln_mu, ln_sigma=ln_sigma)
        self.cfg = c
        self.routers = routers
        self.n_planted = n_planted
        self.n_hot = n_hot
        h = ctypes.c_void_p()
        rc = self.lib.tg_setup(ctypes.byref(c), ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"traffic recipe rejected (code {rc})")
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None):
            self.lib.tg_free(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover - finaliser
        try:
            self.close()
        except Exception:
            pass

    def count(self, t: int, router: int = 0) -> int:
        return int(self.lib.tg_count(self._h, t, router))

    def fill(self, t: int, router: int = 0, n: int | None = None) -> np.ndarray:
        n = self.count(t, router) if n is None else n
        out = np.empty((n, 2), dtype=np.uint32)
        if n:
            rc = self.lib.tg_fill(self._h, t, router, out.ctypes.data, n)
            if rc:
                raise RuntimeError(f"tg_fill failed ({rc})")
        return out

    def fill_many(self, jobs, out: np.ndarray | None = None):
        """jobs: list of (slot, router). Returns a list of (n,2) arrays (views into one buffer)."""
        jobs = list(jobs)
        counts = np.array([self.count(t, r) for t, r in jobs], dtype=np.uint64)
        total = int(counts.sum())
        if out is None:
            out = np.empty((total, 2), dtype=np.uint32)
        offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        views = [out[offs[i]:offs[i + 1]] for i in range(len(jobs))]
        if jobs:
            slots = np.array([t for t, _ in jobs], dtype=np.uint32)
            routers = np.array([r for _, r in jobs], dtype=np.uint32)
            ptrs = (ctypes.c_void_p * len(jobs))(*[v.ctypes.data for v in views])
            rc = self.lib.tg_fill_batch(self._h, slots.ctypes.data, routers.ctypes.data,
                                        counts.ctypes.data, ptrs, len(jobs), _threads())
            if rc:
                raise RuntimeError(f"tg_fill_batch failed ({rc})")
        return views

    def slot(self, t: int):
        """All routers' packets of slot t (list indexed by router)."""
        return self.fill_many([(t, r) for r in range(self.routers)])

    def planted_ips(self) -> np.ndarray:
        return np.array([self.lib.tg_planted_ip(self._h, p) for p in range(self.n_planted)], dtype=np.uint32)

    def planted_degrees(self) -> np.ndarray:
        return np.array([self.lib.tg_planted_degree(self._h, p) for p in range(self.n_planted)],
                        dtype=np.uint32)

    def planted_active(self, p: int, t: int) -> bool:
        return bool(self.lib.tg_planted_active(self._h, p, t))

    def hot_ips(self) -> np.ndarray:
        return np.array([self.lib.tg_hot_ip(self._h, h) for h in range(self.n_hot)], dtype=np.uint32)


def traffic_for(name_or_spec) -> Traffic:
    spec = workload(name_or_spec) if isinstance(name_or_spec, str) else name_or_spec
    return Traffic(**spec["traffic"])
