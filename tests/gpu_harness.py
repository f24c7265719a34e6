"""Helpers for the GPU parity tests: one seeded workload through the oracle and
through the CUDA library, slot by slot."""
from __future__ import annotations

import numpy as np

import oracle
import paper_1803_11036_gb300 as ssd
import trafficgen as tg


def to_dev(pairs: np.ndarray):
    import torch
    a = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1)
    return torch.from_numpy(a.view(np.int32)).to("cuda:0")


def oracle_flags(flags: int) -> int:
    """The oracle's flags for a library flag set (the method-changing ones)."""
    return ((flags & ssd.SSD_VERIFY_H0) and oracle.VERIFY_H0) | ((flags & ssd.SSD_RHFG_LITERAL) and oracle.RHFG_LITERAL)


def setup(W: dict, flags: int = 0, **caps):
    p_or = oracle.params(W["params"], oracle_flags(flags))
    tabs = tg.hash_tables(W["hash_seed"])
    ctx = ssd.Context(ssd.make_params(W["params"], flags, **caps), tabs)
    return p_or, tabs, ctx


def oracle_regain(p, tabs, sk, method="levelwise"):
    return oracle.regain(p, tabs, sk, method)


def assert_list_equal(got, want, where=""):
    gi, gr = got
    assert np.array_equal(gi, want["ips"]), f"{where}: hosts differ: {len(gi)} vs {len(want['ips'])}"
    assert np.array_equal(gr, want["rk"]), f"{where}: R_k differs"


class Run:
    """Drives n routers of one workload through both sides with the unfused calls
    (advance, scan, merge, regain) or the fused slot close."""

    def __init__(self, name_or_W, flags: int = 0, **caps):
        self.W = tg.workload(name_or_W) if isinstance(name_or_W, str) else name_or_W
        self.p, self.tabs, self.ctx = setup(self.W, flags, **caps)
        self.T = tg.Traffic(**self.W["traffic"])
        self.n = self.T.routers
        self.pipe = oracle.Pipeline(self.p, self.tabs, self.n)
        self.routers = [self.ctx.sketch() for _ in range(self.n)]
        self.glob = self.ctx.sketch()
        self.t = -1

    def slot_pairs(self, t):
        return self.T.slot(t)

    def step_unfused(self, regain_method="levelwise", batch=True):
        """Oracle and GPU through one slot with separate calls; returns (gpu list, oracle result)."""
        self.t += 1
        pairs = self.slot_pairs(self.t)
        want = self.pipe.step(pairs, regain_method)
        if self.t > 0:
            self.ctx.advance(self.routers)
        devs = [to_dev(pr) for pr in pairs]
        if batch:
            self.ctx.scan_batch(self.routers, devs)
        else:
            for sk, d in zip(self.routers, devs):
                self.ctx.scan(sk, d)
        self.ctx.merge(self.routers, self.glob)
        got = self.ctx.regain(self.glob) if regain_method else None
        return got, want

    def step_fused(self, regain_method="levelwise", with_global=True):
        """Oracle: advance, scan, merge, regain. GPU: scan, then close_slot (merge, regain, advance)."""
        self.t += 1
        pairs = self.slot_pairs(self.t)
        want = self.pipe.step(pairs, regain_method)
        devs = [to_dev(pr) for pr in pairs]
        self.ctx.scan_batch(self.routers, devs)
        got = self.ctx.close_slot(self.routers, self.glob if with_global else None)
        return got, want

    def step_slot(self, regain_method="levelwise", with_global=True):
        """Oracle as in step_fused; GPU: one ssd_slot call (scan + close with touches in L2)."""
        self.t += 1
        pairs = self.slot_pairs(self.t)
        want = self.pipe.step(pairs, regain_method)
        devs = [to_dev(pr) for pr in pairs]
        got = self.ctx.slot(self.routers, devs, self.glob if with_global else None)
        return got, want

    def close(self):
        self.ctx.close()
