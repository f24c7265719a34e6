"""The debug build of the library (SSD_DEBUG=1: the kernels check their indices against their
bounds and report a broken one as SSD_STATUS_INTERNAL instead of faulting; guard words around the
candidate tuple buffers are compared when the counters are read) on the small parity cases, every
route: the one-router ssd_slot with touch lists and with pre-hashed pairs, several routers with
the side-stream collection, ssd_scan + ssd_close_slot, the separate calls and the allocation-free
regain. Every list equals the oracle's and no bound is broken. A process loads one build of the
library, so the cases run in a child process."""
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _child() -> None:
    import torch

    import paper_1803_11036_gb300 as ssd
    import trafficgen as tg
    from gpu_harness import Run, assert_list_equal, to_dev
    from paper_1803_11036_gb300 import _abi

    L = _abi.load()
    assert L.ssd_build_flags() == 1, "not the debug build"
    cases = 0

    def clean(run):
        st = run.ctx.stats()
        assert st["status"] == 0, st

    for name, kw, tuning, how in [
            ("tiny", {}, None, "fused"),
            ("tiny", {}, None, "unfused"),
            ("paper_c1", dict(touch_chunk_bytes=2 << 20), None, "slot"),
            ("paper_c1", dict(touch_chunk_bytes=2 << 20), dict(collect_touches=1), "slot"),
            ("paper_c1", {}, None, "unfused"),
            ("edge_small", dict(touch_chunk_bytes=4 << 20), None, "slot"),
            ("stress_small", {}, dict(combine_touches=1), "fused")]:
        run = Run(name, **kw)
        if tuning:
            run.ctx.tuning = tuning
        step = {"fused": lambda: run.step_fused("pruned"), "unfused": lambda: run.step_unfused("pruned"),
                "slot": lambda: run.step_slot("pruned")}[how]
        for _ in range(min(run.W["slots"], 6)):
            got, want = step()
            assert_list_equal(got, want, f"{name} {how} slot {run.t}")
            clean(run)
            cases += 1
        if how == "unfused" and name == "paper_c1":   # the allocation-free regain on the last merge
            import ctypes
            tabs = torch.from_numpy(tg.hash_tables(run.W["hash_seed"]).view(np.int32)).cuda()
            rec = torch.from_numpy(run.glob.export().view(np.int16)).cuda()
            ips = torch.empty(1 << 16, dtype=torch.int32, device="cuda")
            rk = torch.empty(1 << 16, dtype=torch.int32, device="cuda")
            n = ctypes.c_uint64()
            prm = ssd.make_params(run.W["params"])
            _abi.check(L.ssd_regain_static(ctypes.byref(prm), 0, 0, 0, ctypes.c_void_p(tabs.data_ptr()),
                                           ctypes.c_void_p(rec.data_ptr()), ctypes.c_void_p(ips.data_ptr()),
                                           ctypes.c_void_p(rk.data_ptr()), 1 << 16, ctypes.byref(n),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
                       "ssd_regain_static")
            want_ips, _ = run.ctx.regain(run.glob)
            assert np.array_equal(ips[:n.value].cpu().numpy().view(np.uint32), want_ips)
        run.close()
    print(f"debug build: {cases} slots, every list equal to the oracle's, no bound broken")


@pytest.mark.gpu
def test_debug_build_keeps_every_bound():
    env = dict(os.environ, SSD_DEBUG="1")
    code = f"import sys; sys.path[:0] = [{ROOT!r}, {HERE!r}]; import test_gpu_debug_build as t; t._child()"
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1200,
                         cwd=ROOT)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    assert "no bound broken" in out.stdout
