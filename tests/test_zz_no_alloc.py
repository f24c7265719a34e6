"""The allocation-free regain (ssd_regain_static) against ssd_regain.

ssd_regain_static serves callers that cannot allocate device memory (their
device memory is held by another allocator, or their datapath must not pay
cudaMalloc's device synchronisation): it keeps its scratch in one fixed device
array inside the library. Called twice in a row on different RSEAs, through the
C ABI, it must give exactly the list ssd_regain gives - the array keeps the
previous call's contents, so the second call checks that nothing leaks over.
This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

import paper_1803_11036_gb300 as ssd
import trafficgen as tg
from gpu_harness import Run, to_dev
from paper_1803_11036_gb300 import _abi

pytestmark = pytest.mark.gpu


def _static_regain(params, tables_dev, recorders_dev, cap=1 << 16, view=(0, 0, 0)):
    import torch
    ips = torch.empty(cap, dtype=torch.int32, device="cuda:0")
    rk = torch.empty(cap, dtype=torch.int32, device="cuda:0")
    n = ctypes.c_uint64()
    rc = _abi.load().ssd_regain_static(ctypes.byref(params), *view, ctypes.c_void_p(tables_dev.data_ptr()),
                                       ctypes.c_void_p(recorders_dev.data_ptr()), ctypes.c_void_p(ips.data_ptr()),
                                       ctypes.c_void_p(rk.data_ptr()), cap, ctypes.byref(n),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _abi.check(rc, "ssd_regain_static")
    m = n.value
    return ips[:m].cpu().numpy().view(np.uint32), rk[:m].cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("wl,flags", [("paper_c1", 0), ("stress_small", ssd.SSD_VERIFY_H0)])
def test_static_regain_equals_regain_twice(wl, flags):
    import torch
    run = Run(wl, flags)
    tables_dev = torch.from_numpy(tg.hash_tables(run.W["hash_seed"]).view(np.int32)).to("cuda:0")
    params = ssd.make_params(run.W["params"], flags)
    checked = 0
    k = run.W["params"]["k"]
    at = (k - 1, k + 1)   # once the window holds k slots the lists are not empty
    for t in range(k + 2):
        run.step_unfused(None)
        if t not in at:
            continue
        want_ips, want_rk = run.ctx.regain(run.glob)
        rec = torch.from_numpy(run.glob.export().view(np.int16)).to("cuda:0")
        got_ips, got_rk = _static_regain(params, tables_dev, rec)
        assert np.array_equal(got_ips, want_ips) and np.array_equal(got_rk, want_rk), (wl, t)
        assert len(want_ips) > 0
        checked += 1
    assert checked == 2
    run.close()


def test_static_regain_rejects_too_many_columns():
    import torch
    p = ssd.make_params(dict(log2_eta=5, q=21, r=5, delta=6, k=4, theta=20))
    tables_dev = torch.zeros(2048, dtype=torch.int32, device="cuda:0")
    rec = torch.zeros(16, dtype=torch.int16, device="cuda:0")  # never read: the size check comes first
    with pytest.raises(ssd.SSDError) as e:
        _static_regain(p, tables_dev, rec)
    assert e.value.code == ssd.SSD_ECAPACITY


def test_static_regain_of_an_ip_group_sketch():
    """A sketch that counts one IP group (the top two bits of the host): given that view, the
    allocation-free regain lists only the group's hosts, as ssd_regain does, on two calls in a row;
    a view outside the rules is refused."""
    import torch
    W = tg.workload("paper_c1")
    tabs = tg.hash_tables(W["hash_seed"])
    params = ssd.make_params(W["params"])
    ctx = ssd.Context(params, tabs)
    gb, g = 2, 1
    sk = ctx.sketch().set_view(ssd.SSD_SIDE_CNET, gb, g)
    gl = ctx.sketch()
    tables_dev = torch.from_numpy(tabs.view(np.int32)).to("cuda:0")
    T = tg.traffic_for(W)
    checked = 0
    for t in range(W["params"]["k"] + 1):
        ctx.scan(sk, to_dev(T.slot(t)[0]))
        ctx.close_slot([sk], gl)
        if t < W["params"]["k"] - 1:
            continue
        want_ips, want_rk = ctx.regain(gl)
        assert len(want_ips) > 0 and ((want_ips >> np.uint32(32 - gb)) == g).all()
        rec = torch.from_numpy(gl.export().view(np.int16)).to("cuda:0")
        got_ips, got_rk = _static_regain(params, tables_dev, rec, view=gl.view)
        assert np.array_equal(got_ips, want_ips) and np.array_equal(got_rk, want_rk), t
        checked += 1
    assert checked == 2
    with pytest.raises(ssd.SSDError) as e:
        _static_regain(params, tables_dev, rec, view=(0, 2, 4))   # group needs more than 2 bits
    assert e.value.code == _abi.SSD_EINVAL
    ctx.close()
