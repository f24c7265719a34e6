"""The limits of the parameter space and of the ABI, against the oracle slot by slot: r = 8 (the
most rows), q = 24 (the most columns: a 3 GiB RSEA at eta = 32), 128 routers in one call (the
most; 129 is refused), and the degenerate ends of the method: theta = 1 (every touched estimator
is hot) with k = 1, and the longest window k = 65534."""
import numpy as np
import pytest

import oracle
import paper_1803_11036_gb300 as ssd
import trafficgen as tg
from gpu_harness import Run, assert_list_equal

pytestmark = pytest.mark.gpu


def run_slots(run, n, step):
    nonempty = 0
    for _ in range(n):
        if step == "slot":
            got, want = run.step_slot("pruned", with_global=True)
        else:
            got, want = run.step_unfused("pruned")
            st = run.ctx.stats()
            assert st["level"] == [int(x) for x in want["levels"]]
        assert_list_equal(got, want, f"slot {run.t}")
        assert np.array_equal(run.glob.export(), run.pipe.global_sk), run.t
        nonempty += len(want["ips"]) > 0
    return nonempty


@pytest.mark.parametrize("step", ["slot", "unfused"])
def test_eight_rows(step):
    """r = SSD_MAX_R = 8 with delta = 4, q = 12: (r-2)*delta + q = 36 bits of windows."""
    W = tg.workload("paper_c1")
    W["params"] = dict(log2_eta=11, q=12, r=8, delta=4, k=4, theta=1024)
    run = Run(W)
    assert run_slots(run, 4, step) > 0
    run.close()


@pytest.mark.parametrize("step", ["slot", "unfused"])
def test_most_columns(step):
    """q = 24, the largest number of columns (2^24 per row): eta = 32, r = 3, delta = 8, a 3 GiB
    RSEA; the bucket index is at its largest (2^16 buckets per row)."""
    W = tg.workload("tiny")
    W["params"] = dict(log2_eta=5, q=24, r=3, delta=8, k=3, theta=40)
    run = Run(W)
    assert run.ctx.sketch_bytes == 3 << 30
    assert run_slots(run, 3, step) > 0
    run.close()


def test_most_routers():
    """128 routers (SSD_MAX_ROUTERS) in one ssd_scan_batch + ssd_close_slot and in one ssd_slot;
    129 are refused."""
    W = tg.workload("tiny")
    W["traffic"]["routers"] = 128
    run = Run(W)
    assert run.n == 128
    for _ in range(2):
        got, want = run.step_fused("pruned")
        assert_list_equal(got, want, f"slot {run.t}")
        assert np.array_equal(run.glob.export(), run.pipe.global_sk)
    for _ in range(2):
        got, want = run.step_slot("pruned", with_global=True)
        assert_list_equal(got, want, f"slot {run.t}")
        assert np.array_equal(run.glob.export(), run.pipe.global_sk)
    extra = run.ctx.sketch()
    with pytest.raises(ssd.SSDError) as e:
        run.ctx.close_slot(run.routers + [extra])
    assert e.value.code == ssd._abi.SSD_EINVAL
    run.close()


@pytest.mark.parametrize("step", ["slot", "unfused"])
def test_threshold_one_discrete_window(step):
    """theta = 1, k = 1: the threshold is one recorder below k, so every estimator touched in the
    slot is hot and nearly every host seen in it is listed, phantoms included."""
    W = tg.workload("tiny")
    W["params"] = dict(W["params"], theta=1, k=1)
    W["traffic"]["k"] = 1
    run = Run(W)
    assert run.ctx.threshold == 1
    assert run_slots(run, 3, step) == 3
    run.close()


def test_longest_window():
    """k = 65534, the longest window (a recorder at 65534 still counts; 65535 means never)."""
    W = tg.workload("tiny")
    W["params"] = dict(W["params"], k=65534)
    run = Run(W)
    assert run_slots(run, 4, "unfused") > 0
    run.close()
