"""The pair level on the tensor cores (k_pairs_tc: the popcounts of the ANDed "recorder < k"
bitmaps of HSE(0) x HSE(1) as one fp8 GEMM of the bitmaps read as 0/1 vectors, f32 sums in tensor
memory) against the oracle: with pair_level 0 (tensor cores) and 1 (CUDA-core tiles) every slot's
list, R_k and per-level candidate counts equal the oracle's pruned regain. The workloads' hot sets
span several 128 x 256 tiles with ragged edges (stress_small, with more planted hosts above the
threshold, has over 256 hot estimators in rows 0 and 1), and the small bitmaps of eta < 128 fall
back to the CUDA cores."""
import pytest

import trafficgen as tg
from gpu_harness import Run, assert_list_equal

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pair_level", [0, 1])
@pytest.mark.parametrize("wl", ["tiny", "paper_c1", "corelink_small", "stress_small"])
def test_pair_level_matches_oracle(wl, pair_level):
    W = tg.workload(wl)
    if wl == "stress_small":   # 600 planted hosts, most of them above the threshold
        W["traffic"].update(n_planted=600, planted_lo=1100, planted_hi=2000)
    run = Run(W)
    run.ctx.tuning = dict(pair_level=pair_level)
    biggest = 0
    for _ in range(min(run.W["slots"], 8)):
        got, want = run.step_fused("pruned")
        assert_list_equal(got, want, f"{wl} slot {run.t}")
        st = run.ctx.stats()
        assert st["level"] == [int(x) for x in want["levels"]], run.t
        biggest = max(biggest, min(st["hot"][0], st["hot"][1]))
    if wl == "stress_small":
        assert biggest > 256     # more than one tile in both directions
    run.close()
