"""bench.py's contract on the CPU: the reference arm (the oracle timed on the host) prints one JSON
line with every key the contract names; the committed chunk profile's DRAM traffic is used only
while the kernel's code and the launch's chunk size match it; comments and layout do not count as
code for that match."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "Mpps" and d["steps"] == 2
    assert d["higher_is_better"] is True and d["config"]["workload"] == "corelink_c2"
    assert {"value", "unit", "cores", "kind", "sample"} <= set(d["cpu_baseline"])
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "Mpps", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_profile_traffic_needs_matching_code_and_chunk(tmp_path):
    prof = tmp_path / "chunk_pass_w.md"
    prof.write_text(f"traffic_bytes_per_launch: 1.13e9\nkernel_source_sha256_16: {bench.kernel_source_hash()}\n"
                    "chunk_estimators: 131072\n")
    assert bench.profiled_traffic("w", 131072, str(prof)) == 1.13e9
    assert bench.profiled_traffic("w", 262144, str(prof)) is None          # another chunk size
    prof.write_text("traffic_bytes_per_launch: 1.13e9\nkernel_source_sha256_16: 0123456789abcdef\n"
                    "chunk_estimators: 131072\n")
    assert bench.profiled_traffic("w", 131072, str(prof)) is None          # the kernel changed since
    assert bench.profiled_traffic("no_such_workload", 131072) is None
    prof.write_text(f"traffic_bytes_per_launch: 1.13e9\nkernel_source_sha256_16: {bench.kernel_source_hash()}\n"
                    "chunk_estimators: 131072\ncollect_touches: 1\n")
    assert bench.profiled_traffic("w", 131072, str(prof), collect=1) == 1.13e9
    assert bench.profiled_traffic("w", 131072, str(prof), collect=0) is None   # another route


def test_code_tokens_ignore_comments_not_strings():
    a = bench._code_tokens('int a; // note\n/* block\n */ asm("x; // kept");\n\n  int   b;')
    b = bench._code_tokens('int a;\nasm("x; // kept"); int b;')
    assert a == b
    assert bench._code_tokens('asm("x");') != bench._code_tokens('asm("y");')


def test_gbps_conventions():
    g = bench.gbps(1000.0)          # 1 Gpps of 800-byte packets
    assert g["si"] == 6400.0 and g["paper_convention"] == 6250.0


def test_step_rooflines_split():
    """The per-step block: the scan's marginal cost is the pass with the scan minus the close-only
    pass; each fraction is algorithmic bytes / time / peak, where the close-only pass reads every
    recorder once (rec_bytes) and the slot's pass adds the scan's 18 B per packet."""
    s = bench.step_rooflines(pk=6.25e6, scan_ms=1.0, scan_pk=6.25e6, slot_pass=[1.9, 2.1], slot_tail=[0.14],
                             close_pass=[1.7, 1.7], close_tail=[0.13], rec_bytes=5.0e9, r=5, peak=6000.0)
    assert abs(s["scan_in_slot"]["ms_per_slice"] - 0.3) < 1e-9
    assert s["scan_standalone"]["algorithmic_bytes_per_packet"] == 18
    assert abs(s["scan_standalone"]["frac"] - 18 * 6.25e6 / 1e-3 / 1e9 / 6000.0) < 1e-4
    assert abs(s["scan_in_slot"]["frac"] - 18 * 6.25e6 / 0.3e-3 / 1e9 / 6000.0) < 1e-4
    assert s["scan_in_slot"]["target_met"] is False
    assert s["slot_pass"]["algorithmic_bytes"] == 5.0e9 + 18 * 6.25e6
    assert abs(s["slot_pass"]["frac"] - (5.0e9 + 18 * 6.25e6) / 2.0e-3 / 1e9 / 6000.0) < 1e-4
    assert abs(s["close_pass"]["frac"] - 5.0e9 / 1.7e-3 / 1e9 / 6000.0) < 1e-4
    assert s["regain_tail"]["ms_per_slice"] == 0.14
    fast = bench.step_rooflines(pk=6.25e6, scan_ms=1.0, scan_pk=6.25e6, slot_pass=[1.701], slot_tail=[0.1],
                                close_pass=[1.7], close_tail=[0.1], rec_bytes=1e9, r=5, peak=6000.0)
    assert fast["scan_in_slot"]["target_met"] is True


def test_cpu_baseline_reports_each_oracle_step():
    import trafficgen as tg
    r = bench.cpu_baseline(tg.workload("tiny"), budget_s=0.2, min_slots=3)
    assert r["kind"] == "oracle" and r["cores"] == 1 and r["value"] > 0 and r["cpu_model"]
    st = r["steps"]
    for key in ("scan_ns_per_packet", "advance_ms_per_slot", "merge_ms_per_slot", "regain_ms_per_slot"):
        assert st[key] >= 0
    n = int(r["sample"].split()[0])
    # the steps are parts of the timed slots
    per_slot_ms = st["advance_ms_per_slot"] + st["merge_ms_per_slot"] + st["regain_ms_per_slot"]
    assert per_slot_ms * n / 1e3 <= r["seconds"] * 1.05 + 0.05


def test_tuning_flag_parses_a_stated_configuration(monkeypatch):
    import json
    t = {"touch_chunk_bytes": 67108864, "scan_unroll": 8, "collect_touches": 1}
    monkeypatch.setattr("sys.argv", ["bench.py", "--tuning", json.dumps(t), "--steps", "2"])
    args = bench.parse()
    assert json.loads(args.tuning) == t and args.steps == 2 and not args.no_tune
