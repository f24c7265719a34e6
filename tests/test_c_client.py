"""The C ABI from C: tests/c_client.c compiles as C99 with every warning an error against
include/ssd.h, links against the built libssd.so and runs its host-only part (no GPU)."""
import os
import subprocess

from paper_1803_11036_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_client_builds_and_runs(tmp_path):
    lib = _abi.load() and _abi.lib_path()
    exe = str(tmp_path / "c_client")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_client.c"), "-o", exe, "-L", os.path.dirname(lib),
                           "-lssd", "-Wl,-rpath," + os.path.dirname(lib)])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    assert "threshold 806" in out.stdout and "refusals ok" in out.stdout
