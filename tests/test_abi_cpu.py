"""The C-ABI library without a GPU: it builds, loads, exports every declared
symbol, and its host-only calls (parameter checks, threshold) agree with the
oracle's independent implementation."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1803_11036_gb300 as ssd
from paper_1803_11036_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ssd.h")).read()
    return re.findall(r"^SSD_API\s+[\w\s\*]+?\b(ssd_\w+)\(", text, flags=re.M)


def test_library_exports_every_declared_symbol():
    L = _abi.load()
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(_abi.SIGNATURES), set(names) ^ set(_abi.SIGNATURES)
    assert L.ssd_version() == 103


def test_only_the_abi_is_exported():
    """-fvisibility=hidden: the shared object exports the ssd_* entry points and nothing of ours beside."""
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.lib_path()], capture_output=True, text=True).stdout
    ours = [ln.split()[-1] for ln in out.splitlines() if " T " in ln]
    assert set(declared_symbols()) <= set(ours)
    assert all(n.startswith("ssd_") or n.startswith("_") for n in ours if "ssd" in n.lower())


def test_strerror_covers_codes():
    L = _abi.load()
    for code in range(0, -7, -1):
        assert L.ssd_strerror(code).decode() != "unknown error"
    assert L.ssd_strerror(-99).decode() == "unknown error"


def _random_params(rng):
    return dict(log2_eta=int(rng.integers(4, 17)), q=int(rng.integers(3, 27)), r=int(rng.integers(2, 10)),
                delta=int(rng.integers(0, 26)), k=int(rng.choice([0, 1, 5, 65534, 65535])),
                theta=int(rng.choice([0, 1, 1024, 5000])))


def test_params_check_agrees_with_oracle():
    """Two independent validators of the paper's constraints (delta < q, (r-2)*delta+q >= 32,
    k <= 65534) agree wherever both domains overlap."""
    rng = np.random.default_rng(0)
    agree = 0
    for _ in range(4000):
        d = _random_params(rng)
        lib_ok = ssd.params_ok(ssd.make_params(d))
        orc_ok = oracle.check_params(oracle.params(d))
        in_lib_domain = 5 <= d["log2_eta"] <= 15 and 3 <= d["r"] <= 8
        if in_lib_domain:
            assert lib_ok == orc_ok, d
            agree += 1
        else:
            assert not lib_ok
    assert agree > 500


@pytest.mark.parametrize("eta,theta", [(2048, 1024), (64, 40), (32, 1), (32768, 1024), (256, 77), (4096, 9999)])
def test_threshold_matches_oracle(eta, theta):
    """Floating point decides the integer threshold; both sides decide it in double on the host."""
    p = ssd.make_params(dict(log2_eta=int(np.log2(eta)), q=14, r=5, delta=6, k=4, theta=theta))
    assert ssd.threshold(p) == oracle.threshold(eta, theta)[0]


def test_create_without_gpu_fails_cleanly():
    """With no CUDA device the context cannot be created; the call returns an error code."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = _abi.load()
    p = ssd.make_params(dict(log2_eta=11, q=14, r=5, delta=6, k=4, theta=1024))
    tables = np.zeros(2048, np.uint32)
    h = ctypes.c_void_p()
    rc = L.ssd_create(ctypes.byref(p), tables.ctypes.data, 0, ctypes.byref(h))
    assert rc in (_abi.SSD_ECUDA, _abi.SSD_EINVAL)
    assert not h.value


def test_debug_build_compiles_and_says_so():
    """The debug library (-DSSD_DEBUG=1) builds for sm_103a, exports the same ABI and reports
    itself; the release library does not."""
    from paper_1803_11036_gb300 import _build
    path = _build.build(debug=True)
    D = ctypes.CDLL(path)
    D.ssd_build_flags.restype = ctypes.c_int
    assert D.ssd_build_flags() == 1
    for n in declared_symbols():
        assert hasattr(D, n), n
    assert _abi.load().ssd_build_flags() == 0
