import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def golden():
    with open(os.path.join(GOLDEN, "paper_examples.json")) as f:
        return json.load(f)


@pytest.fixture(scope="session")
def cuda_device():
    """The CUDA device used by gpu tests; skips nothing: a gpu test without a GPU is a failure."""
    import torch
    assert torch.cuda.is_available(), "gpu tests need a CUDA device"
    return torch.device("cuda:0")
