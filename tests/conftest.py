import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def gpu_available():
    import torch
    return torch.cuda.is_available()


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_printed(name="printed_velocities.txt"):
    """Values the paper prints, from a text fixture under tests/golden/:
    {key: (value, citation)}; '#' starts a comment line."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, value, cite = line.split(None, 2)
            out[key] = (float(value), cite)
    return out


@pytest.fixture(scope="session")
def printed():
    return {k: v for k, (v, _) in read_printed().items()}
