import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU statistics test")


def golden(name):
    return os.path.join(ROOT, "tests", "golden", name)


def read_gas_values():
    out = {}
    with open(golden("paper_gas_values.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()[:2]
            out[k] = float(v)
    return out
