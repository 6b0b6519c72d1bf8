import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built "
        "liblbm.so")
    config.addinivalue_line("markers", "slow: long CPU test")


def read_golden(name):
    """key = value lines (comments with #) or whitespace tables."""
    path = os.path.join(ROOT, "tests", "golden", name)
    out = {}
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if "=" in line:
                k, v = line.split("=", 1)
                out[k.strip()] = float(v)
            else:
                rows.append(line.split())
    return out if out else rows
