import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: long CPU test")


def read_golden(name):
    """Parse a golden fixture: blocks '<label> <rows> <cols>' followed by rows."""
    import numpy as np

    path = os.path.join(ROOT, "tests", "golden", name)
    blocks = {}
    cur = None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0].isalpha() or parts[0][0].isalpha():
                cur = parts[0]
                blocks[cur] = []
                continue
            blocks[cur].append([float(v) for v in parts])
    return {k: np.array(v) for k, v in blocks.items()}
