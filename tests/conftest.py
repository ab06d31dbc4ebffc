import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the sm_103a library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


def load_golden_matrices(name):
    """Parse tests/golden/<name>: blocks of 'matrix <id> <rows> <cols> <rank>' + rows."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", name)
    out = {}
    lines = [l for l in open(path) if l.strip() and not l.startswith("#")]
    i = 0
    while i < len(lines):
        _, mid, r, c, rk = lines[i].split()
        r, c, rk = int(r), int(c), int(rk)
        M = np.array([[float(v) for v in lines[i + 1 + q].split()] for q in range(r)])
        assert M.shape == (r, c)
        out[mid] = (M, rk)
        i += 1 + r
    return out
