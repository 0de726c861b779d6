import os
import sys
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers",
                            "gpu: needs a CUDA GPU and the built libhz.so")
    config.addinivalue_line("markers", "slow: longer CPU test")


def load_golden(name):
    """Parse a tests/golden/*.txt fixture: '[key]' headers followed by rows
    of numbers (fractions allowed, 'C' read as 0); '#' lines are comments."""
    out, key, rows = {}, None, []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                if key is not None:
                    out[key] = np.array(rows, dtype=np.float64)
                key, rows = line[1:-1], []
                continue
            rows.append([0.0 if t == "C" else float(Fraction(t))
                         for t in line.split()])
    if key is not None:
        out[key] = np.array(rows, dtype=np.float64)
    return out


@pytest.fixture
def golden():
    return load_golden
