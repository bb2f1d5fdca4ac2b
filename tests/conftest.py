import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")


def load_golden(name):
    """Rows of a tests/golden text fixture: integer columns then one value
    expression (sqrt, pi and fractions allowed)."""
    import math
    path = os.path.join(ROOT, "tests", "golden", name)
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            ints = tuple(int(p) for p in parts[:-1])
            val = eval(parts[-1], {"__builtins__": {}}, {"sqrt": math.sqrt, "pi": math.pi})
            rows.append((ints, float(val)))
    return rows
