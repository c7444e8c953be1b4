import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU test")


def read_golden(name):
    """Parse a ``key | v1, v2, ...`` fixture from tests/golden (``#`` comments)."""
    import math
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = [p.strip() for p in line.split("|")]
            vals = []
            for part in parts:
                items = [s.strip() for s in part.split(",")]
                try:
                    vals.append([float(eval(s, {"sqrt": math.sqrt, "__builtins__": {}})) for s in items])
                except Exception:
                    vals.append(items)
            rows.append(vals)
    return rows


@pytest.fixture
def golden():
    return read_golden
