import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU-only checks")


def load_golden(name):
    """Parse a golden text fixture: '# ...' comment lines, then 'key: numbers' lines.

    Repeated keys are collected into a list of rows.
    """
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(":")
            vals = np.array([float(t) for t in rest.split()])
            key = key.strip()
            if key in out:
                prev = out[key]
                out[key] = (prev if isinstance(prev, list) else [prev]) + [vals]
            else:
                out[key] = vals
    return out


@pytest.fixture
def golden():
    return load_golden
