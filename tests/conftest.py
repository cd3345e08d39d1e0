"""Shared pytest configuration: the ``gpu`` marker and small helpers."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def read_golden(name):
    """Parses a ``key value`` fixture from tests/golden (``#`` starts a comment)."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                out[k] = float(v)
    return out


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


def rel_err_max(a, b, floor_frac=1e-3):
    """max over cells and components of |a-b| / max(|b|, floor_frac * max_cells |b_comp|)."""
    a = np.asarray(a, np.float64).reshape(-1, 4)
    b = np.asarray(b, np.float64).reshape(-1, 4)
    floor = floor_frac * np.abs(b).max(axis=0)
    den = np.maximum(np.abs(b), np.maximum(floor, 1e-300))
    return float((np.abs(a - b) / den).max())
