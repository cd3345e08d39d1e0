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
    """Largest relative error over cells and components of states a against b.

    Each component q is compared as |a - b| / max(|b|, floor_frac * S_q), where
    S_q is the largest magnitude over cells of the physical quantity q belongs
    to: density for q = 0, the momentum vector (rho u, rho v) for q = 1, 2 (so
    a momentum component that is zero everywhere is judged against the flow's
    momentum, not against its own rounding noise), energy for q = 3.
    """
    a = np.asarray(a, np.float64).reshape(-1, 4)
    b = np.asarray(b, np.float64).reshape(-1, 4)
    mom = np.hypot(b[:, 1], b[:, 2]).max() if b.size else 0.0
    scale = np.array([np.abs(b[:, 0]).max(), mom, mom, np.abs(b[:, 3]).max()]) if b.size else 0.0
    den = np.maximum(np.abs(b), np.maximum(floor_frac * scale, 1e-300))
    return float((np.abs(a - b) / den).max()) if b.size else 0.0
