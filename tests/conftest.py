"""Shared fixtures.  Tests marked `gpu` need a CUDA device and the built library."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU case")


_MODE_CACHE = {}


def oracle_modes(cryst):
    """Oracle modes, cached per (crystal name, grid, fc2 bytes)."""
    import oracle.modes as om
    key = (cryst.name, tuple(cryst.grid), cryst.fc2_val.tobytes())
    if key not in _MODE_CACHE:
        _MODE_CACHE[key] = om.modes(cryst)
    return _MODE_CACHE[key]


@pytest.fixture(scope="session")
def sc4():
    from paper_2104_04895_gb300 import synth
    return synth.workload(1)


@pytest.fixture
def rng():
    return np.random.Generator(np.random.PCG64(12345))
