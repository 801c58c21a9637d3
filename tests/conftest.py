import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def synth():
    from paper_2510_07764_gb300 import synth
    return synth


@pytest.fixture(scope="session")
def small_lens(synth):
    """Lens grid around u = 0.3445 (M = 1.4, R = 12 km) at the paper's density."""
    return synth.LensSpec(u_min=0.30, u_max=0.40, n_u=129, n_cpsi=512)


@pytest.fixture(scope="session")
def atm(synth):
    return synth.atm_table()


def rel_err(a, b, floor_frac=1e-6):
    """Per-bin relative error where |b| >= floor_frac * max|b|."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m = np.abs(b) >= floor_frac * np.max(np.abs(b))
    return np.max(np.abs(a[m] - b[m]) / np.abs(b[m])) if m.any() else 0.0
