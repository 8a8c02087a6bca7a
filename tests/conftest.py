import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 and the CUDA library (run with -m gpu)")
    config.addinivalue_line("markers", "slow: longer CPU checks")


def phys(h: np.ndarray) -> np.ndarray:
    """Grid field of a half spectrum (numpy, independent of both paths)."""
    n = h.shape[0]
    return np.fft.irfft2(h, s=(n, n))


def dot(a: np.ndarray, b: np.ndarray) -> float:
    """Euclidean inner product over grid values of two half spectra or grids."""
    A = phys(a) if np.iscomplexobj(a) else a
    B = phys(b) if np.iscomplexobj(b) else b
    return float(np.sum(A * B))


def rel(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle
