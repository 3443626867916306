import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def ora():
    import oracle

    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def rng():
    return np.random.default_rng(12345)


def rel_err(x, ref, floor_frac=0.1, scale=None):
    """Per-row error |x - ref| / max(|ref|, floor_frac * rms|ref|) for (n, 3) arrays.

    With `scale` (per row: the sum of the magnitudes of the terms summed into
    ref), the denominator is at least that scale: a sum whose terms cancel is
    rounded relative to its terms, not to its small result."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    nr = np.linalg.norm(ref, axis=1)
    rms = np.sqrt((nr ** 2).mean()) if nr.size else 0.0
    den = np.maximum(nr, floor_frac * rms)
    if scale is not None:
        den = np.maximum(den, np.asarray(scale, dtype=np.float64))
    den = np.where(den > 0, den, 1.0)
    return np.linalg.norm(x - ref, axis=1) / den
