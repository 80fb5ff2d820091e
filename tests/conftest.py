import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running statistical check")


@pytest.fixture(scope="session")
def orc():
    """The oracle package (built on first use)."""
    import oracle

    oracle.lib()
    return oracle


def binned_mean_sem(x, nbins=50):
    """Mean and standard error from equal-size bins of a time series."""
    x = np.asarray(x, dtype=np.float64)
    n = (x.size // nbins) * nbins
    bins = x[:n].reshape(nbins, -1).mean(axis=1)
    return bins.mean(), bins.std(ddof=1) / np.sqrt(nbins)
