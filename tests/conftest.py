import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")


def normwise(x, y):
    """max|x - y| / max|y| over a whole tensor (the project's error metric)."""
    import numpy as np
    x = np.asarray(x)
    y = np.asarray(y)
    den = np.abs(y).max()
    return float(np.abs(x - y).max() / (den if den > 0 else 1.0))
