import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


def rel_max_err(x, ref):
    """Relative max-norm error max|x - ref| / max|ref| (ref all-zero: absolute)."""
    import numpy as np
    x = np.asarray(x)
    ref = np.asarray(ref)
    den = float(np.max(np.abs(ref))) if ref.size else 0.0
    num = float(np.max(np.abs(x - ref))) if ref.size else 0.0
    return num / den if den > 0 else num
