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


def check_best_timed(best, trials):
    """The tuner's choice is one of its timed configurations, and its time
    (the median of that configuration's timings: the leaders of a search are
    timed three times, interleaved) lies within that configuration's
    recorded times."""
    names = [k for k in best[0] if k != "ms"]

    def key(cfg):
        return tuple(tuple(a[k] for k in names) for a in cfg)

    times = [t[0]["ms"] for t in trials if key(t) == key(best)]
    assert times, "the chosen configuration was never timed"
    assert min(times) - 1e-9 <= best[0]["ms"] <= max(times) + 1e-9
