"""The roofline arithmetic of bench.py on the host: the flop model F1 and
its least value over the valid tuples of an axis, against the worked numbers
of the single small configuration (L = 1024, M = 2047) and against a brute
force over every m up to the explicit size."""
import importlib.util
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_model_flops_of_the_small_configuration(bench):
    # (m, q) = (512, 4): 4 (15*512*9 + 6*512 + 24*1024) + 2*1024
    assert bench.model_flops(1024, 512, 4) == 389120
    # (1024, 2): the least-flop tuple of L = 1024, M = 2047
    assert bench.model_flops(1024, 1024, 2) == 370688
    assert bench.floor_flops(1024) == 370688


def test_smooth_numbers_and_floor_by_brute_force(bench):
    def good(n):
        for f in (2, 3, 5, 7):
            while n % f == 0:
                n //= f
        return n == 1

    assert bench.smooth_upto(100) == [n for n in range(1, 101) if good(n)]
    for L in (64, 100, 1536, 3000):
        M = 2 * L - 1
        top = next(n for n in range(M, 4 * M) if good(n))
        brute = min(bench.model_flops(L, m, -(-M // m)) for m in range(16, top + 1) if good(m))
        assert math.isclose(bench.floor_flops(L), brute, rel_tol=0, abs_tol=1e-6)
