"""Host-side parameter search: candidate enumeration (Section 4.2 grid) and
the tuning database, including corrupt records (host fault injection).
No GPU needed: plans in HDC_TUNE_CACHED_ONLY mode never launch."""
import ctypes as C
import math

import pytest

import paper_2306_10016_gb300 as hdc


@pytest.fixture(scope="module")
def lib():
    hdc.build()
    return hdc.lib()


def F1(L, m, q):
    return q * (15 * m * math.log2(m) + 6 * m + 24 * L) + 2 * L if m > 1 else q * (6 * m + 24 * L) + 2 * L


@pytest.mark.parametrize("L", [1, 6, 100, 1024, 3000, 1 << 16])
def test_candidates_valid_and_within_ratio(lib, L):
    M = 2 * L - 1
    c = hdc.tune_candidates(L, M, hdc.HDC_C128, 1.5, 1)
    assert c, "no candidate"
    best = min(t["model_flops"] for t in c)
    for t in c:
        assert hdc.is_good_size(t["m"])
        assert t["p"] == -(-L // t["m"]) and t["q"] == -(-M // t["m"]) and t["D"] == t["q"]
        assert abs(t["model_flops"] - F1(L, t["m"], t["q"])) <= 1e-9 * t["model_flops"]
        assert t["model_flops"] <= 1.5 * best * (1 + 1e-12)
    flops = [t["model_flops"] for t in c]
    assert flops == sorted(flops)
    # the q = 1 explicit choice and a q = 2 choice are both in for powers of two
    if L >= 16 and (L & (L - 1)) == 0:
        ms = {t["m"] for t in c}
        assert 2 * L in ms and L in ms


def test_candidates_short_axis_keeps_explicit(lib):
    # M = 7 < m_min = 16: the explicit size still qualifies
    c = hdc.tune_candidates(4, 7, hdc.HDC_C128, 1.5, 16)
    assert c and c[0]["m"] == 7 or any(t["m"] == 7 for t in c)


def _db_plan(path, L, mode=hdc.HDC_TUNE_CACHED_ONLY):
    h = C.c_void_p()
    arr = lambda v: (C.c_int64 * 1)(v)
    rc = hdc.lib().hdc_plan_create(C.byref(h), 1, arr(L), arr(2 * L - 1), None, None, hdc.HDC_C128, 1, mode,
                                   str(path).encode(), None)
    return rc, h


def test_tuning_db_lookup_and_corrupt_lines(lib, tmp_path):
    db = tmp_path / "tune.txt"
    key = "v1 unknown 1 1 1 1000 1999"      # no device on this host: key 'unknown'
    db.write_text("\n".join([
        "garbage without a bar",
        key + " | 500 2 4",                          # truncated record: skipped
        key + " | five hundred 2 4 1 0.5",           # non-numeric: skipped
        "v1 unknown 1 1 1 999 1997 | 1000 1 2 2 0.1",  # another problem
        key + " | 512 2 4 4 0.25",                   # the valid record
        "",
    ]))
    rc, h = _db_plan(db, 1000)
    if rc == hdc.HDC_ERR_NOT_TUNED:
        pytest.skip("a CUDA device is visible: the database key carries its name")
    assert rc == hdc.HDC_OK
    m, p, q, D = [(C.c_int64 * 1)() for _ in range(4)]
    assert lib.hdc_plan_params(h, m, p, q, D) == hdc.HDC_OK
    assert (m[0], p[0], q[0], D[0]) == (512, 2, 4, 4)
    assert lib.hdc_plan_workspace(h) > 0
    lib.hdc_plan_destroy(h)
    # a problem with no record
    rc, _ = _db_plan(db, 777)
    assert rc == hdc.HDC_ERR_NOT_TUNED
    # a missing database file
    rc, _ = _db_plan(tmp_path / "missing.txt", 1000)
    assert rc == hdc.HDC_ERR_NOT_TUNED


def test_plan_fixed_and_explicit_on_host(lib):
    h = C.c_void_p()
    arr = lambda *v: (C.c_int64 * len(v))(*v)
    assert lib.hdc_plan_create(C.byref(h), 1, arr(1024), arr(2047), arr(512), arr(1), hdc.HDC_C128, 1,
                               hdc.HDC_FIXED, None, None) == hdc.HDC_OK
    m, p, q, D = [(C.c_int64 * 1)() for _ in range(4)]
    lib.hdc_plan_params(h, m, p, q, D)
    assert (m[0], p[0], q[0], D[0]) == (512, 2, 4, 1)
    lib.hdc_plan_destroy(h)
    assert lib.hdc_plan_create(C.byref(h), 1, arr(1024), arr(2047), None, None, hdc.HDC_C128, 1,
                               hdc.HDC_EXPLICIT, None, None) == hdc.HDC_OK
    lib.hdc_plan_params(h, m, p, q, D)
    assert (m[0], p[0], q[0], D[0]) == (2048, 1, 1, 1)
    lib.hdc_plan_destroy(h)
    # the literal p = 1 of the L=1024, m=512 configuration cannot be planned either
    assert lib.hdc_plan_create(C.byref(h), 1, arr(1024), arr(2046), arr(512), None, hdc.HDC_C128, 1,
                               hdc.HDC_FIXED, None, None) == hdc.HDC_ERR_ALIAS


def test_unequal_candidates_valid_and_near_lf():
    """Every unequal candidate validates; lam > 1 only with f's size m in
    [Lf/2, 2 Lf]; lam = 1 is always among them; sorted by model flops."""
    for Lf, Lg in ((1024, 1 << 22), (100, 1000), (7, 20), (1, 50), (5000, 5000)):
        c = hdc.tune_unequal_candidates(Lf, Lg)
        assert c
        assert any(t["lam"] == 1 for t in c)
        fl = [t["model_flops"] for t in c]
        assert fl == sorted(fl)
        for t in c:
            mg = t["m"] * t["lam"]
            pf, pg, qg, D = hdc.validate_unequal_axis(Lf, Lg, t["m"], t["lam"])
            assert qg == t["q"] == -(-(Lf + Lg - 1) // mg)
            if t["lam"] > 1:
                assert 2 * t["m"] >= Lf and t["m"] <= 2 * Lf


def test_unequal_validation_errors():
    with pytest.raises(hdc.HDCError) as e:
        hdc.validate_unequal_axis(7, 20, 4, 2, M=25)
    assert e.value.code == hdc.HDC_ERR_ALIAS
    with pytest.raises(hdc.HDCError) as e:
        hdc.validate_unequal_axis(7, 20, 4, 11)
    assert e.value.code == hdc.HDC_ERR_UNSUPPORTED_SIZE
    with pytest.raises(hdc.HDCError) as e:
        hdc.validate_unequal_axis(0, 20, 4, 1)
    assert e.value.code == hdc.HDC_ERR_PARAM
    assert hdc.validate_unequal_axis(7, 20, 4, 2) == (2, 3, 4, 4)
