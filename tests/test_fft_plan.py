"""The FFT engine's radix plans (host logic, no GPU): every {2,3,5}-smooth length is
factored completely into supported radices, the double-float plans avoid radix 10, powers
of two keep the radix-8 plan, and mixed lengths take no more stages than the plain
radix-8/4/2/3/5 factorisation."""
import numpy as np
import pytest

from paper_1308_0730_gb300 import mvd


@pytest.fixture(scope="module")
def lib():
    return mvd.load()


def _smooth(n):
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


def _plain_stage_count(L):
    a = n3 = n5 = 0
    while L % 2 == 0:
        L //= 2
        a += 1
    while L % 3 == 0:
        L //= 3
        n3 += 1
    while L % 5 == 0:
        L //= 5
        n5 += 1
    q, rem = divmod(a, 3)
    return q + (rem != 0) + n3 + n5  # 8s, then one 4 or 2 (or 4 4 for an 8 2), then 3s and 5s


@pytest.mark.parametrize("precision", ["precise", "mixed", "fast"])
def test_plans_factor_every_smooth_length(lib, precision):
    allowed = {2, 3, 4, 5, 6, 8, 9} | ({10} if precision == "fast" else set())
    for L in range(2, 2049):
        plan = mvd.mvd_fft_plan(L, precision)
        if not _smooth(L):
            assert plan == [], L
            continue
        assert int(np.prod(plan)) == L, (L, plan)
        assert set(plan) <= allowed, (L, plan)
        if L & (L - 1) == 0:  # powers of two: radix 8 with one 4 or 2 (4 4 instead of 8 2)
            assert all(r == 8 for r in plan[:-2]) and set(plan) <= {8, 4, 2}, (L, plan)
            assert plan.count(2) <= 1 and (plan.count(2) == 0 or len(plan) == 1), (L, plan)
        else:
            assert plan == sorted(plan, reverse=True), (L, plan)
            assert len(plan) <= _plain_stage_count(L), (L, plan)


def test_known_plans(lib):
    assert mvd.mvd_fft_plan(270, "precise") == [9, 6, 5]
    assert mvd.mvd_fft_plan(270, "fast") == [10, 9, 3]
    assert mvd.mvd_fft_plan(256, "precise") == [8, 8, 4]
    assert mvd.mvd_fft_plan(16, "fast") == [4, 4]
    assert mvd.mvd_fft_plan(7, "fast") == []


def test_plan_arguments(lib):
    import ctypes

    buf = (ctypes.c_int * 2)()
    assert lib.mvd_fft_plan(270, mvd.MVD_PRECISE, buf, 2) == -1  # three stages do not fit
    assert lib.mvd_fft_plan(270, 7, buf, 2) == -1
    assert lib.mvd_fft_plan(270, mvd.MVD_PRECISE, None, 8) == -1
    assert lib.mvd_fft_plan(1, mvd.MVD_FAST, buf, 2) == 0
