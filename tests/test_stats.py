"""The Wilson score interval of the reported logical error rates, against scipy's independent
implementation and the closed forms of its edge cases."""
import pytest

from paper_2605_17796_gb300.stats import wilson95


def test_against_scipy():
    stats = pytest.importorskip("scipy.stats")
    for n in (1, 7, 100, 4096, 10 ** 6):
        for k in sorted({0, 1, n // 3, n // 2, n - 1, n}):
            ci = stats.binomtest(k, n).proportion_ci(confidence_level=0.95, method="wilson")
            lo, hi = wilson95(k, n)
            assert abs(lo - ci.low) < 1e-12 and abs(hi - ci.high) < 1e-12, (k, n)


def test_closed_forms():
    z2 = 1.959963984540054 ** 2
    for n in (10, 1000, 10 ** 6):
        lo, hi = wilson95(0, n)
        assert lo < 1e-15 and abs(hi - z2 / (n + z2)) < 1e-15
        lo2, hi2 = wilson95(n, n)
        assert abs(lo2 - (1 - hi)) < 1e-15 and abs(hi2 - 1.0) < 1e-15
        for k in (1, n // 4, n // 2):
            a, b = wilson95(k, n)
            c, d = wilson95(n - k, n)
            assert abs(a - (1 - d)) < 1e-12 and abs(b - (1 - c)) < 1e-12 and a <= k / n <= b
    assert wilson95(0, 0) == [0.0, 1.0]
