"""Confidence bounds of logical error rates (no device code, no heavy imports)."""
from __future__ import annotations

Z95 = 1.959963984540054          # the standard normal quantile of 0.975


def wilson95(k: int, n: int):
    """Wilson score interval (95 %) of a binomial proportion k / n: the p whose score statistic
    |k/n - p| / sqrt(p (1 - p) / n) is at most z, in closed form. [0, 1] for n = 0."""
    if n == 0:
        return [0.0, 1.0]
    z = Z95
    ph = k / n
    den = 1 + z * z / n
    c = (ph + z * z / (2 * n)) / den
    h = z / den * (ph * (1 - ph) / n + z * z / (4 * n * n)) ** 0.5
    return [max(0.0, c - h), min(1.0, c + h)]
