"""Closed-form pins for the Sec. 4.2 comparison metrics r1, r2, theta."""

import math

import numpy as np

from oracle import metrics


def test_metrics_closed_forms():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    assert metrics.r1(x, x) == 0.0 and metrics.r2(x, x) == 0.0
    # y = 2x: |x-y| = |x|, |x|+|y| = 3|x|  ->  r = 2/3 in both norms
    assert abs(metrics.r1(x, 2 * x) - 2 / 3) < 1e-14
    assert abs(metrics.r2(x, 2 * x) - 2 / 3) < 1e-14
    # theta is the angle between x and y viewed as real vectors
    assert abs(metrics.theta(x, 1j * x) - math.pi / 2) < 1e-12
    assert abs(metrics.theta(x, -x) - math.pi) < 1e-7
    assert metrics.theta(x, 3.0 * x) < 1e-7
