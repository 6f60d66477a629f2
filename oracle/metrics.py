"""Comparison metrics of Sec. 4.2 (as used by ComputeFstatTest).

r_{1,2}(x, y) = 2 |x - y|_{1,2} / (|x|_{1,2} + |y|_{1,2})
theta(x, y)   = arccos[ Re(x* . y) / (|x|_2 |y|_2) ]
"""

from __future__ import annotations

import numpy as np


def r1(x, y) -> float:
    x, y = np.asarray(x), np.asarray(y)
    return float(2.0 * np.sum(np.abs(x - y)) / (np.sum(np.abs(x)) + np.sum(np.abs(y))))


def r2(x, y) -> float:
    x, y = np.asarray(x), np.asarray(y)
    return float(2.0 * np.linalg.norm(x - y) / (np.linalg.norm(x) + np.linalg.norm(y)))


def theta(x, y) -> float:
    x, y = np.asarray(x), np.asarray(y)
    c = np.real(np.vdot(x, y)) / (np.linalg.norm(x) * np.linalg.norm(y))
    return float(np.arccos(np.clip(c, -1.0, 1.0)))
