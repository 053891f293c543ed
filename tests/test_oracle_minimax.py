"""The oracle's minimax polynomial (Remez) against what fixes it independently.

* n = 0 has a closed form: the constant c equioscillating at x = eps and x = 1,
  1 - sqrt(eps) c = -(1 - c), so c = 2 / (1 + sqrt(eps)), delta = (1 - sqrt(eps)) / (1 + sqrt(eps)).
* Chebyshev's alternation theorem: the error 1 - sqrt(x) P(x) of the minimax polynomial reaches
  +-delta with alternating signs at n + 2 points of [eps, 1].
* It is never worse than the interpolant of the same degree.
* Sec. 2, eq. 2: the paper quotes delta = A exp(-b n sqrt(eps)), A = 0.41, b = 2.1, for this
  kind of polynomial: over the configurations' range the measured delta stays within a factor
  1.5 of the law and its decay rate in n sqrt(eps) is 2.1 to 5 %.
* A planted mistake (the weight sqrt(x) dropped from the levelled system) breaks the pins.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import chebyshev as ch


def error_fn(c, eps, theta):
    y = -np.cos(theta)
    x = ((1.0 - eps) * y + 1.0 + eps) / 2.0
    return 1.0 - np.sqrt(x) * np.polynomial.chebyshev.chebval(y, c)


@pytest.mark.parametrize("eps", [0.01, 4e-4])
def test_degree_zero_closed_form(eps):
    c, d = ch.minimax_coeffs(0, eps)
    s = math.sqrt(eps)
    assert c[0] == pytest.approx(2.0 / (1.0 + s), rel=1e-12)
    assert d == pytest.approx((1.0 - s) / (1.0 + s), rel=1e-12)


@pytest.mark.parametrize("n,eps", [(5, 0.05), (40, 0.01), (120, 0.002)])
def test_equioscillation(n, eps):
    c, d = ch.minimax_coeffs(n, eps)
    theta = np.linspace(0.0, math.pi, 200 * (n + 2) + 1)
    e = error_fn(c, eps, theta)
    assert np.abs(e).max() <= d * (1 + 1e-4)
    # alternating extrema of size delta: count sign-alternating points where |e| > (1 - 1e-3) delta
    big = e[np.abs(e) > (1 - 1e-3) * d]
    alternations = 1 + int(np.count_nonzero(np.diff(np.sign(big)) != 0))
    assert alternations >= n + 2


@pytest.mark.parametrize("n,eps", [(8, 0.1), (64, 0.01), (200, 4e-4)])
def test_never_worse_than_the_interpolant(n, eps):
    _, d = ch.minimax_coeffs(n, eps)
    di = ch.approximation_error(ch.chebyshev_coeffs(n, eps), eps)
    assert d < di


def test_paper_delta_law():
    """eq. 2 with the paper's A and b, at sqrt(eps) = 0.02 (configs 2-4) and 0.1."""
    for s in (0.02, 0.1):
        ns = [100, 150, 200, 250] if s == 0.02 else [20, 40, 60, 80]
        deltas = [ch.minimax_coeffs(n, s * s)[1] for n in ns]
        for n, d in zip(ns, deltas):
            assert 1 / 1.5 < d / ch.delta_law(n, s) < 1.5, (n, s, d)
        slope = -np.polyfit([n * s for n in ns], np.log(deltas), 1)[0]
        assert slope == pytest.approx(ch.DELTA_B, rel=0.05), slope


def test_planted_mistake_is_caught():
    """Drop the relative-error weight sqrt(x) from the levelled system: the result is a
    (worse) polynomial that fails the equioscillation pin."""
    real_sqrt = np.sqrt
    n, eps = 40, 0.01
    c_good, d_good = ch.minimax_coeffs(n, eps)

    def wrong_minimax():
        # the same exchange with the weight removed: minimise |1/sqrt(x) - P(x)| instead
        i = np.arange(n + 2)
        y = -np.cos(math.pi * i / (n + 1))
        T = np.cos(np.outer(np.arccos(y), np.arange(n + 1)))
        M = np.hstack([T, ((-1.0) ** i)[:, None]])
        x = ((1.0 - eps) * y + 1.0 + eps) / 2.0
        return np.linalg.solve(M, 1.0 / real_sqrt(x))[: n + 1]

    c_bad = wrong_minimax()
    theta = np.linspace(0.0, math.pi, 200 * (n + 2) + 1)
    assert np.abs(error_fn(c_bad, eps, theta)).max() > 1.5 * d_good
