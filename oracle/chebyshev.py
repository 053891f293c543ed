"""Polynomial approximation P(x) ~ x^{-1/2} on [eps, 1] (oracle, FP64).

Paper, Sec. 2: sign(H_w) ~ Q P(Q^2) with Q = H_w / ||H_w||, P a degree-n
polynomial approximating x^{-1/2}; its error is delta = |1 - sqrt(x) P(x)| and
obeys the empirical law delta = A exp(-b n sqrt(eps)) with A = 0.41, b = 2.1
(eq. 2), where x = Q^2 ranges over [eps, 1] outside the small space.

The paper names the polynomial family only through its citation; this oracle
uses the Chebyshev interpolant of x^{-1/2} at the n + 1 Chebyshev-Gauss nodes
of y = (2 x - 1 - eps) / (1 - eps) in [-1, 1]:

    P(x) = sum_{k=0}^{n} c_k T_k(y),
    c_k  = (2 - [k == 0]) / (n + 1) * sum_j f(x_j) cos(k theta_j),
    theta_j = pi (j + 1/2) / (n + 1),  y_j = cos(theta_j),

so ``c[0]`` is already the coefficient of T_0 in the sum (the halving is
folded in).
"""
from __future__ import annotations

import math

import numpy as np

#: eq. 2 constants (Sec. 2).
DELTA_A = 0.41
DELTA_B = 2.1


def delta_law(n, sqrt_eps, A=DELTA_A, b=DELTA_B):
    """delta = A exp(-b n sqrt(eps)) (Sec. 2, eq. 2)."""
    return A * math.exp(-b * n * sqrt_eps)


def order_for_delta(delta, sqrt_eps, A=DELTA_A, b=DELTA_B):
    """The order n that eq. 2 gives for a target delta (real-valued)."""
    return math.log(A / delta) / (b * sqrt_eps)


def chebyshev_coeffs(n, eps):
    """Coefficients c_0..c_n of the Chebyshev interpolant of x^{-1/2} on [eps, 1]."""
    j = np.arange(n + 1)
    theta = math.pi * (j + 0.5) / (n + 1)
    y = np.cos(theta)
    x = ((1.0 - eps) * y + 1.0 + eps) / 2.0
    f = 1.0 / np.sqrt(x)
    c = np.empty(n + 1)
    for k in range(n + 1):
        c[k] = 2.0 / (n + 1) * np.sum(f * np.cos(k * theta))
    c[0] /= 2.0
    return c


def to_y(x, eps):
    """The map [eps, 1] -> [-1, 1] on which the Chebyshev basis lives."""
    return (2.0 * x - 1.0 - eps) / (1.0 - eps)


def eval_poly(c, eps, x):
    """P(x) = sum_k c_k T_k(y(x)) by the forward three-term recurrence of T_k."""
    y = to_y(np.asarray(x, dtype=np.float64), eps)
    t_prev = np.ones_like(y)
    total = c[0] * t_prev
    if len(c) == 1:
        return total
    t_cur = y.copy()
    total = total + c[1] * t_cur
    for k in range(2, len(c)):
        t_prev, t_cur = t_cur, 2.0 * y * t_cur - t_prev
        total = total + c[k] * t_cur
    return total


def approximation_error(c, eps, num=20001):
    """delta = max over [eps, 1] of |1 - sqrt(x) P(x)| (Sec. 2), on a dense grid.

    The grid is uniform in theta (y = cos theta), which resolves the
    oscillations of the error near both ends.
    """
    theta = np.linspace(0.0, math.pi, num)
    x = ((1.0 - eps) * np.cos(theta) + 1.0 + eps) / 2.0
    return float(np.max(np.abs(1.0 - np.sqrt(x) * eval_poly(c, eps, x))))
