"""Polynomial approximation P(x) ~ x^{-1/2} on [eps, 1] (oracle, FP64).

Paper, Sec. 2: sign(H_w) ~ Q P(Q^2) with Q = H_w / ||H_w||, P a degree-n
polynomial approximating x^{-1/2}; its error is delta = |1 - sqrt(x) P(x)| and
obeys the empirical law delta = A exp(-b n sqrt(eps)) with A = 0.41, b = 2.1
(eq. 2), where x = Q^2 ranges over [eps, 1] outside the small space.

The paper names the polynomial family only through its citation (a minimax
construction, whose error eq. 2 describes).  This oracle has both: the minimax
polynomial by the Remez exchange (``minimax_coeffs``, below) and the Chebyshev
interpolant of x^{-1/2} at the n + 1 Chebyshev-Gauss nodes of
y = (2 x - 1 - eps) / (1 - eps) in [-1, 1]:

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


def minimax_coeffs(n, eps, max_iter=80, rtol=1e-6):
    """The degree-n polynomial of least relative error for x^{-1/2} on [eps, 1].

    Minimises delta = max over [eps, 1] of |1 - sqrt(x) P(x)| over polynomials P of degree n
    (the minimax construction the paper's eq. 2 describes, Sec. 2) by the Remez exchange
    algorithm, in the same basis P = sum_k c_k T_k(y), y = (2x - 1 - eps)/(1 - eps):

    * on a reference of n + 2 points y_0 < ... < y_{n+1}, solve
      sqrt(x_i) P(x_i) + (-1)^i E = 1 for c_0..c_n and the levelled error E;
    * take as the next reference the n + 2 alternating extrema of 1 - sqrt(x) P(x)
      (a grid uniform in theta, y = -cos(theta), 64 points per oscillation, each extremum
      refined by a parabola in theta);
    * stop when the largest error exceeds |E| by less than rtol, or by less than 1e-3 and
      by more than half the previous excess (the error function itself is computed with a
      rounding of ~1e-14, which at delta ~ 1e-10 bounds how level it can get).

    Returns (c, delta) with delta the largest |error| on the final grid.
    """
    i = np.arange(n + 2)
    y_ref = -np.cos(math.pi * i / (n + 1))  # Chebyshev extrema, ascending
    sgn = (-1.0) ** i
    theta = np.linspace(0.0, math.pi, 64 * (n + 2) + 1)
    c, delta = None, None
    prev_excess = float("inf")
    for _ in range(max_iter):
        x_ref = ((1.0 - eps) * y_ref + 1.0 + eps) / 2.0
        T = np.cos(np.outer(np.arccos(np.clip(y_ref, -1.0, 1.0)), np.arange(n + 1)))
        M = np.empty((n + 2, n + 2))
        M[:, : n + 1] = np.sqrt(x_ref)[:, None] * T
        M[:, n + 1] = sgn
        sol = np.linalg.solve(M, np.ones(n + 2))
        c, E = sol[: n + 1], sol[n + 1]

        def err_at(th):
            y = -np.cos(th)
            x = ((1.0 - eps) * y + 1.0 + eps) / 2.0
            return 1.0 - np.sqrt(x) * np.polynomial.chebyshev.chebval(y, c)

        e = err_at(theta)
        # local extrema of e on the grid (endpoints included), refined by a parabola in theta
        ext = [0]
        for k in range(1, len(e) - 1):
            if (e[k] - e[k - 1]) * (e[k + 1] - e[k]) <= 0.0 and e[k] != e[k - 1]:
                ext.append(k)
        ext.append(len(e) - 1)
        pts, vals = [], []
        h = theta[1] - theta[0]
        for k in ext:
            th = theta[k]
            if 0 < k < len(e) - 1:
                den = e[k - 1] - 2.0 * e[k] + e[k + 1]
                if den != 0.0:
                    th = theta[k] + 0.5 * h * (e[k - 1] - e[k + 1]) / den
            pts.append(th)
            vals.append(float(err_at(np.array([th]))[0]))
        # alternating subsequence: of neighbours with equal sign keep the larger |error|
        alt_t, alt_v = [], []
        for th, v in zip(pts, vals):
            if alt_v and np.sign(v) == np.sign(alt_v[-1]):
                if abs(v) > abs(alt_v[-1]):
                    alt_t[-1], alt_v[-1] = th, v
            else:
                alt_t.append(th)
                alt_v.append(v)
        while len(alt_t) > n + 2:  # drop the smaller of the two ends
            if abs(alt_v[0]) < abs(alt_v[-1]):
                alt_t.pop(0)
                alt_v.pop(0)
            else:
                alt_t.pop()
                alt_v.pop()
        delta = max(abs(v) for v in alt_v)
        if len(alt_t) < n + 2:
            raise RuntimeError("Remez: fewer than n + 2 alternating extrema")
        y_ref = -np.cos(np.array(alt_t))
        sgn = np.sign(np.array(alt_v))
        excess = (delta - abs(E)) / abs(E)
        if excess <= rtol or (excess < 1e-3 and excess > 0.5 * prev_excess):
            break
        prev_excess = excess
    return c, delta
