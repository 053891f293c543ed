"""Conjugate gradient for D(m) x = b (oracle, FP64).

Paper, Sec. 3.2: the propagator D^{-1} psi is computed with a CG method.  The
paper's solver is adaptive and multi-mass; the oracle is the plain textbook
form, CG on the normal equations D^+ D x = D^+ b from x0 = 0 (CGNE), which
reaches the same solution.  It stops when the true relative residual
||b - D x|| / ||b|| is at most ``tol``.
"""
from __future__ import annotations

import numpy as np

from .dirac import inner, norm


def cgne(apply_D, apply_Ddag, b, tol=1e-10, maxiter=10000, check_every=1):
    """Solve D x = b; returns (x, iterations, true relative residual)."""
    bnorm = norm(b)
    x = np.zeros_like(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    r = apply_Ddag(b)
    p = r.copy()
    rr = np.real(inner(r, r))
    true_res = 1.0
    for it in range(1, maxiter + 1):
        Ap = apply_Ddag(apply_D(p))
        alpha = rr / np.real(inner(p, Ap))
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = np.real(inner(r, r))
        if it % check_every == 0:
            true_res = norm(b - apply_D(x)) / bnorm
            if true_res <= tol:
                return x, it, true_res
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, maxiter, true_res
