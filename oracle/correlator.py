"""Pion correlator from point-source propagators (oracle, FP64).

Paper, Sec. 4: energy shifts come from ratios of correlation functions with
and without the field.  The correlator the derivative is taken of (the paper
does not write it out) is the connected pseudoscalar one built from the 12
spin-colour point-source solutions S_j = D(m)^{-1} b_j:

    C(t) = sum_{x, y, z} sum_j sum_{spin, colour} |S_j(x, y, z, t)|^2 .
"""
from __future__ import annotations

import numpy as np


def pion_correlator(S):
    """C(t) from propagator columns S[j, t, z, y, x, spin, colour]."""
    return np.sum(np.abs(S) ** 2, axis=(0, 2, 3, 4, 5, 6))
