"""Matrix sign function, overlap operator D_ov and massive D(m) (oracle, FP64).

Paper, Sec. 2:
  * eq. 1:   D_ov = 1 + gamma5 sign(H_w),  H_w = gamma5 D_w;
  * large space: sign(H_w) ~ Q P(Q^2), Q = H_w / ||H_w||, P ~ x^{-1/2};
  * small space: computed exactly from a few eigenvectors of Q near zero.

Reading of the split (the paper does not spell out the algebra): with an
orthonormal set v_1..v_N (normally the N eigenvectors of Q of smallest |lambda|)
and signs s_i = sign(lambda_i),

    sign(H_w) x = sum_i s_i v_i <v_i, x>  +  Q P(Q^2) (x - sum_i v_i <v_i, x>).

P(Q^2) is evaluated as sum_k c_k T_k(Y) with Y = (2 Q^2 - (1 + eps)) / (1 - eps)
by the forward three-term recurrence T_{k+1} = 2 Y T_k - T_{k-1}.

The massive operator is D(m) = (1 - m/2) D_ov + m (the normalisation that
matches eq. 1's D_ov = 1 + gamma5 sign); m = 0 gives D_ov.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import chebyshev
from .dirac import gamma5, hermitian_wilson


@dataclass
class OverlapParams:
    """What fixes the approximated operator: Wilson mass, boundary factors,
    ||H_w||, the interval [eps, 1] of Q^2 and the Chebyshev coefficients."""

    m0: float
    hw_norm: float
    eps: float
    degree: int
    bc: tuple = (1, 1, 1, 1)
    coeffs: Optional[np.ndarray] = field(default=None, repr=False)

    def __post_init__(self):
        if self.coeffs is None:
            self.coeffs = chebyshev.chebyshev_coeffs(self.degree, self.eps)


@dataclass
class SmallSpace:
    """The exactly treated eigen-space: vectors V[N, ...site..., 4, 3] and signs."""

    V: np.ndarray
    signs: np.ndarray

    @classmethod
    def from_eigenpairs(cls, V, lam):
        # sign(0) is read as +1; it does not occur for random fields.
        return cls(np.asarray(V), np.where(np.asarray(lam) >= 0, 1.0, -1.0))

    @classmethod
    def empty(cls, site_shape):
        return cls(np.zeros((0,) + tuple(site_shape) + (4, 3), np.complex128), np.zeros(0))


def apply_Q(U, psi, p: OverlapParams, phase=0.0):
    """Q psi = H_w psi / ||H_w|| (Sec. 2)."""
    return hermitian_wilson(U, psi, p.m0, p.bc, phase) / p.hw_norm


def apply_Y(U, psi, p: OverlapParams, phase=0.0):
    """Y psi, the map of Q^2 from [eps, 1] onto [-1, 1]."""
    q2 = apply_Q(U, apply_Q(U, psi, p, phase), p, phase)
    return (2.0 * q2 - (1.0 + p.eps) * psi) / (1.0 - p.eps)


def apply_poly_Q2(U, psi, p: OverlapParams, phase=0.0):
    """P(Q^2) psi = sum_k c_k T_k(Y) psi (forward recurrence)."""
    c = p.coeffs
    t_prev = psi
    total = c[0] * t_prev
    if len(c) == 1:
        return total
    t_cur = apply_Y(U, psi, p, phase)
    total = total + c[1] * t_cur
    for k in range(2, len(c)):
        t_prev, t_cur = t_cur, 2.0 * apply_Y(U, t_cur, p, phase) - t_prev
        total = total + c[k] * t_cur
    return total


def _flat(a, lead):
    return a.reshape(a.shape[:lead] + (-1,))


def project(small: SmallSpace, psi):
    """(y_s, x_perp): y_s = sum_i s_i v_i <v_i, psi>, x_perp = psi - sum_i v_i <v_i, psi>.

    ``psi`` may carry leading right-hand-side axes.
    """
    n = small.V.shape[0]
    if n == 0:
        return np.zeros_like(psi), psi
    site_nd = small.V.ndim - 1
    lead = psi.ndim - site_nd
    Vf = small.V.reshape(n, -1)
    pf = psi.reshape(psi.shape[:lead] + (-1,))
    C = pf @ Vf.conj().T  # <v_i, psi>
    ys = (C * small.signs) @ Vf
    perp = pf - C @ Vf
    return ys.reshape(psi.shape), perp.reshape(psi.shape)


def sign_hw(U, psi, p: OverlapParams, small: SmallSpace, phase=0.0):
    """sign(H_w) psi ~ V diag(s) V^+ psi + Q P(Q^2) (1 - V V^+) psi (Sec. 2)."""
    ys, perp = project(small, psi)
    return ys + apply_Q(U, apply_poly_Q2(U, perp, p, phase), p, phase)


def sign_hw_dag(U, psi, p: OverlapParams, small: SmallSpace, phase=0.0):
    """The exact adjoint of ``sign_hw``: V diag(s) V^+ + (1 - V V^+) P(Q^2) Q.

    Equal to ``sign_hw`` when V spans an invariant subspace of Q.
    """
    qp = apply_poly_Q2(U, apply_Q(U, psi, p, phase), p, phase)
    ys, _ = project(small, psi)
    _, perp = project(small, qp)
    return ys + perp


def overlap(U, psi, mass, p: OverlapParams, small: SmallSpace, phase=0.0):
    """D(m) psi = (1 - m/2) (psi + gamma5 sign(H_w) psi) + m psi  (eq. 1; m = 0: D_ov)."""
    d_ov = psi + gamma5(sign_hw(U, psi, p, small, phase))
    return (1.0 - mass / 2.0) * d_ov + mass * psi


def overlap_dag(U, psi, mass, p: OverlapParams, small: SmallSpace, phase=0.0):
    """D(m)^+ psi = (1 - m/2) (psi + sign^+ gamma5 psi) + m psi."""
    d_ov = psi + sign_hw_dag(U, gamma5(psi), p, small, phase)
    return (1.0 - mass / 2.0) * d_ov + mass * psi
