"""Derivatives with respect to the background field (oracle, FP64).

Paper, Sec. 4: the electric field enters as a U(1) phase on the links; the
energy shifts follow from correlators computed at several field values.  The
derivative of the correlator with respect to the field is not in the paper;
it is the continuous form of the finite differences the background-field
method takes, and these functions define it plainly:

* ``dhw_dphi``: dH_w/dphi.  With the phase exp(i phi t) on the x links only
  the x hops depend on phi; differentiating exp(i phi t) U_x(n) and
  exp(-i phi t) U_x(n - x)^+ brings the factors i t and -i t.
* ``split_sign_derivative``: the exact derivative of the implemented sign
  function F(H) = sum_{i<=N} sign(l_i) P_i + sum_{i>N} q(l_i) P_i (the N
  eigenvalues of smallest |l| in the first sum) by the Daleckii-Krein formula
  dF = sum_ij F[l_i, l_j] P_i dH P_j, with the divided differences
  F[a, b] = (F(a) - F(b)) / (a - b) and F[a, a] = F'(a).
"""
from __future__ import annotations

import numpy as np

from . import chebyshev
from .dirac import GAMMA, ID4, backward_link, bc_factors, colour_mult, colour_mult_dag, gamma5, neighbour, spin_mult


def dwilson_dphi(U, psi, bc=(1, 1, 1, 1), phase=0.0):
    """dD_w/dphi psi: the x hops of D_w with exp(+-i phi t) replaced by their derivatives."""
    bcf = bc_factors(bc)
    t = np.arange(U.shape[1])
    d_fwd = (1j * t * np.exp(1j * phase * t))[:, None, None, None, None, None]    # d/dphi e^{i phi t}
    d_bwd = (-1j * t * np.exp(-1j * phase * t))[:, None, None, None, None]        # d/dphi e^{-i phi t}
    # forward hop: (1 - gamma_x) [i t e^{i phi t} U_x(n)] psi(n + x)
    fwd = colour_mult(U[0] * d_fwd, neighbour(psi, 0, +1, bcf[0]))
    # backward hop: (1 + gamma_x) [-i t e^{-i phi t} U_x(n - x)^+] psi(n - x)
    bwd = d_bwd[..., None] * colour_mult_dag(backward_link(U[0], 0), neighbour(psi, 0, -1, bcf[0]))
    return -0.5 * (spin_mult(ID4 - GAMMA[0], fwd) + spin_mult(ID4 + GAMMA[0], bwd))


def dhw_dphi(U, psi, bc=(1, 1, 1, 1), phase=0.0):
    """dH_w/dphi psi = gamma5 dD_w/dphi psi."""
    return gamma5(dwilson_dphi(U, psi, bc, phase))


def q_function(theta, coeffs, eps):
    """q(theta) = theta P(theta^2), the large-space approximation of sign (Sec. 2)."""
    return theta * chebyshev.eval_poly(coeffs, eps, theta ** 2)


def q_derivative(theta, coeffs, eps):
    """dq/dtheta = P(theta^2) + 2 theta^2 P'(theta^2), P' from the Chebyshev series."""
    dc = np.polynomial.chebyshev.chebder(coeffs) * (2.0 / (1.0 - eps))  # dP/dx, dy/dx = 2/(1 - eps)
    x = theta ** 2
    y = chebyshev.to_y(x, eps)
    return chebyshev.eval_poly(coeffs, eps, x) + 2.0 * x * np.polynomial.chebyshev.chebval(y, dc)


def split_sign_derivative(H, dH, hw_norm, n_ev, coeffs, eps, degenerate_tol=1e-9):
    """Exact derivative dF of the split sign operator along dH (dense; Daleckii-Krein).

    H, dH: dense Hermitian matrices (H_w and dH_w/dphi).  Eigenvalues of H are
    l = hw_norm * theta; F is sign on the n_ev smallest |theta| and q elsewhere.
    """
    lam, W = np.linalg.eigh(H)
    theta = lam / hw_norm
    order = np.lexsort((theta, np.abs(theta)))
    low = np.zeros(len(theta), bool)
    low[order[:n_ev]] = True
    F = np.where(low, np.where(theta >= 0, 1.0, -1.0), q_function(theta, coeffs, eps))
    dF = np.where(low, 0.0, q_derivative(theta, coeffs, eps) / hw_norm)  # dF/dl on the diagonal
    diff = lam[:, None] - lam[None, :]
    close = np.abs(diff) < degenerate_tol * np.abs(lam).max()
    with np.errstate(divide="ignore", invalid="ignore"):
        dd = (F[:, None] - F[None, :]) / diff
    # (near-)equal eigenvalues: the derivative; they are never split between the two spaces
    dd = np.where(close, 0.5 * (dF[:, None] + dF[None, :]), dd)
    K = W.conj().T @ dH @ W
    return W @ (dd * K) @ W.conj().T
