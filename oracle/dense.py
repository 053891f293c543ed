"""Dense-matrix tools for tiny lattices (oracle, FP64).

On 2^4 and 4^4 lattices the operators are small enough (192 and 3072 rows) to
write out as matrices.  A dense Hermitian eigendecomposition of H_w then gives
the exact sign(H_w) and the exact spectral form of the split operator of
Sec. 2, which pin the polynomial path.
"""
from __future__ import annotations

import numpy as np

from . import chebyshev
from .dirac import hermitian_wilson


def operator_matrix(apply, vec_shape):
    """Matrix of a linear map on fields of shape ``vec_shape`` (columns = images of unit vectors)."""
    dim = int(np.prod(vec_shape))
    basis = np.eye(dim, dtype=np.complex128).reshape((dim,) + tuple(vec_shape))
    images = apply(basis)
    return images.reshape(dim, dim).T


def hw_matrix(U, m0, bc=(1, 1, 1, 1), phase=0.0):
    site = U.shape[1:5]
    return operator_matrix(lambda v: hermitian_wilson(U, v, m0, bc, phase), site + (4, 3))


def low_modes(H, hw_norm, n_ev):
    """The n_ev eigenpairs of Q = H / hw_norm of smallest |lambda|.

    Ties in |lambda| are broken by lambda ascending.  Returns (lambda, W) with
    W[:, i] the i-th eigenvector, and the full spectrum (lam_all, W_all).
    """
    lam_all, W_all = np.linalg.eigh(H)
    lam_all = lam_all / hw_norm
    order = np.lexsort((lam_all, np.abs(lam_all)))
    sel = order[:n_ev]
    return lam_all[sel], W_all[:, sel], lam_all, W_all


def split_sign_matrix(lam_all, W_all, n_ev, coeffs, eps):
    """Exact spectral form of the implemented sign function.

    F(Q) = sum_{i <= N} sign(lambda_i) P_i + sum_{i > N} q(lambda_i) P_i with
    q(lambda) = lambda P(lambda^2), the N eigenvalues of smallest |lambda| in
    the first sum.
    """
    order = np.lexsort((lam_all, np.abs(lam_all)))
    f = lam_all * chebyshev.eval_poly(coeffs, eps, lam_all ** 2)
    small = order[:n_ev]
    f[small] = np.where(lam_all[small] >= 0, 1.0, -1.0)
    return (W_all * f) @ W_all.conj().T


def exact_sign_matrix(lam_all, W_all):
    return (W_all * np.where(lam_all >= 0, 1.0, -1.0)) @ W_all.conj().T


def vectors_to_fields(W, site_shape):
    """Columns of W as fields V[N, ...site..., 4, 3]."""
    return W.T.reshape((W.shape[1],) + tuple(site_shape) + (4, 3)).copy()
