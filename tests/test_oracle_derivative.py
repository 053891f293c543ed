"""Pins of the oracle's field derivatives and correlator.

dH_w/dphi against a central finite difference of H_w; the Daleckii-Krein
derivative of the split sign operator against finite differences in which the
eigen-split is recomputed at phi +- h (the background-field method's own
quantity); the correlator against an explicit-loop sum and the Frobenius norm
of the dense propagator.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from oracle import correlator, dense, derivative, dirac
from oracle import overlap as ov

M0 = -1.5


@pytest.mark.parametrize("bc,phase", [((0, 1, 1, 0), 0.0), ((1, 1, 1, -1), 0.3), ((-1, 0, 1, 1), -0.8)])
def test_dhw_dphi_matches_finite_difference(bc, phase):
    dims = (4, 2, 2, 6)
    U = synth.random_su3_field(dims, 0.5, 1)
    x = synth.gaussian_spinor(dims, 2, 2)
    h = 1e-5
    fd = (dirac.hermitian_wilson(U, x, M0, bc, phase + h) - dirac.hermitian_wilson(U, x, M0, bc, phase - h)) / (2 * h)
    an = derivative.dhw_dphi(U, x, bc, phase)
    assert np.abs(fd - an).max() / np.abs(an).max() < 1e-8


def test_dhw_dphi_is_hermitian():
    dims = (2, 2, 2, 4)
    U = synth.random_su3_field(dims, 0.5, 3)
    dH = dense.operator_matrix(lambda v: derivative.dhw_dphi(U, v, (0, 1, 1, 0), 0.2), synth.site_shape(dims) + (4, 3))
    assert np.abs(dH - dH.conj().T).max() < 1e-14


def _split(U, bc, phase, hw, n_ev, coeffs, eps):
    H = dense.hw_matrix(U, M0, bc, phase)
    lam_all, W_all = np.linalg.eigh(H)
    return dense.split_sign_matrix(lam_all / hw, W_all, n_ev, coeffs, eps)


@pytest.mark.parametrize("n_ev", [0, 6])
def test_split_sign_derivative_matches_finite_difference(n_ev):
    assert split_derivative_error(n_ev) < 1e-6


def split_derivative_error(n_ev):
    """max |dF_DK - dF_FD| / max |dF_DK| on 2^3 x 4 (Dirichlet x and t, phase 0.15)."""
    dims, bc, phase = (2, 2, 2, 4), (0, 1, 1, 0), 0.15
    U = synth.random_su3_field(dims, 0.4, 5)
    site = synth.site_shape(dims) + (4, 3)
    hw, eps, degree = 6.5, 1e-3, 60
    coeffs = ov.OverlapParams(m0=M0, hw_norm=hw, eps=eps, degree=degree).coeffs
    H = dense.hw_matrix(U, M0, bc, phase)
    dH = dense.operator_matrix(lambda v: derivative.dhw_dphi(U, v, bc, phase), site)
    an = derivative.split_sign_derivative(H, dH, hw, n_ev, coeffs, eps)
    h = 1e-5
    fd = (_split(U, bc, phase + h, hw, n_ev, coeffs, eps) - _split(U, bc, phase - h, hw, n_ev, coeffs, eps)) / (2 * h)
    return np.abs(an - fd).max() / np.abs(an).max()


def test_correlator_matches_loops_and_frobenius_norm():
    dims = (2, 2, 2, 4)
    rng = np.random.default_rng(9)
    S = rng.standard_normal((12,) + synth.site_shape(dims) + (4, 3)) + 1j * rng.standard_normal((12,) + synth.site_shape(dims) + (4, 3))
    C = correlator.pion_correlator(S)
    for t in range(dims[3]):
        s = 0.0
        for j in range(12):
            for z in range(dims[2]):
                for y in range(dims[1]):
                    for x in range(dims[0]):
                        s += float(np.sum(np.abs(S[j, t, z, y, x]) ** 2))
        assert C[t] == pytest.approx(s, rel=1e-13)
    assert C.sum() == pytest.approx(np.linalg.norm(S.ravel()) ** 2, rel=1e-13)
