"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins catch them.

Each case patches one piece of the oracle with a typical bug -- a sign, a
missing dagger, a shifted index, a dropped halving -- and asserts that the
corresponding pin measure in ``test_oracle_pins`` moves far outside its
tolerance.  This shows the pins can fail, not only that they pass.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from oracle import chebyshev, derivative, dirac
from oracle import overlap as ov

import test_oracle_derivative as dpins
import test_oracle_pins as pins


def _free_error():
    dims = (4, 6, 2, 8)
    return pins.free_plane_wave_error(dims, (1, 1, 1, -1), pins.lattice_momenta(dims, True, 12))


def test_flipped_gamma_sign_is_caught(monkeypatch):
    g = dirac.GAMMA.copy()
    g[0] = -g[0]
    monkeypatch.setattr(dirac, "GAMMA", g)
    assert _free_error() > 0.1


def test_transposed_gamma_is_caught(monkeypatch):
    monkeypatch.setattr(dirac, "GAMMA", np.ascontiguousarray(dirac.GAMMA.transpose(0, 2, 1)))
    assert _free_error() > 0.1


def test_swapped_hop_direction_is_caught(monkeypatch):
    orig = dirac.neighbour
    monkeypatch.setattr(dirac, "neighbour", lambda psi, mu, d, bc: orig(psi, mu, -d, bc))
    assert _free_error() > 0.1


def test_missing_dagger_on_backward_link_is_caught(monkeypatch):
    monkeypatch.setattr(dirac, "colour_mult_dag", dirac.colour_mult)
    assert pins.hermiticity_error((4, 4, 2, 6), (1, 1, 1, -1), 0.0) > 1e-3
    assert pins.gauge_covariance_error((4, 2, 6, 4), (1, 1, 1, 1), 0.0) > 1e-3


def test_backward_link_at_wrong_site_is_caught(monkeypatch):
    monkeypatch.setattr(dirac, "backward_link", lambda u, mu: u)
    assert pins.gauge_covariance_error((4, 2, 6, 4), (1, 1, 1, 1), 0.0) > 1e-3


def test_conjugated_field_phase_is_caught(monkeypatch):
    orig = dirac.link
    monkeypatch.setattr(dirac, "link", lambda U, mu, phase=0.0: orig(U, mu, -phase))
    assert pins.brute_force_error((2, 2, 2, 4), (0, 1, -1, 0), 0.4) > 1e-3


def test_unhalved_chebyshev_c0_is_caught(monkeypatch):
    orig = chebyshev.chebyshev_coeffs

    def bad(n, eps):
        c = orig(n, eps)
        c[0] *= 2
        return c

    monkeypatch.setattr(chebyshev, "chebyshev_coeffs", bad)
    c = chebyshev.chebyshev_coeffs(64, 0.01)
    ref = np.polynomial.chebyshev.chebinterpolate(lambda y: 1 / np.sqrt(((0.99) * y + 1.01) / 2), 64)
    assert np.abs(c - ref).max() > 0.1
    assert chebyshev.approximation_error(c, 0.01) > 0.5


@pytest.fixture(scope="module")
def setup():
    return pins.small_lattice_setup()


def test_dropped_small_space_signs_are_caught(setup):
    U, params, small, lam_q, W_all, phase = setup
    bad = ov.SmallSpace(small.V, np.ones_like(small.signs))
    assert np.any(small.signs < 0)
    assert pins.dense_split_error((U, params, bad, lam_q, W_all, phase)) > 1e-3


def test_missing_projector_is_caught(setup, monkeypatch):
    orig = ov.project

    def bad(small, psi):
        ys, _ = orig(small, psi)
        return ys, psi

    monkeypatch.setattr(ov, "project", bad)
    assert pins.dense_split_error(setup) > 1e-3


def test_dagger_without_gamma5_is_caught(setup, monkeypatch):
    """D(m)^+ that applies sign^+ to psi instead of gamma5 psi."""
    def bad(U, psi, mass, p, small, phase=0.0):
        d_ov = psi + ov.sign_hw_dag(U, psi, p, small, phase)
        return (1.0 - mass / 2.0) * d_ov + mass * psi

    monkeypatch.setattr(ov, "overlap_dag", bad)
    assert pins.shifted_family_error(setup, 0.3) > 1e-3


def test_wrong_mass_normalisation_is_caught(setup, monkeypatch):
    """D(m) = (1 + m/2) D_ov + m in place of (1 - m/2) D_ov + m."""
    orig = ov.overlap

    def bad(U, psi, mass, p, small, phase=0.0):
        return orig(U, psi, mass, p, small, phase) + mass * (orig(U, psi, 0.0, p, small, phase))

    monkeypatch.setattr(ov, "overlap", bad)
    U, params, small, _, _, _ = setup
    x = synth.gaussian_spinor((2, 2, 2, 2), 1, 41)[0]
    assert np.linalg.norm(ov.overlap(U, x, 2.0, params, small) - 2.0 * x) > 1e-3
    assert pins.shifted_family_error(setup, 0.3) > 1e-3


def test_wrong_interval_map_is_caught(setup, monkeypatch):
    """Y = (2 Q^2 - (1 - eps)) / (1 - eps): the interval [eps, 1] mapped off [-1, 1]."""
    def bad(U, psi, p, phase=0.0):
        q2 = ov.apply_Q(U, ov.apply_Q(U, psi, p, phase), p, phase)
        return (2.0 * q2 - (1.0 - p.eps) * psi) / (1.0 - p.eps)

    monkeypatch.setattr(ov, "apply_Y", bad)
    assert pins.dense_split_error(setup) > 1e-3


def test_recurrence_without_factor_two_is_caught(setup, monkeypatch):
    """T_{k+1} = Y T_k - T_{k-1} in place of 2 Y T_k - T_{k-1}."""
    def bad(U, psi, p, phase=0.0):
        c = p.coeffs
        t_prev, t_cur = psi, ov.apply_Y(U, psi, p, phase)
        total = c[0] * t_prev + c[1] * t_cur
        for k in range(2, len(c)):
            t_prev, t_cur = t_cur, ov.apply_Y(U, t_cur, p, phase) - t_prev
            total = total + c[k] * t_cur
        return total

    monkeypatch.setattr(ov, "apply_poly_Q2", bad)
    assert pins.dense_split_error(setup) > 1e-3


def test_flipped_field_derivative_is_caught(monkeypatch):
    """dH_w/dphi with the wrong sign, against the central difference of H_w in phi."""
    dims, bc, phase, h = (2, 2, 2, 4), (0, 1, 1, 0), 0.3, 1e-5
    U = synth.random_su3_field(dims, 0.4, 2)
    x = synth.gaussian_spinor(dims, 1, 3)[0]
    fd = (dirac.hermitian_wilson(U, x, -1.5, bc, phase + h) - dirac.hermitian_wilson(U, x, -1.5, bc, phase - h)) / (2 * h)
    good = derivative.dhw_dphi(U, x, bc, phase)
    assert np.linalg.norm(good - fd) < 1e-6 * np.linalg.norm(fd)
    orig = derivative.dwilson_dphi
    monkeypatch.setattr(derivative, "dwilson_dphi", lambda *a, **k: -orig(*a, **k))
    assert np.linalg.norm(derivative.dhw_dphi(U, x, bc, phase) - fd) > 0.5 * np.linalg.norm(fd)


def test_derivative_without_chain_factor_is_caught(monkeypatch):
    """dq/dtheta = P + theta^2 P' (the chain-rule factor 2 of d(theta^2) dropped)."""
    def bad(theta, coeffs, eps):
        dc = np.polynomial.chebyshev.chebder(coeffs) * (2.0 / (1.0 - eps))
        x = theta ** 2
        return chebyshev.eval_poly(coeffs, eps, x) + x * np.polynomial.chebyshev.chebval(chebyshev.to_y(x, eps), dc)

    monkeypatch.setattr(derivative, "q_derivative", bad)
    assert dpins.split_derivative_error(0) > 1e-3
