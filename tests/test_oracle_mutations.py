"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins catch them.

Each case patches one piece of the oracle with a typical bug -- a sign, a
missing dagger, a shifted index, a dropped halving -- and asserts that the
corresponding pin measure in ``test_oracle_pins`` moves far outside its
tolerance.  This shows the pins can fail, not only that they pass.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import chebyshev, dirac
from oracle import overlap as ov

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
