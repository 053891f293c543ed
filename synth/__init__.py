"""Seeded synthetic inputs for the overlap-operator library and its oracle.

This module is the only code shared by the CPU oracle (``oracle/``) and the
CUDA path's tests and benchmark.  It holds none of the method's arithmetic:
it draws random SU(3) gauge links, random spinors, point sources and random
gauge transformations, and returns them as numpy arrays in the library's ABI
layouts:

* lattice extents ``dims = (Lx, Ly, Lz, Lt)``; site index ``x`` fastest;
* gauge field  ``U[mu, t, z, y, x, a, b]``  complex128, ``mu = 0..3 <-> x,y,z,t``;
* spinor field ``psi[rhs, t, z, y, x, s, c]`` complex128 (4 spins, 3 colours).

The paper's gauge ensemble (nHYP-smeared 2+1-flavour domain-wall
configurations on 24^3 x 64, Sec. 4) is not available; random links
``U = exp(i eps H)`` with ``H = sum_a h_a lambda_a`` (Gell-Mann matrices,
``h_a ~ N(0,1)``) stand in for it.  Smaller ``eps`` gives smoother fields.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "site_shape",
    "volume",
    "gell_mann",
    "random_su3_field",
    "random_gauge_transform",
    "gaussian_spinor",
    "point_sources",
    "unit_gauge",
]


def site_shape(dims):
    """Array shape of the site index for extents (Lx, Ly, Lz, Lt): (Lt, Lz, Ly, Lx)."""
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def volume(dims):
    v = 1
    for d in dims:
        v *= int(d)
    return v


def gell_mann():
    """The eight Gell-Mann matrices, normalised to tr(l_a l_b) = 2 delta_ab."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def _exp_i_hermitian(h, eps):
    """exp(i eps h) for a batch of Hermitian 3x3 matrices, by eigendecomposition."""
    w, v = np.linalg.eigh(h)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ik,...k,...jk->...ij", v, ph, v.conj())


def _random_su3(rng, shape, eps):
    h = rng.standard_normal(shape + (8,))
    lam = gell_mann()
    H = np.einsum("...a,aij->...ij", h, lam)
    return _exp_i_hermitian(H, eps)


def random_su3_field(dims, eps, seed=0):
    """Gauge field U[4, Lt, Lz, Ly, Lx, 3, 3] of random SU(3) links exp(i eps H)."""
    rng = np.random.default_rng(seed)
    return _random_su3(rng, (4,) + site_shape(dims), eps)


def unit_gauge(dims):
    """The free field: every link is the 3x3 identity."""
    U = np.zeros((4,) + site_shape(dims) + (3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def random_gauge_transform(dims, seed=7, eps=1.0):
    """One random SU(3) matrix per site, g[Lt, Lz, Ly, Lx, 3, 3]."""
    rng = np.random.default_rng(seed)
    return _random_su3(rng, site_shape(dims), eps)


def gaussian_spinor(dims, nrhs=1, seed=1, normalise=True):
    """Complex Gaussian spinors psi[nrhs, Lt, Lz, Ly, Lx, 4, 3]; each of unit norm."""
    rng = np.random.default_rng(seed)
    shape = (nrhs,) + site_shape(dims) + (4, 3)
    psi = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    if normalise:
        n = np.sqrt(np.sum(np.abs(psi) ** 2, axis=tuple(range(1, psi.ndim)), keepdims=True))
        psi = psi / n
    return psi


def point_sources(dims, spins_colours=None, site=(0, 0, 0, 0)):
    """Unit point sources delta(n, site) e_{s,c}; default: all 12 (s, c), rhs = 3 s + c.

    ``site`` is given as (x, y, z, t).
    """
    if spins_colours is None:
        spins_colours = [(s, c) for s in range(4) for c in range(3)]
    x, y, z, t = site
    psi = np.zeros((len(spins_colours),) + site_shape(dims) + (4, 3), dtype=np.complex128)
    for j, (s, c) in enumerate(spins_colours):
        psi[j, t, z, y, x, s, c] = 1.0
    return psi
