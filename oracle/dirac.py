"""Wilson Dirac operator D_w and H_w = gamma5 D_w (oracle, FP64).

Paper, Sec. 2 (eq. 1 and the sentence after it): H_w is gamma5 times the
Wilson Dirac operator.  The paper does not give the convention; this oracle
uses the standard one with Wilson parameter r = 1,

    D_w psi(n) = (4 + m0) psi(n)
                 - 1/2 sum_mu [ (1 - gamma_mu) U_mu(n)        psi(n + mu)
                              + (1 + gamma_mu) U_mu(n - mu)^+ psi(n - mu) ],

in the Euclidean chiral basis gamma_k = [[0, -i s_k], [i s_k, 0]],
gamma_4 = [[0, 1], [1, 0]], gamma5 = gamma1 gamma2 gamma3 gamma4
= diag(1, 1, -1, -1).  Directions mu = 0..3 are x, y, z, t.

Boundary conditions (Sec. 4: Dirichlet in the field direction and in time)
are a factor per direction applied to every hop that crosses the lattice edge:
1 periodic, -1 antiperiodic, 0 Dirichlet.  The background field (Sec. 4,
U_mu -> exp(-i q A_mu) U_mu) enters as the phase exp(i phi t) on the x links,
phi = q E.

Fields use the ABI layouts of ``synth``: U[mu, t, z, y, x, a, b] and
psi[..., t, z, y, x, spin, colour] with any number of leading axes.
"""
from __future__ import annotations

import numpy as np

_S1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_S2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_S3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)

#: gamma_mu for mu = x, y, z, t (Euclidean chiral basis).
GAMMA = np.array(
    [np.block([[_Z2, -1j * s], [1j * s, _Z2]]) for s in (_S1, _S2, _S3)]
    + [np.block([[_Z2, _I2], [_I2, _Z2]])]
)
#: gamma5 = gamma1 gamma2 gamma3 gamma4.
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ID4 = np.eye(4, dtype=np.complex128)

BC_FACTOR = {"periodic": 1.0, "antiperiodic": -1.0, "dirichlet": 0.0}


def bc_factors(bc):
    """Boundary factor per direction from names or numbers."""
    return tuple(BC_FACTOR[b] if isinstance(b, str) else float(b) for b in bc)


def _site_axis(field_ndim, mu, trailing):
    """Axis of direction mu in an array whose last ``trailing`` axes are internal."""
    lead = field_ndim - trailing - 4
    return lead + 3 - mu


def spin_mult(m, psi):
    """(m psi) for a 4x4 spin matrix m acting on psi[..., spin, colour]."""
    return np.einsum("st,...tc->...sc", m, psi)


def colour_mult(u, psi):
    """(u psi) for colour matrices u[..., a, b] acting on psi[..., spin, b]."""
    return np.einsum("...ab,...sb->...sa", u, psi)


def colour_mult_dag(u, psi):
    """(u^+ psi) for colour matrices u[..., a, b]."""
    return np.einsum("...ba,...sb->...sa", u.conj(), psi)


def gamma5(psi):
    return spin_mult(GAMMA5, psi)


def link(U, mu, phase=0.0):
    """U_mu(n) including the background-field phase exp(i phase t) on x links."""
    u = U[mu]
    if mu == 0 and phase != 0.0:
        lt = u.shape[0]
        ph = np.exp(1j * phase * np.arange(lt))
        u = u * ph[:, None, None, None, None, None]
    return u


def backward_link(u, mu):
    """U_mu(n - mu) at every site n: the link that arrives at n from behind."""
    return np.roll(u, 1, axis=3 - mu)


def neighbour(psi, mu, direction, bc):
    """psi(n + direction*mu) with the boundary factor on hops across the edge.

    ``direction`` is +1 (forward) or -1 (backward).
    """
    ax = _site_axis(psi.ndim, mu, 2)
    shifted = np.roll(psi, -direction, axis=ax)
    if bc != 1.0:
        L = psi.shape[ax]
        edge = [slice(None)] * psi.ndim
        # forward: sites n_mu = L-1 fetched the wrapped value from n_mu = 0;
        # backward: sites n_mu = 0 fetched it from n_mu = L-1.
        edge[ax] = L - 1 if direction > 0 else 0
        shifted = shifted.copy()
        shifted[tuple(edge)] *= bc
    return shifted


def wilson(U, psi, m0, bc=(1, 1, 1, 1), phase=0.0):
    """D_w psi (Sec. 2; the Wilson operator in the convention stated above)."""
    bcf = bc_factors(bc)
    out = (4.0 + m0) * psi
    for mu in range(4):
        u = link(U, mu, phase)
        u_back = backward_link(u, mu)
        fwd = colour_mult(u, neighbour(psi, mu, +1, bcf[mu]))
        bwd = colour_mult_dag(u_back, neighbour(psi, mu, -1, bcf[mu]))
        out = out - 0.5 * (spin_mult(ID4 - GAMMA[mu], fwd) + spin_mult(ID4 + GAMMA[mu], bwd))
    return out


def hermitian_wilson(U, psi, m0, bc=(1, 1, 1, 1), phase=0.0):
    """H_w psi = gamma5 D_w psi (Sec. 2, text after eq. 1)."""
    return gamma5(wilson(U, psi, m0, bc, phase))


def inner(a, b):
    """<a, b> = sum conj(a) b over everything."""
    return np.vdot(a.ravel(), b.ravel())


def norm(a):
    return float(np.sqrt(np.real(inner(a, a))))
