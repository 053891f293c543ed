"""Field derivatives and the pion correlator on the GPU against the oracle.

dH_w/dphi and dD(m)/dphi (through the small space and the polynomial) against
the oracle's stencil and its dense Daleckii-Krein derivative; the correlator
and timeslice inner products against numpy; dC(t)/dE from the autograd
function and from the tangent solve against the oracle's central finite
difference in E with the eigen-split recomputed at E +- h.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from oracle import correlator as ocorr
from oracle import dense, derivative, dirac
from oracle import overlap as ov

pytestmark = pytest.mark.gpu

M0 = -1.5
BC_NUM = {0: 1.0, 1: -1.0, 2: 0.0}


def obc(bc):
    return tuple(BC_NUM[b] for b in bc)


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1111_6288_gb300 as P

    return P


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def relerr(got, want):
    return float(np.abs(got - want).max() / np.abs(want).max())


@pytest.mark.parametrize("dims,bc,phases", [((6, 4, 3, 6), (2, 0, 0, 2), [0.4, 0.0]), ((4, 4, 4, 4), (0, 0, 0, 1), [0.1])])
def test_dhw_dphi_matches_oracle(P, dims, bc, phases):
    import torch

    U = synth.random_su3_field(dims, 0.4, 3)
    x = synth.gaussian_spinor(dims, len(phases), 4)
    ctx = P.Context(P.Params(dims=dims, bc=bc, m0=M0, eps=0.01, poly_degree=8, max_nrhs=4))
    ctx.set_gauge(dev(U))
    out = torch.empty_like(dev(x))
    P.apply_dHdphi(ctx, dev(x), out, phase=phases)
    got = out.cpu().numpy()
    want = np.stack([derivative.dhw_dphi(U, x[j], obc(bc), phases[j]) for j in range(len(phases))])
    assert relerr(got, want) < 1e-12
    ctx.close()


def small_problem(dims, bc, phase, n_ev, degree, seed=0):
    """Dense spectrum of a small lattice and parameters whose interval covers the large space."""
    U = synth.random_su3_field(dims, 0.3, seed)
    H = dense.hw_matrix(U, M0, obc(bc), phase)
    hw = 6.5
    lam_all, W_all = np.linalg.eigh(H)
    th = np.sort(np.abs(lam_all / hw))
    eps = (0.9 * th[n_ev]) ** 2
    lam, W, _, _ = dense.low_modes(H, hw, n_ev)
    V = dense.vectors_to_fields(W, synth.site_shape(dims))
    site = synth.site_shape(dims) + (4, 3)
    dH = dense.operator_matrix(lambda v: derivative.dhw_dphi(U, v, obc(bc), phase), site)
    return U, H, dH, hw, eps, lam, V


# Degree 700 keeps the polynomial error delta near 1e-13 on this field's interval: the
# small-to-large-space block of the derivative uses sign(l) for q(l), which costs delta/gap.
# n_ev = 5 puts the cut in a gap (|t| 0.0201 | 0.0224); 6 would split a near-degenerate pair.
@pytest.mark.parametrize("n_ev", [0, 5])
def test_dDdphi_matches_dense_daleckii_krein(P, n_ev):
    import torch

    dims, bc, phase, degree, mass = (4, 2, 2, 4), (2, 0, 0, 2), 0.3, 700, 0.1
    U, H, dH, hw, eps, lam, V = small_problem(dims, bc, phase, n_ev, degree)
    coeffs = ov.OverlapParams(m0=M0, hw_norm=hw, eps=eps, degree=degree).coeffs
    dF = derivative.split_sign_derivative(H, dH, hw, n_ev, coeffs, eps)
    ctx = P.Context(P.Params(dims=dims, bc=bc, m0=M0, eps=eps, poly_degree=degree, max_nrhs=4))
    ctx.set_gauge(dev(U))
    if n_ev:
        P.deflate(ctx, dev(V), lam, phase=phase)
    else:
        P.deflate(ctx, None, [], phase=phase)  # an empty small space for this field value
    x = synth.gaussian_spinor(dims, 2, 7)
    out = torch.empty_like(dev(x))
    P.apply_dDdphi(ctx, dev(x), out, mass, phase=[phase, phase])
    got = out.cpu().numpy()
    for j in range(2):
        want = (1 - mass / 2) * dirac.gamma5((dF @ x[j].ravel()).reshape(x[j].shape))
        # the low-high block drops same-sign divided differences of size delta / gap
        assert relerr(got[j], want) < 1e-8
    ctx.close()


def test_correlator_and_inner_products(P):
    import torch

    dims = (4, 4, 2, 6)
    S = synth.gaussian_spinor(dims, 3, 11, normalise=False)
    T = synth.gaussian_spinor(dims, 3, 12, normalise=False)
    ctx = P.Context(P.Params(dims=dims, eps=0.01, poly_degree=4, max_nrhs=4))
    C = P.correlator(ctx, dev(S))
    assert np.allclose(C, ocorr.pion_correlator(S), rtol=1e-13)
    ip = P.inner(ctx, dev(S), dev(T), per_timeslice=True)
    want = np.einsum("jtzyxsc,jtzyxsc->jt", S.conj(), T)
    assert np.allclose(ip, want, rtol=1e-12, atol=1e-12)
    ip1 = P.inner(ctx, dev(S), dev(T))
    assert np.allclose(ip1, want.sum(axis=1), rtol=1e-12)
    ctx.close()


def oracle_correlator(U, bc, hw, eps, degree, n_ev, mass, phase, sources):
    """C(t) from dense solves with the eigen-split recomputed at this phase."""
    site = synth.site_shape(U.shape[1:5][::-1])
    H = dense.hw_matrix(U, M0, obc(bc), phase)
    lam_all, W_all = np.linalg.eigh(H)
    coeffs = ov.OverlapParams(m0=M0, hw_norm=hw, eps=eps, degree=degree).coeffs
    F = dense.split_sign_matrix(lam_all / hw, W_all, n_ev, coeffs, eps)
    G5 = np.kron(np.eye(int(np.prod(site))), np.kron(dirac.GAMMA5, np.eye(3)))
    D = (1 - mass / 2) * (np.eye(F.shape[0]) + G5 @ F) + mass * np.eye(F.shape[0])
    S = np.linalg.solve(D, sources.reshape(len(sources), -1).T).T.reshape(sources.shape)
    return ocorr.pion_correlator(S)


def test_dC_dE_matches_oracle_finite_difference(P):
    import torch

    dims, bc, degree, mass, n_ev = (4, 2, 2, 4), (2, 0, 0, 2), 700, 0.1, 5
    charge, E = 2.0 / 3.0, 0.2
    phase = charge * E
    U, H, dH, hw, eps, lam, V = small_problem(dims, bc, phase, n_ev, degree)
    sources = synth.point_sources(dims, site=(1, 0, 1, 1))
    h = 1e-5
    Cp = oracle_correlator(U, bc, hw, eps, degree, n_ev, mass, charge * (E + h), sources)
    Cm = oracle_correlator(U, bc, hw, eps, degree, n_ev, mass, charge * (E - h), sources)
    fd = (Cp - Cm) / (2 * h)
    C0 = oracle_correlator(U, bc, hw, eps, degree, n_ev, mass, phase, sources)

    ctx = P.Context(P.Params(dims=dims, bc=bc, m0=M0, eps=eps, poly_degree=degree, max_nrhs=12))
    ctx.set_gauge(dev(U))
    P.deflate(ctx, dev(V), lam, phase=phase)
    src = dev(sources)
    C, dC = P.correlator_jacobian(ctx, src, E, charge, mass, tol=1e-13)
    assert relerr(C, C0) < 1e-10
    assert relerr(dC, fd) < 1e-5
    # the autograd function: gradient of a weighted sum of the correlator
    g = np.linspace(0.5, 2.0, dims[3])
    Et = torch.tensor(E, dtype=torch.float64, requires_grad=True)
    Ct = P.pion_correlator(Et, ctx, src, charge, mass, tol=1e-13)
    assert relerr(Ct.detach().numpy(), C0) < 1e-10
    (Ct * torch.from_numpy(g)).sum().backward()
    want = float(np.dot(g, fd))
    assert abs(Et.grad.item() - want) < 1e-5 * abs(want)
    ctx.close()


def test_dC_dE_config4_shape_against_library_finite_difference(P):
    """The background-field configuration's derivative at a size the test suite affords: 8 x 4 x 4 x 8,
    Dirichlet x and t, 16 eigenvectors of Q per phase from the library's eigensolver (recomputed at
    E +- h), the minimax polynomial n = 527 on [4e-4, 1], m = 0.02, the 12 point sources, q = 2/3,
    E = 1e-4: dC/dE from the tangent solve (ov_dcorr_dE) against the central difference of C at
    E +- 1e-5 from FP64-accurate solves (1e-13), to 1e-5 of the largest |dC/dE|.  (The library's FP64
    operator and solve are pinned against the oracle at small size by the other tests; the full-size
    case runs as bench.py --derivative-case.)"""
    import torch

    dims, bc, mass, charge, E, h = (8, 4, 4, 8), (2, 0, 0, 2), 0.02, 2.0 / 3.0, 1e-4, 1e-5
    U = dev(synth.random_su3_field(dims, 0.2, 0))
    ctx = P.Context(P.Params(dims=dims, bc=bc, m0=M0, eps=4e-4, poly_degree=527, poly_kind=1, precision=0,
                             inner_precision=1, max_nrhs=12, adaptive_order=1))
    ctx.set_gauge(U)
    for e in (E, E + h, E - h):
        P.eigensolve_Q(ctx, 16, phase=charge * e, tol=1e-11, max_iter=300)
    src = dev(synth.point_sources(dims, site=(4, 0, 0, 4)))
    C0, dC = P.correlator_jacobian(ctx, src, E, charge, mass, tol=1e-13)
    Cs = {}
    for e in (E + h, E - h):
        x = torch.zeros_like(src)
        P.solve_overlap(ctx, src, x, mass, tol=1e-13, phase=[charge * e] * 12)
        Cs[e] = P.correlator(ctx, x)
    fd = (Cs[E + h] - Cs[E - h]) / (2 * h)
    err = float(np.abs(dC - fd).max() / np.abs(fd).max())
    print(f"config-4 shape: dC/dE vs FD {err:.2e}, max |dC/dE| {np.abs(dC).max():.3e}")
    assert err < 1e-5
    ctx.close()
