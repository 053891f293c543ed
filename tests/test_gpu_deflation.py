"""CG deflation with the low modes of D_ov (Sec. 3.2) against the oracle.

The library's Lanczos gives the lowest eigenpairs of the chiral-sector operator
A0 = P_s [2 (1 + s F)] P_s, F the implemented sign function (exact small space plus
the polynomial); the dense reference is that matrix built from the oracle's spectral
form of F on a 4^4 lattice.  Deflated solves must reach the tolerance against the
oracle's operator and take fewer inner iterations than undeflated ones.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from oracle import dense, dirac
from oracle import overlap as ov

pytestmark = pytest.mark.gpu

M0 = -1.5
HW = 6.5
EPS4 = 0.002  # covers the 4^4 field's large-space spectrum (see test_gpu_parity)
DEGREE = 200


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


@pytest.fixture(scope="module")
def lat():
    """4^4 field, 8 exact H_w modes per phase (phases 0 and 0.2), the dense implemented sign."""
    dims, bc = (4, 4, 4, 4), (0, 0, 0, 1)
    U = synth.random_su3_field(dims, 0.3, 0)
    coeffs = ov.OverlapParams(m0=M0, hw_norm=HW, eps=EPS4, degree=DEGREE).coeffs
    out = dict(dims=dims, bc=bc, U=U, banks={}, F={})
    for phase in (0.0, 0.2):
        H = dense.hw_matrix(U, M0, (1.0, 1.0, 1.0, -1.0), phase)
        lam, W, lam_all, W_all = dense.low_modes(H, HW, 8)
        assert np.sort(np.abs(lam_all))[8] ** 2 > EPS4
        out["banks"][phase] = (lam, dense.vectors_to_fields(W, synth.site_shape(dims)))
        out["F"][phase] = dense.split_sign_matrix(lam_all, W_all, 8, coeffs, EPS4)
    return out


def sector_index(chi, nsite):
    spin = (np.arange(12 * nsite) // 3) % 4
    return np.nonzero(spin < 2 if chi > 0 else spin >= 2)[0]


def make_ctx(P, d, adaptive=0):
    ctx = P.Context(P.Params(dims=d["dims"], bc=d["bc"], m0=M0, eps=EPS4, poly_degree=DEGREE, precision=1,
                             inner_precision=1, max_nrhs=4, adaptive_order=adaptive))
    ctx.set_gauge(dev(d["U"]))
    for phase, (lam, V) in d["banks"].items():
        P.deflate(ctx, dev(V), lam, phase=phase)
    return ctx


@pytest.mark.parametrize("chi,phase", [(1, 0.0), (-1, 0.0), (1, 0.2)])
def test_overlap_low_modes_match_dense(P, lat, chi, phase):
    d = lat
    nsite = 256
    F = d["F"][phase]
    G5 = np.kron(np.eye(nsite), np.kron(dirac.GAMMA5, np.eye(3)))
    assert np.allclose(G5, G5.conj().T)
    idx = sector_index(chi, nsite)
    A0 = 2.0 * (np.eye(F.shape[0]) + chi * F)
    want = np.linalg.eigvalsh(A0[np.ix_(idx, idx)])[:8]
    ctx = make_ctx(P, d)
    theta, res = P.eigensolve_overlap(ctx, 8, chirality=chi, phase=phase, krylov=80)
    print(f"chi {chi:+d} phase {phase}: Ritz {theta[:4]} dense {want[:4]} residuals <= {res.max():.1e}")
    assert np.allclose(theta, want, atol=2e-5 * 4)
    assert res.max() < 1e-3
    ctx.close()


@pytest.mark.parametrize("mass,phase,adaptive", [(0.1, 0.0, 0), (0.02, 0.0, 1), (0.02, 0.2, 1)])
def test_deflated_solve_matches_oracle(P, lat, mass, phase, adaptive):
    import torch

    d, tol = lat, 1e-10
    b = synth.point_sources(d["dims"], [(0, 1), (3, 2)])
    phases = [phase, phase]
    iters = {}
    xs = {}
    for defl in (False, True):
        ctx = make_ctx(P, d, adaptive)
        if defl:
            for chi in (1, -1):
                P.eigensolve_overlap(ctx, 16, chirality=chi, phase=phase)
        xd = torch.zeros_like(dev(b))
        st = P.solve_overlap(ctx, dev(b), xd, mass, tol=tol, phase=phases)
        assert st.true_residual <= tol
        iters[defl] = st.inner_iters
        xs[defl] = xd.cpu().numpy()
        print(f"m {mass} phase {phase} deflated {defl}: {ctx.last_info}")
        ctx.close()
    lam, V = d["banks"][phase]
    small = ov.SmallSpace.from_eigenpairs(V, lam)
    p = ov.OverlapParams(m0=M0, hw_norm=HW, eps=EPS4, degree=DEGREE, bc=(1.0, 1.0, 1.0, -1.0))
    for j in range(2):
        r = b[j] - ov.overlap(d["U"], xs[True][j], mass, p, small, phase)
        assert np.linalg.norm(r) / np.linalg.norm(b[j]) <= 2 * tol
    assert iters[True] < iters[False]


@pytest.mark.parametrize("inner", ["f64", "f16", "bf16"])
def test_deflated_solve_in_other_inner_precisions(P, lat, inner):
    """The same deflated, adaptive-order solve with an FP64 inner CG (deflated with the spaces' FP64
    vectors) and with FP16 / BF16 storage of the inner CG's polynomial loops (FP32 arithmetic): each
    must reach the tolerance against the oracle's operator; the 16-bit ones take more outer cycles."""
    import torch

    d, tol, mass, phase = lat, 1e-10, 0.02, 0.2
    prec = {"f64": 0, "f16": 2, "bf16": 3}[inner]
    ctx = P.Context(P.Params(dims=d["dims"], bc=d["bc"], m0=M0, eps=EPS4, poly_degree=DEGREE,
                             precision=1 if inner == "f64" else prec, inner_precision=1, max_nrhs=4,
                             adaptive_order=1))
    ctx.set_gauge(dev(d["U"]))
    for ph, (lam, V) in d["banks"].items():
        P.deflate(ctx, dev(V), lam, phase=ph)
    for chi in (1, -1):
        P.eigensolve_overlap(ctx, 16, chirality=chi, phase=phase)
    ctx.set_inner_precision(prec)
    b = synth.point_sources(d["dims"], [(0, 1), (3, 2)])
    xd = torch.zeros_like(dev(b))
    st = P.solve_overlap(ctx, dev(b), xd, mass, tol=tol, phase=[phase, phase])
    print(f"inner {inner}: outer {st.outer_iters}, inner {st.inner_iters}: {ctx.last_info}")
    assert st.true_residual <= tol
    x = xd.cpu().numpy()
    lam, V = d["banks"][phase]
    small = ov.SmallSpace.from_eigenpairs(V, lam)
    p = ov.OverlapParams(m0=M0, hw_norm=HW, eps=EPS4, degree=DEGREE, bc=(1.0, 1.0, 1.0, -1.0))
    for j in range(2):
        r = b[j] - ov.overlap(d["U"], x[j], mass, p, small, phase)
        assert np.linalg.norm(r) / np.linalg.norm(b[j]) <= 2 * tol
    ctx.close()
