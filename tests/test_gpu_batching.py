"""Batching of right-hand sides (spin-colour sources x field values).

A batch runs the same per-thread arithmetic as the same right-hand sides one
at a time (the Wilson kernel's right-hand-side block only changes which
threads share a block), so batched operator applications and solves must equal
the one-at-a-time results exactly.  A 12-source, two-field solve with the
library's own eigensolver banks checks the multi-phase path end to end.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from oracle import dense
from oracle import overlap as ov

pytestmark = pytest.mark.gpu
M0 = -1.5


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
def setup(P):
    dims, bc = (6, 4, 4, 6), (2, 0, 0, 2)
    U = synth.random_su3_field(dims, 0.3, 8)
    site = synth.site_shape(dims)
    rng = np.random.default_rng(3)
    banks = {}
    for phase, nev in [(0.0, 4), (0.2, 6)]:
        A = rng.standard_normal((12 * 576, nev)) + 1j * rng.standard_normal((12 * 576, nev))
        Qm, _ = np.linalg.qr(A)
        banks[phase] = (dense.vectors_to_fields(Qm, site), rng.standard_normal(nev))
    return dims, bc, U, banks


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_overlap_equals_one_at_a_time(P, setup, precision):
    import torch

    dims, bc, U, banks = setup
    ctx = P.Context(P.Params(dims=dims, bc=bc, m0=M0, eps=0.02, poly_degree=40, precision=precision, max_nrhs=8))
    ctx.set_gauge(dev(U))
    for phase, (V, lam) in banks.items():
        P.deflate(ctx, dev(V), lam, phase=phase)
    phases = [0.0, 0.2, 0.2, 0.0, 0.2, 0.0, 0.0]
    x = dev(synth.gaussian_spinor(dims, len(phases), 5)).to(ctx.spinor_dtype())
    yb = torch.empty_like(x)
    P.apply_overlap(ctx, x, yb, mass=0.05, phase=phases)
    for j, ph in enumerate(phases):
        y1 = torch.empty_like(x[j:j + 1])
        P.apply_overlap(ctx, x[j:j + 1].contiguous(), y1, mass=0.05, phase=[ph])
        assert torch.equal(y1[0], yb[j])
    assert ctx.tune_info  # the right-hand-side block was tuned for this batch
    ctx.close()


def test_batched_solve_equals_one_at_a_time(P, setup):
    """The solver needs real eigenvectors in its banks (the chiral-sector inner operator
    assumes sign^2 = 1): they come from the library's eigensolver here."""
    import torch

    dims, bc, U, _ = setup
    ctx = P.Context(P.Params(dims=dims, bc=bc, m0=M0, eps=1e-3, poly_degree=150, precision=1, inner_precision=1,
                             max_nrhs=8))
    ctx.set_gauge(dev(U))
    for phase in (0.0, 0.2):
        P.eigensolve_Q(ctx, 6, phase=phase, tol=1e-11, max_iter=300)
    phases = [0.2, 0.0, 0.2]
    b = dev(synth.point_sources(dims, [(0, 0), (2, 1), (3, 2)], site=(1, 2, 0, 3)))
    xb = torch.zeros_like(b)
    st = P.solve_overlap(ctx, b, xb, 0.1, tol=1e-10, phase=phases)
    assert st.true_residual <= 1e-10
    for j, ph in enumerate(phases):
        x1 = torch.zeros_like(b[j:j + 1])
        P.solve_overlap(ctx, b[j:j + 1].contiguous(), x1, 0.1, tol=1e-10, phase=[ph])
        # the batch keeps iterating until every right-hand side converges, so a right-hand
        # side can take one more outer cycle than alone: compare to the solve tolerance
        rel = (x1[0] - xb[j]).norm() / x1[0].norm()
        assert float(rel) < 1e-8
    ctx.close()


def test_twelve_sources_two_fields_with_library_banks(P):
    import torch

    dims, bc, mass = (8, 8, 8, 8), (2, 0, 0, 2), 0.05
    U = dev(synth.random_su3_field(dims, 0.2, 0))
    ctx = P.Context(P.Params(dims=dims, bc=bc, m0=M0, eps=0.002, poly_degree=200, precision=1, inner_precision=1,
                             max_nrhs=24))
    ctx.set_gauge(U)
    phases = []
    for phase in [0.0, 2.0 / 3.0 * 0.01]:
        lam, _ = P.eigensolve_Q(ctx, 8, phase=phase, tol=1e-10, max_iter=300)
        phases += [phase] * 12
    b = dev(np.concatenate([synth.point_sources(dims)] * 2))
    x = torch.zeros_like(b)
    st = P.solve_overlap(ctx, b, x, mass, tol=1e-10, phase=phases)
    assert st.status == 0 and st.true_residual <= 1e-10
    # residual of two columns with the library's FP64 operator (independent apply)
    ctx64 = P.Context(P.Params(dims=dims, bc=bc, m0=M0, eps=0.002, poly_degree=200, max_nrhs=2))
    ctx64.set_gauge(U)
    for phase in [0.0, 2.0 / 3.0 * 0.01]:
        lam, V = P.eigensolve_Q(ctx, 8, phase=phase, tol=1e-10, max_iter=300, register=False, want_vectors=True)
        P.deflate(ctx64, V, lam, phase=phase)
    for j in (0, 17):
        r = torch.empty_like(x[j:j + 1])
        P.apply_overlap(ctx64, x[j:j + 1].contiguous(), r, mass=mass, phase=[phases[j]])
        rel = (b[j] - r[0]).norm() / b[j].norm()
        assert float(rel) <= 2e-10
    ctx.close()
    ctx64.close()


@pytest.fixture(scope="module")
def config3_small():
    """The batched configuration's shape on 4 x 4 x 2 x 4: Dirichlet x and t, two field values, the 12
    lowest |lambda| eigenvectors of Q per field value from the oracle's dense spectrum, and an interval
    [eps, 1] that holds the rest of both spectra.  (With m0 = -1.5 the Dirichlet faces carry near-zero
    surface modes of H_w, |lambda|/||H_w|| from 4e-3 up, so the small space must take a dozen of them.)"""
    dims, bc = (4, 4, 2, 4), (2, 0, 0, 2)
    obc = (0.0, 1.0, 1.0, 0.0)
    U = synth.random_su3_field(dims, 0.3, 0)
    hw, n_ev = 6.5, 12
    banks, cut = {}, []
    for phase in (0.0, 0.3):
        H = dense.hw_matrix(U, M0, obc, phase)
        lam, W, lam_all, _ = dense.low_modes(H, hw, n_ev)
        banks[phase] = (lam, dense.vectors_to_fields(W, synth.site_shape(dims)))
        cut.append(np.sort(np.abs(lam_all))[n_ev])
    eps = (0.9 * min(cut)) ** 2
    return dict(dims=dims, bc=bc, obc=obc, U=U, hw=hw, banks=banks, eps=eps)


@pytest.mark.parametrize("inner", ["f32", "f16"])
def test_config3_shape_batched_solve_against_oracle(P, config3_small, inner):
    """12 spin-colour point sources x 2 field values in one solve_overlap call (24 right-hand sides;
    48 chiral systems in the inner CG, 24 per bank, so the small-space projection may take the
    tensor cores), adaptive order, FP32 or FP16-stored inner CG; every column's residual is taken
    with the oracle's D(m) and must meet the tolerance."""
    import torch

    d, mass, tol, degree = config3_small, 0.02, 1e-10, 300
    prec = {"f32": P.OV_PREC_F32, "f16": P.OV_PREC_F16}[inner]
    ctx = P.Context(P.Params(dims=d["dims"], bc=d["bc"], m0=M0, eps=d["eps"], poly_degree=degree, precision=prec,
                             inner_precision=prec, max_nrhs=24, adaptive_order=1))
    ctx.set_gauge(dev(d["U"]))
    phases = []
    for phase, (lam, V) in d["banks"].items():
        P.deflate(ctx, dev(V), lam, phase=phase)
        phases += [phase] * 12
    b = np.concatenate([synth.point_sources(d["dims"])] * 2)
    x = torch.zeros_like(dev(b))
    st = P.solve_overlap(ctx, dev(b), x, mass, tol=tol, phase=phases)
    print(f"{inner}: {st.outer_iters} outer, {st.inner_iters} inner; {ctx.last_info}; {ctx.tune_info}")
    assert st.status == 0 and st.true_residual <= tol
    xs = x.cpu().numpy()
    for j in range(24):
        lam, V = d["banks"][phases[j]]
        p = ov.OverlapParams(m0=M0, hw_norm=d["hw"], eps=d["eps"], degree=degree, bc=d["obc"])
        r = b[j] - ov.overlap(d["U"], xs[j], mass, p, ov.SmallSpace.from_eigenpairs(V, lam), phases[j])
        assert np.linalg.norm(r) / np.linalg.norm(b[j]) <= 2 * tol, j
    ctx.close()


@pytest.fixture(scope="module")
def config5_small():
    """The largest configuration's parameters on 4 x 4 x 2 x 4: links exp(i 0.15 H), Dirichlet x and
    t, sqrt(eps) = 0.01 and the minimax polynomial of degree 1054 (delta 1.2e-10), the five field
    phases 0, +-(2/3) E, +-(1/3) E of the up and down quark charges (E = 0.3 here, so that the
    phases matter on four time slices), and per phase the 12 lowest |lambda| eigenvectors of Q from
    the oracle's dense spectrum (the surface modes, |lambda| from 4.2e-3 to 0.035; the rest of each
    spectrum lies above 0.045, inside [sqrt(eps), 1])."""
    from oracle import chebyshev

    dims, bc = (4, 4, 2, 4), (2, 0, 0, 2)
    obc = (0.0, 1.0, 1.0, 0.0)
    U = synth.random_su3_field(dims, 0.15, 0)
    hw, n_ev, eps, degree = 6.5, 12, 1e-4, 1054
    banks = {}
    for phase in (0.0, 0.2, -0.2, 0.1, -0.1):
        lam, W, lam_all, _ = dense.low_modes(dense.hw_matrix(U, M0, obc, phase), hw, n_ev)
        assert np.sort(np.abs(lam_all))[n_ev] > np.sqrt(eps)
        banks[phase] = (lam, dense.vectors_to_fields(W, synth.site_shape(dims)))
    coeffs, delta = chebyshev.minimax_coeffs(degree, eps)
    return dict(dims=dims, bc=bc, obc=obc, U=U, hw=hw, banks=banks, eps=eps, degree=degree, coeffs=coeffs,
                delta=delta)


def test_config5_shape_batched_solve_against_oracle(P, config5_small):
    """12 spin-colour point sources x 5 field phases in one solve_overlap call (60 right-hand sides,
    120 chiral systems), m = 0.01, tol 1e-10, the degree-1054 minimax polynomial on [1e-4, 1],
    adaptive order, FP32 inner CG.  The library's FP64 residual of every column meets the tolerance;
    two columns per phase (spin-colour 0 and 11) are checked with the oracle's D(m), each about 2100
    oracle Wilson applications."""
    import torch

    d, mass, tol = config5_small, 0.01, 1e-10
    assert d["delta"] < 2e-10
    ctx = P.Context(P.Params(dims=d["dims"], bc=d["bc"], m0=M0, eps=d["eps"], poly_degree=d["degree"],
                             poly_kind=1, precision=P.OV_PREC_F32, inner_precision=P.OV_PREC_F32, max_nrhs=60,
                             adaptive_order=1))
    ctx.set_gauge(dev(d["U"]))
    phases = []
    for phase, (lam, V) in d["banks"].items():
        P.deflate(ctx, dev(V), lam, phase=phase)
        phases += [phase] * 12
    b = np.concatenate([synth.point_sources(d["dims"])] * 5)
    x = torch.zeros_like(dev(b))
    st = P.solve_overlap(ctx, dev(b), x, mass, tol=tol, phase=phases)
    print(f"{st.outer_iters} outer, {st.inner_iters} inner; {ctx.last_info}")
    assert st.status == 0 and st.true_residual <= tol
    xs = x.cpu().numpy()
    p = ov.OverlapParams(m0=M0, hw_norm=d["hw"], eps=d["eps"], degree=d["degree"], bc=d["obc"], coeffs=d["coeffs"])
    for j in [k for ph in range(5) for k in (12 * ph, 12 * ph + 11)]:
        lam, V = d["banks"][phases[j]]
        r = b[j] - ov.overlap(d["U"], xs[j], mass, p, ov.SmallSpace.from_eigenpairs(V, lam), phases[j])
        assert np.linalg.norm(r) / np.linalg.norm(b[j]) <= 2 * tol, j
    ctx.close()
