"""16-bit storage (FP16 with a per-site scale, BF16) against the FP64 oracle.

Links and the vectors of the Chebyshev recurrence are stored in 16 bits and
computed in FP32; the small-space projection and the final H_w application are
FP32.  Each test states the error it measures (printed) and holds it to a bound
in units of the format's unit roundoff u (FP16: 2^-11, its 11-bit significand on
the per-site-scaled numbers; BF16: 2^-8):

* one Wilson application: the input, the two stored link rows (the third row is
  rebuilt from them) and the output are each rounded once, and every output
  component sums O(10) rounded terms of O(1): 16 u bounds the max-relative error
  (measured ~0.6 u for FP16, ~0.9 u for BF16 in a dense CPU emulation of the
  same formats);
* sign(H_w) at degree 200: every recurrence vector is rounded at each of the 400
  steps and the Clenshaw recurrence carries these errors to the result; the dense
  emulation gives 4 u (FP16) and 5 u (BF16) on the case below, and 40 u bounds
  it.  A format error (wrong scale, wrong plane) gives errors of O(1).
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from oracle import dense, dirac
from oracle import overlap as ov

pytestmark = pytest.mark.gpu

M0 = -1.5
BC_NUM = {0: 1.0, 1: -1.0, 2: 0.0}
U16 = {2: 2.0 ** -11, 3: 2.0 ** -8}  # unit roundoff of OV_PREC_F16, OV_PREC_BF16
NAME = {2: "FP16", 3: "BF16"}
EPS4 = 0.002  # covers the large-space spectrum of the 4^4 field below (smallest |Q|^2 > 0.002)


def obc(bc):
    return tuple(BC_NUM[b] for b in bc)


def relerr(got, want):
    return float(np.abs(got - want).max() / np.abs(want).max())


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1111_6288_gb300 as P

    return P


def dev(a, dtype=None):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


def ctx_for(P, dims, bc, precision, degree=30, eps=0.01, max_nrhs=8):
    return P.Context(P.Params(dims=dims, bc=bc, m0=M0, eps=eps, poly_degree=degree, precision=precision,
                              inner_precision=1, max_nrhs=max_nrhs))


def run(P, ctx, fn, x, **kw):
    import torch

    xd = dev(x, torch.complex64)
    out = torch.empty_like(xd)
    fn(ctx, xd, out, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("precision", [2, 3])
@pytest.mark.parametrize("dims,bc,phases", [((4, 4, 4, 4), (0, 0, 0, 1), [0.0, 0.3]),
                                             ((6, 4, 3, 6), (2, 0, 0, 2), [0.4, -0.2, 0.0])])
def test_wilson_16bit_error_is_stated(P, precision, dims, bc, phases):
    U = synth.random_su3_field(dims, 0.4, 11)
    x = synth.gaussian_spinor(dims, len(phases), 12)
    ctx = ctx_for(P, dims, bc, precision)
    ctx.set_gauge(dev(U))
    for herm in (False, True):
        got = run(P, ctx, P.apply_wilson, x, phase=phases, hermitian=herm)
        f = dirac.hermitian_wilson if herm else dirac.wilson
        want = np.stack([f(U, x[j], M0, obc(bc), phases[j]) for j in range(len(phases))])
        err = relerr(got, want)
        print(f"{NAME[precision]} {'H_w' if herm else 'D_w'} {dims}: max-relative error {err:.2e} "
              f"({err / U16[precision]:.2f} u)")
        assert err < 16 * U16[precision]
    ctx.close()


@pytest.fixture(scope="module")
def lat4():
    dims, bc = (4, 4, 4, 4), (0, 0, 0, 1)
    U = synth.random_su3_field(dims, 0.3, 0)
    H = dense.hw_matrix(U, M0, obc(bc))
    lam, W, lam_all, _ = dense.low_modes(H, 6.5, 8)
    assert np.sort(np.abs(lam_all))[0] ** 2 > EPS4  # low_modes returns eigenvalues of Q
    return dict(dims=dims, bc=bc, U=U, lam=lam, V=dense.vectors_to_fields(W, synth.site_shape(dims)))


@pytest.mark.parametrize("precision", [2, 3])
def test_sign_16bit_error_is_stated(P, lat4, precision):
    d, degree = lat4, 200
    ctx = ctx_for(P, d["dims"], d["bc"], precision, degree=degree, eps=EPS4)
    ctx.set_gauge(dev(d["U"]))
    P.deflate(ctx, dev(d["V"]), d["lam"])
    x = synth.gaussian_spinor(d["dims"], 1, 5)
    got = run(P, ctx, P.apply_sign_Hw, x)
    p = ov.OverlapParams(m0=M0, hw_norm=6.5, eps=EPS4, degree=degree, bc=obc(d["bc"]))
    want = ov.sign_hw(d["U"], x[0], p, ov.SmallSpace.from_eigenpairs(d["V"], d["lam"]))
    err = relerr(got[0], want)
    print(f"{NAME[precision]} sign(H_w), n = {degree}: max-relative error {err:.2e} ({err / U16[precision]:.1f} u)")
    assert err < 40 * U16[precision]
    ctx.close()


@pytest.mark.parametrize("precision", [2, 3])
def test_overlap_16bit_with_field_and_batch(P, precision):
    """D(m) at two field phases, Dirichlet x and t, each phase with its own 6 exact low modes
    and an interval covering the rest of its spectrum: every system against the oracle, and
    the batch equal bit for bit to one system at a time."""
    dims, bc, n_ev, degree, mass = (4, 4, 4, 4), (2, 0, 0, 2), 6, 100, 0.05
    U = synth.random_su3_field(dims, 0.3, 21)
    site = synth.site_shape(dims)
    modes, eps = {}, 1.0
    for phase in (0.0, 0.25):
        H = dense.hw_matrix(U, M0, obc(bc), phase)
        lam, W, lam_all, _ = dense.low_modes(H, 6.5, n_ev)
        modes[phase] = (lam, dense.vectors_to_fields(W, site))
        eps = min(eps, (0.9 * np.sort(np.abs(lam_all))[n_ev]) ** 2)
    ctx = ctx_for(P, dims, bc, precision, degree=degree, eps=eps)
    ctx.set_gauge(dev(U))
    for phase, (lam, V) in modes.items():
        P.deflate(ctx, dev(V), lam, phase=phase)
    phases = [0.25, 0.0, 0.25]
    x = synth.gaussian_spinor(dims, 3, 23)
    got = run(P, ctx, P.apply_overlap, x, mass=mass, phase=phases)
    p = ov.OverlapParams(m0=M0, hw_norm=6.5, eps=eps, degree=degree, bc=obc(bc))
    for j in range(3):
        lam, V = modes[phases[j]]
        want = ov.overlap(U, x[j], mass, p, ov.SmallSpace.from_eigenpairs(V, lam), phases[j])
        err = relerr(got[j], want)
        print(f"{NAME[precision]} D(m) phase {phases[j]}: max-relative error {err:.2e} ({err / U16[precision]:.1f} u)")
        assert err < 40 * U16[precision]
        one = run(P, ctx, P.apply_overlap, x[j:j + 1], mass=mass, phase=[phases[j]])
        assert np.array_equal(one[0], got[j])
    ctx.close()
