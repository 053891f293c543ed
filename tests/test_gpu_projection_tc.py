"""The small-space projection (Sec. 2, Fig. 1) on the tensor cores and on the CUDA cores, against the
oracle, through the C ABI (ov_project_small).

The tcgen05 path computes C = V^+ X by a split-K TF32 GEMM with the three-term (hi/lo) split and
X - V C, V diag(s) C by a second TF32 GEMM; both must be as accurate as the FP32 CUDA-core path.
The cases span ragged contractions (24 V floats not a multiple of the 32-float K-tile), ragged
output tiles (12 V complex positions not a multiple of 128), banks that are not a multiple of 16 or
exceed one 128-row tile, and batches of 8, 13, 27 and 40 vectors (the last in two groups).

Tolerance: the inputs and the FP32 bank carry FP32 rounding (6e-8 relative); C sums about 24 V
products.  The three-term TF32 split represents each operand to 2^-22 and drops the lo x lo product
(2^-22), about 7e-7 per product against 6e-8 for FP32, and X - V C, V s C sum 2N such products: the
largest error then reaches a few times 1e-6 of the largest output component (3e-6 measured at
N = 130) where plain FP32 on the CUDA cores stays near 4e-7.  5e-6 bounds both.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from oracle import overlap as ov

pytestmark = pytest.mark.gpu

TOL = 5e-6


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1111_6288_gb300 as P

    return P


def orthonormal_bank(dims, n_ev, seed):
    rng = np.random.default_rng(seed)
    site = synth.site_shape(dims) + (4, 3)
    m = int(np.prod(site))
    A = rng.standard_normal((m, n_ev)) + 1j * rng.standard_normal((m, n_ev))
    Q, _ = np.linalg.qr(A)
    V = np.ascontiguousarray(Q.T.reshape((n_ev,) + site))
    lam = np.where(rng.random(n_ev) < 0.4, -1.0, 1.0) * (0.01 + rng.random(n_ev))
    return V, lam


def relerr(got, want):
    return float(np.abs(got - want).max() / np.abs(want).max())


@pytest.mark.parametrize("dims,n_ev,nrhs", [((5, 3, 3, 7), 20, 8), ((5, 3, 3, 7), 20, 13), ((6, 4, 3, 6), 130, 27),
                                            ((5, 3, 3, 7), 37, 40), ((8, 8, 8, 8), 64, 24)])
def test_tensor_core_projection_matches_oracle(P, dims, n_ev, nrhs):
    import torch

    V, lam = orthonormal_bank(dims, n_ev, 7)
    x = synth.gaussian_spinor(dims, nrhs, 8)
    ctx = P.Context(P.Params(dims=dims, eps=0.01, poly_degree=4, precision=P.OV_PREC_F32,
                             inner_precision=P.OV_PREC_F32, max_nrhs=nrhs))
    P.deflate(ctx, torch.from_numpy(V).cuda(), lam)
    small = ov.SmallSpace.from_eigenpairs(V, lam)
    ys_want, xp_want = ov.project(small, x)
    xd = torch.from_numpy(x).to(torch.complex64).cuda()
    errs = {}
    for method in (1, 2):
        ctx.set_projection(method)
        ys = torch.full_like(xd, float("nan"))
        xp = torch.full_like(xd, float("nan"))
        P.project_small(ctx, xd, ys, xp)
        torch.cuda.synchronize()
        P.sync(ctx)
        got_ys, got_xp = ys.cpu().numpy(), xp.cpu().numpy()
        assert np.all(np.isfinite(got_ys)) and np.all(np.isfinite(got_xp))
        errs[method] = (relerr(got_ys, ys_want), relerr(got_xp, xp_want))
    print(f"{dims} N {n_ev} k {nrhs}: cuda cores {errs[1]}, tensor cores {errs[2]}")
    for method in (1, 2):
        assert max(errs[method]) < TOL, errs
    ctx.close()


def test_timed_choice_keeps_the_result(P):
    """Method 0 times both paths on the call's buffers and keeps the faster; the output is the same
    projection either way."""
    import torch

    dims, n_ev, nrhs = (6, 4, 3, 6), 24, 12
    V, lam = orthonormal_bank(dims, n_ev, 3)
    x = synth.gaussian_spinor(dims, nrhs, 4)
    ctx = P.Context(P.Params(dims=dims, eps=0.01, poly_degree=4, precision=P.OV_PREC_F32,
                             inner_precision=P.OV_PREC_F32, max_nrhs=nrhs))
    P.deflate(ctx, torch.from_numpy(V).cuda(), lam)
    ctx.set_projection(0)
    xd = torch.from_numpy(x).to(torch.complex64).cuda()
    ys, xp = torch.empty_like(xd), torch.empty_like(xd)
    P.project_small(ctx, xd, ys, xp)
    torch.cuda.synchronize()
    assert "projection N 24 k 12" in ctx.tune_info
    ys_want, xp_want = ov.project(ov.SmallSpace.from_eigenpairs(V, lam), x)
    assert relerr(ys.cpu().numpy(), ys_want) < TOL and relerr(xp.cpu().numpy(), xp_want) < TOL
    ctx.close()
