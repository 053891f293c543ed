"""The Wilson kernel that stages whole x-rows in shared memory (bulk copies on an mbarrier).

On lattices whose x-rows tile a thread block (Lx a multiple of 4, rows x Lx a multiple of 32
sites), launch_shape | 32 selects it.  It must agree with the oracle like the plain kernel and
give the same bits as the plain kernel, which accumulates the hops in the same order (z, t,
x, y), for every right-hand-side block and register budget, in FP32 and 16-bit storage.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from oracle import dirac

pytestmark = pytest.mark.gpu

M0 = -1.5
BC_NUM = {0: 1.0, 1: -1.0, 2: 0.0}
DIMS, BC = (8, 8, 4, 6), (2, 0, 1, 2)  # 384-site slices of 8 rows; Dirichlet x, t, antiperiodic z
PHASES = [0.3, 0.0, -0.2]
TOL = {1: 2e-6, 2: 16 * 2.0 ** -11, 3: 16 * 2.0 ** -8}  # one H_w (see test_gpu_parity / test_gpu_half)
TILED = [1 | 32, 1 | 16 | 32, 2 | 32, 4 | 32]


def obc(bc):
    return tuple(BC_NUM[b] for b in bc)


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1111_6288_gb300 as P

    return P


def ctx_for(P, precision, shape, degree=16, eps=0.05):
    import torch

    ctx = P.Context(P.Params(dims=DIMS, bc=BC, m0=M0, eps=eps, poly_degree=degree, precision=precision,
                             inner_precision=1, max_nrhs=4, launch_shape=shape))
    ctx.set_gauge(torch.from_numpy(synth.random_su3_field(DIMS, 0.3, 31)).cuda())
    for ph in set(PHASES):
        P.deflate(ctx, None, [], phase=ph)  # empty small spaces: the polynomial acts on everything
    return ctx


def run(P, ctx, fn, x, **kw):
    import torch

    xd = torch.from_numpy(np.ascontiguousarray(x)).to(torch.complex64).cuda()
    out = torch.empty_like(xd)
    fn(ctx, xd, out, **kw)
    P.sync(ctx)
    return out.cpu().numpy()


@pytest.mark.parametrize("precision", [1, 2, 3])
@pytest.mark.parametrize("shape", TILED)
def test_tiled_wilson_matches_oracle(P, precision, shape):
    U = synth.random_su3_field(DIMS, 0.3, 31)
    x = synth.gaussian_spinor(DIMS, 3, 32)
    ctx = ctx_for(P, precision, shape)
    got = run(P, ctx, P.apply_wilson, x, phase=PHASES, hermitian=True).astype(np.complex128)
    want = np.stack([dirac.hermitian_wilson(U, x[j], M0, obc(BC), PHASES[j]) for j in range(3)])
    err = float(np.abs(got - want).max() / np.abs(want).max())
    assert err < TOL[precision], err
    plain = run(P, ctx_for(P, precision, shape & 15), P.apply_wilson, x, phase=PHASES, hermitian=True)
    assert np.array_equal(plain, got.astype(np.complex64))
    ctx.close()


@pytest.mark.parametrize("precision", [1, 2, 3])
def test_tiled_overlap_equals_plain_bitwise(P, precision):
    """D(m) through the whole recurrence: the plain one-system kernel, every tiled shape on the
    batch of three, and one system at a time with the tiled kernel give the same bits."""
    x = synth.gaussian_spinor(DIMS, 3, 33)
    ref = run(P, ctx_for(P, precision, 1), P.apply_overlap, x, mass=0.05, phase=PHASES)
    assert np.isfinite(ref).all() and np.abs(ref).max() > 0
    for shape in TILED:
        ctx = ctx_for(P, precision, shape)
        assert np.array_equal(run(P, ctx, P.apply_overlap, x, mass=0.05, phase=PHASES), ref), shape
        one = run(P, ctx, P.apply_overlap, x[1:2], mass=0.05, phase=PHASES[1:2])
        assert np.array_equal(one[0], ref[1]), shape
        ctx.close()


def test_tuner_offers_the_tiled_kernel(P):
    import torch

    ctx = ctx_for(P, 1, 0)
    x = torch.from_numpy(synth.gaussian_spinor(DIMS, 2, 34)).to(torch.complex64).cuda()
    P.apply_sign_Hw(ctx, x, torch.empty_like(x), phase=[0.0, 0.0])
    P.sync(ctx)
    assert "t:" in ctx.tune_info
    ctx.close()
