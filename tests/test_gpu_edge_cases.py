"""Edge cases and failure detection on the GPU (no fault is provoked: every
failure here is detected on the host and returned as a status)."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from oracle import dirac

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
def ctx4(P):
    dims = (4, 4, 4, 4)
    ctx = P.Context(P.Params(dims=dims, bc=(0, 0, 0, 1), m0=M0, eps=0.002, poly_degree=60, max_nrhs=4, max_iter=0))
    ctx.set_gauge(dev(synth.random_su3_field(dims, 0.3, 0)))
    yield ctx
    ctx.close()


def test_nan_in_the_right_hand_side_is_reported(P, ctx4):
    import torch

    b = dev(synth.point_sources((4, 4, 4, 4), [(0, 0)]))
    b[0, 1, 1, 1, 1, 0, 0] = float("nan")
    x = torch.zeros_like(b)
    with pytest.raises(P.OvlError) as e:
        P.solve_overlap(ctx4, b, x, 0.1)
    assert e.value.code == 6


def test_iteration_cap_returns_not_converged_with_the_best_iterate(P):
    import torch

    dims = (4, 4, 4, 4)
    ctx = P.Context(P.Params(dims=dims, bc=(0, 0, 0, 1), m0=M0, eps=0.002, poly_degree=60, max_nrhs=2, max_iter=3))
    ctx.set_gauge(dev(synth.random_su3_field(dims, 0.3, 0)))
    b = dev(synth.point_sources(dims, [(1, 1)]))
    x = torch.zeros_like(b)
    st = P.solve_overlap(ctx, b, x, 0.1, raise_on_error=False)
    assert st.status == 4 and st.inner_iters == 3
    assert 0.0 < st.true_residual < 1.0 and float(x.norm()) > 0.0
    ctx.close()


def test_bounded_wait_timeout_is_reported_and_the_context_survives(P, ctx4):
    """A device wait that runs out (an mbarrier nothing completes, ~1 ms bound) is reported by
    the next sync as OV_ERR_TIMEOUT, once; the context keeps working afterwards."""
    import torch

    P.sync(ctx4)
    P.selftest_bounded_wait(ctx4)
    with pytest.raises(P.OvlError) as e:
        P.sync(ctx4)
    assert e.value.code == 7
    P.sync(ctx4)  # the flag was cleared
    x = dev(synth.gaussian_spinor(ctx4.dims, 1, 9))
    y = torch.empty_like(x)
    P.apply_wilson(ctx4, x, y, hermitian=True)
    P.sync(ctx4)
    assert torch.isfinite(y).all()


def test_zero_right_hand_side_gives_zero(P, ctx4):
    import torch

    b = torch.zeros((2,) + ctx4.site_shape + (4, 3), dtype=torch.complex128, device="cuda")
    b[1] = dev(synth.point_sources((4, 4, 4, 4), [(2, 2)]))[0]
    x = torch.zeros_like(b)
    st = P.solve_overlap(ctx4, b, x, 0.1)
    assert st.status == 0 and float(x[0].abs().max()) == 0.0 and st.true_residual <= 1e-10


def test_argument_errors(P, ctx4):
    import torch

    x = dev(synth.gaussian_spinor((4, 4, 4, 4), 1, 1))
    with pytest.raises(P.OvlError) as e:
        P.apply_wilson(ctx4, x, x)  # in == out
    assert e.value.code == 1
    big = dev(synth.gaussian_spinor((4, 4, 4, 4), 5, 1))
    with pytest.raises(P.OvlError) as e:
        P.apply_wilson(ctx4, big, torch.empty_like(big))  # more than max_nrhs
    assert e.value.code == 1
    with pytest.raises(P.OvlError) as e:
        P.apply_overlap(ctx4, x, torch.empty_like(x), mass=float("inf"))
    assert e.value.code == 1


# ---------------------------------------------------------------------------
# the workload's full size (16^3 x 32) in the bench's launch configuration
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def full(P):
    dims = (16, 16, 16, 32)
    U = synth.random_su3_field(dims, 0.2, 0)
    return dims, U


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-6)])
def test_wilson_full_size_matches_oracle(P, full, precision, tol):
    import torch

    dims, U = full
    ctx = P.Context(P.Params(dims=dims, bc=(0, 0, 0, 1), m0=M0, eps=4e-4, poly_degree=527, precision=precision,
                             inner_precision=precision, max_nrhs=2))
    ctx.set_gauge(dev(U))
    x = synth.gaussian_spinor(dims, 2, 1)
    xd = dev(x).to(ctx.spinor_dtype())
    y = torch.empty_like(xd)
    P.apply_wilson(ctx, xd, y, phase=[0.0, 1e-4], hermitian=True)
    got = y.cpu().numpy()
    for j, ph in enumerate([0.0, 1e-4]):
        want = dirac.hermitian_wilson(U, x[j], M0, (1, 1, 1, -1), ph)
        assert np.abs(got[j] - want).max() / np.abs(want).max() < tol
    ctx.close()


def test_sign_full_size_properties(P, full):
    """Without a small space (|Q| >= 0.0825 > sqrt(eps) here): sign^2 = 1 and
    hermiticity of the FP64 sign within delta; FP32 against FP64."""
    import torch

    dims, U = full
    Ud = dev(U)
    c64 = P.Context(P.Params(dims=dims, bc=(0, 0, 0, 1), m0=M0, eps=4e-4, poly_degree=527, max_nrhs=2))
    c32 = P.Context(P.Params(dims=dims, bc=(0, 0, 0, 1), m0=M0, eps=4e-4, poly_degree=527, precision=1, max_nrhs=2))
    c64.set_gauge(Ud)
    c32.set_gauge(Ud)
    delta = c64.delta
    x = dev(synth.gaussian_spinor(dims, 2, 3))
    s = torch.empty_like(x)
    P.apply_sign_Hw(c64, x, s)
    ss = torch.empty_like(x)
    P.apply_sign_Hw(c64, s, ss)
    assert float((ss - x).norm() / x.norm()) < 10 * delta
    a, b = x[0:1].contiguous(), x[1:2].contiguous()
    lhs = torch.vdot(a.flatten(), s[1].flatten())
    rhs = torch.vdot(s[0].flatten(), b.flatten())
    assert abs(complex(lhs - rhs)) < 1e-12
    s32 = torch.empty_like(x.to(torch.complex64))
    P.apply_sign_Hw(c32, x.to(torch.complex64), s32)
    assert float((s32.to(torch.complex128) - s).norm() / s.norm()) < 1e-5
    c64.close()
    c32.close()
