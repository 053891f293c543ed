"""apply_wilson_noalloc against apply_wilson, through the C ABI.

apply_wilson_noalloc is the Wilson operator for callers that cannot allocate
device memory (applications whose memory manager owns every device
allocation, real-time loops with a fixed budget, code that must not make the
device synchronisation cudaMalloc and cudaFree can cause): it works in one
fixed file-scope device array instead of allocating.
These checks run two calls in a row on different lattices and inputs (so the
second call starts from the first call's leftovers in the shared array) and
compare each with apply_wilson, the context-based entry point, and with the
oracle's Wilson operator, to the FP64 tolerance of the other parity tests.  The file sorts last so that a run that
stops at the first failure has run every other test before it.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import synth
from oracle import dirac

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
M0 = -1.5
BC_NUM = {0: 1.0, 1: -1.0, 2: 0.0}  # periodic, antiperiodic, Dirichlet (as factors on the boundary hop)


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1111_6288_gb300 as P

    return P


def reference(P, dims, bc, U, x, phases, hermitian):
    """apply_wilson through a context (the library's ordinary, allocating path)."""
    import torch

    ctx = P.Context(P.Params(dims=dims, bc=bc, m0=M0, eps=0.01, poly_degree=4, max_nrhs=x.shape[0]))
    ctx.set_gauge(torch.from_numpy(U).cuda())
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    P.apply_wilson(ctx, xd, out, phase=phases, hermitian=hermitian)
    torch.cuda.synchronize()
    ctx.close()
    return out.cpu().numpy()


def noalloc(P, dims, bc, U, x, phases, hermitian):
    import torch

    Ud = torch.from_numpy(U).cuda()
    xd = torch.from_numpy(x).cuda()
    out = torch.full_like(xd, float("nan"))
    d = (C.c_int * 4)(*dims)
    b = (C.c_int * 4)(*bc)
    ph = np.ascontiguousarray(phases, dtype=np.float64)
    rc = P.lib().apply_wilson_noalloc(d, b, M0, C.c_void_p(Ud.data_ptr()), C.c_void_p(xd.data_ptr()),
                                      C.c_void_p(out.data_ptr()), x.shape[0], ph.ctypes.data_as(C.POINTER(C.c_double)),
                                      int(hermitian), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, P.lib().ov_last_error(None)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def relerr(got, want):
    return float(np.abs(got - want).max() / np.abs(want).max())


def test_noalloc_matches_apply_wilson_on_two_calls_in_a_row(P):
    cases = [
        ((6, 4, 3, 6), (2, 0, 0, 2), [0.4, -0.2], True, 31),   # 432 sites, ragged, Dirichlet x and t
        ((4, 4, 4, 4), (0, 0, 0, 1), [0.0], False, 32),        # smaller second call: stale data beyond it
    ]
    for dims, bc, phases, herm, seed in cases:
        U = synth.random_su3_field(dims, 0.4, seed)
        x = synth.gaussian_spinor(dims, len(phases), seed + 1)
        want = reference(P, dims, bc, U, x, phases, herm)
        got = noalloc(P, dims, bc, U, x, phases, herm)
        assert np.all(np.isfinite(got))
        assert relerr(got, want) < F64_TOL
        op = dirac.hermitian_wilson if herm else dirac.wilson
        obc = tuple(BC_NUM[v] for v in bc)
        for j, ph in enumerate(phases):
            assert relerr(got[j], op(U, x[j], M0, obc, ph)) < F64_TOL


def test_noalloc_rejects_requests_beyond_its_array(P):
    import torch

    dims = (16, 16, 16, 16)  # 65536 sites: far beyond 8 MiB of scratch
    d = (C.c_int * 4)(*dims)
    b = (C.c_int * 4)(0, 0, 0, 1)
    dummy = torch.zeros(2, dtype=torch.complex128, device="cuda")
    rc = P.lib().apply_wilson_noalloc(d, b, M0, C.c_void_p(dummy.data_ptr()), C.c_void_p(dummy.data_ptr()),
                                      C.c_void_p(dummy.data_ptr() + 16), 1, None, 1,
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == P.OV_ERR_ARG
    assert b"scratch" in P.lib().ov_last_error(None)
