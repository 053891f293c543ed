"""Host-side checks of libovl that need no GPU: the library builds and loads,
exports every symbol include/ovl.h declares, validates arguments on the host,
and its host routines (Chebyshev coefficients, small Hermitian eigensolver)
agree with independent references."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

from oracle import chebyshev

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ovl():
    import paper_1111_6288_gb300 as P
    from paper_1111_6288_gb300 import build

    if not os.path.exists(P.library_path()):
        build.build()
    return P


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\([^;]*\)\s*;", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for want in ["apply_wilson", "apply_sign_Hw", "apply_overlap", "deflate", "solve_overlap", "ov_create",
                 "ov_destroy", "ov_set_gauge", "ov_eigensolve_Q"]:
        assert want in names


def test_header_is_plain_c(tmp_path):
    """The boundary is a C ABI: the public header compiles as strict C99 (plain pointers, sizes and
    enums; no C++ or framework types)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "uses_ovl.c"
    src.write_text('#include "include/ovl.h"\nint main(void) { return OV_OK; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", ROOT, "-c", str(src),
                        "-o", str(tmp_path / "uses_ovl.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_library_exports_every_declared_symbol(ovl):
    L = ctypes.CDLL(ovl.library_path())
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_library_chebyshev_coefficients_match_oracle(ovl):
    for n, eps in [(13, 0.0036), (200, 0.01), (527, 4e-4), (1054, 1e-4)]:
        got = ovl.chebyshev_coeffs(n, eps)
        want = chebyshev.chebyshev_coeffs(n, eps)
        assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("n", [1, 2, 5, 17, 64])
def test_host_eigh_matches_numpy(ovl, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = A + A.conj().T
    A[0, min(1, n - 1)] += 0  # keep Hermitian
    w, Z = ovl.host_eigh(A)
    assert np.allclose(w, np.linalg.eigvalsh(A), atol=1e-12 * np.abs(w).max())
    assert np.allclose(Z.conj().T @ Z, np.eye(n), atol=1e-12)
    assert np.allclose(A @ Z, Z * w, atol=1e-11 * np.abs(w).max())


def test_host_eigh_degenerate(ovl):
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12)))
    w0 = np.array([1, 1, 1, 2, 2, -3, -3, 0.5, 0.5, 0.5, 0.5, 7.0])
    A = (Q * w0) @ Q.conj().T
    w, Z = ovl.host_eigh(A)
    assert np.allclose(w, np.sort(w0), atol=1e-12)
    assert np.allclose(A @ Z, Z * w, atol=1e-11)


@pytest.mark.parametrize("bad", [dict(dims=(1, 4, 4, 4)), dict(eps=0.0), dict(eps=1.0), dict(poly_degree=0),
                                 dict(precision=7), dict(max_nrhs=0), dict(bc=(0, 0, 0, 5)),
                                 dict(inner_precision=2), dict(inner_precision=3), dict(launch_shape=3),
                                 dict(launch_shape=64), dict(launch_shape=-1), dict(poly_kind=2)])
def test_create_rejects_invalid_parameters(ovl, bad):
    kw = dict(dims=(4, 4, 4, 4))
    kw.update(bad)
    with pytest.raises(ovl.OvlError) as e:
        ovl.Context(ovl.Params(**kw))
    assert e.value.code == 1


@pytest.mark.parametrize("precision", [2, 3])
def test_create_accepts_16bit_storage(ovl, precision):
    ctx = ovl.Context(ovl.Params(dims=(4, 4, 4, 4), precision=precision, inner_precision=1))
    assert ctx.spinor_dtype() == __import__("torch").complex64
    # the solver may use the context's own 16-bit format, not the other one
    ctx.set_inner_precision(precision)
    other = ovl.OV_PREC_BF16 if precision == ovl.OV_PREC_F16 else ovl.OV_PREC_F16
    with pytest.raises(ovl.OvlError) as e:
        ctx.set_inner_precision(other)
    assert e.value.code == ovl.OV_ERR_ARG
    ctx.set_inner_precision(ovl.OV_PREC_F64)
    ctx.close()
    ovl.Context(ovl.Params(dims=(4, 4, 4, 4), precision=precision, inner_precision=precision)).close()
    with pytest.raises(ovl.OvlError):
        ovl.Context(ovl.Params(dims=(4, 4, 4, 4), precision=ovl.OV_PREC_F32, inner_precision=precision))


@pytest.mark.parametrize("shape", [1, 2 | 32, 4 | 16 | 32, 8, 8 | 16])
def test_create_accepts_launch_shapes(ovl, shape):
    ovl.Context(ovl.Params(dims=(4, 4, 4, 4), launch_shape=shape)).close()


def test_create_resolves_norm_bound(ovl):
    ctx = ovl.Context(ovl.Params(dims=(4, 4, 4, 8), m0=-1.5))
    assert ctx.volume == 512
    assert ctx.hw_norm == pytest.approx(6.5)
    ctx.close()


@pytest.mark.parametrize("n,eps", [(64, 0.01), (527, 4e-4)])
def test_library_polynomial_delta_matches_oracle(ovl, n, eps):
    ctx = ovl.Context(ovl.Params(dims=(4, 4, 4, 4), eps=eps, poly_degree=n))
    want = chebyshev.approximation_error(chebyshev.chebyshev_coeffs(n, eps), eps)
    assert ctx.delta == pytest.approx(want, rel=0.05)
    ctx.close()


@pytest.mark.parametrize("n,eps", [(8, 0.1), (64, 0.01), (300, 4e-4)])
def test_poly_delta_of_any_degree_matches_oracle(ovl, n, eps):
    want = chebyshev.approximation_error(chebyshev.chebyshev_coeffs(n, eps), eps)
    assert ovl.poly_delta(n, eps) == pytest.approx(want, rel=0.05)


@pytest.mark.parametrize("n,eps", [(0, 0.01), (8, 0.1), (64, 0.01), (300, 4e-4)])
def test_minimax_coefficients_match_oracle(ovl, n, eps):
    c, d = ovl.minimax_coeffs(n, eps)
    co, do = chebyshev.minimax_coeffs(n, eps)
    assert d == pytest.approx(do, rel=1e-6)
    assert np.abs(c - co).max() <= 1e-9 * np.abs(co).max()


def test_minimax_kind_context_uses_it(ovl):
    ctx = ovl.Context(ovl.Params(dims=(4, 4, 4, 4), eps=4e-4, poly_degree=527, poly_kind=1))
    _, want = chebyshev.minimax_coeffs(527, 4e-4)
    assert ctx.delta == pytest.approx(want, rel=1e-3)
    assert ctx.delta < 1.3e-10  # eq. 2: 1e-10 at n = 527, sqrt(eps) = 0.02
    n = ctx.adaptive_degree(1e-8)
    assert n % 8 == 0 and chebyshev.approximation_error(chebyshev.minimax_coeffs(n, 4e-4)[0], 4e-4) <= 1e-8
    ctx.close()


def test_adaptive_degree_is_the_lowest_meeting_the_target(ovl):
    ctx = ovl.Context(ovl.Params(dims=(4, 4, 4, 4), eps=4e-4, poly_degree=527))
    for target in [1e-3, 3e-6, 1e-8, 5e-10]:
        n = ctx.adaptive_degree(target)
        assert n % 8 == 0 and n < 527
        assert ovl.poly_delta(n, 4e-4) <= target < ovl.poly_delta(n - 8, 4e-4)
    assert ctx.adaptive_degree(1e-10) == 527  # below the full degree's own delta (2.3e-10)
    ctx.close()
    custom = ovl.Context(ovl.Params(dims=(4, 4, 4, 4), eps=0.01, poly_degree=32,
                                    coeffs=list(chebyshev.chebyshev_coeffs(32, 0.01))))
    assert custom.adaptive_degree(1e-2) == 32  # the caller's coefficients are never replaced
    custom.close()


def _raw_ctx(ovl, **kw):
    p = ovl._ovl._Params()
    p.dims[:] = list(kw.get("dims", (4, 4, 4, 4)))
    p.bc[:] = [0, 0, 0, 1]
    p.m0 = -1.5
    p.eps = 0.01
    p.poly_degree = 8
    p.precision = 0
    p.inner_precision = 0
    p.max_nrhs = kw.get("max_nrhs", 2)
    h = ctypes.c_void_p()
    assert ovl.lib().ov_create(ctypes.byref(p), ctypes.byref(h)) == 0
    return h


def test_calls_before_a_gauge_field_are_rejected_on_the_host(ovl):
    """No GPU work is started: the state check comes first (the pointers are never used)."""
    L = ovl.lib()
    h = _raw_ctx(ovl)
    a, b = ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000)
    assert L.apply_wilson(h, a, b, 1, None, 1, None) == 9
    assert b"gauge" in L.ov_last_error(h)
    assert L.apply_sign_Hw(h, a, b, 1, None, None) == 9
    assert L.apply_overlap(h, a, b, 1, 0.1, None, None) == 9
    dC = (ctypes.c_double * 5)()
    assert L.ov_dcorr_dE(h, 0.1, 2.0 / 3.0, 1e-4, a, None, 1, 1e-10, dC, None) == ovl.OV_ERR_STATE
    assert L.ov_dcorr_dE(None, 0.1, 2.0 / 3.0, 1e-4, a, None, 1, 1e-10, dC, None) == ovl.OV_ERR_ARG
    L.ov_destroy(h)


def test_newer_calls_check_their_arguments_on_the_host(ovl):
    """The D_ov eigensolver, the deflation clear, the polynomial utilities and the adaptive
    degree reject or answer before any device work."""
    L = ovl.lib()
    h = _raw_ctx(ovl)
    theta = (ctypes.c_double * 4)()
    res = (ctypes.c_double * 4)()
    assert L.ov_eigensolve_overlap(h, 0.0, 1, 4, 0, 1e-4, 5, theta, res, None) == 9  # no gauge yet
    assert L.ov_clear_overlap_deflation(h, 0.0, 0) == 0  # nothing registered: nothing to free
    assert L.ov_clear_overlap_deflation(None, 0.0, 0) == 1
    assert L.ov_eigensolve_overlap(None, 0.0, 1, 4, 0, 1e-4, 5, theta, res, None) == 1
    assert L.ov_set_eigensolver_memory(h, 0) == 1
    assert L.ov_set_eigensolver_memory(h, -5) == 1
    assert L.ov_set_eigensolver_memory(h, 1) == 0
    assert L.ov_set_eigensolver_memory(None, 1 << 34) == 1
    L.ov_destroy(h)
    out = (ctypes.c_double * 8)()
    assert L.ov_minimax_coeffs(-1, 0.01, out) < 0
    assert L.ov_minimax_coeffs(4, 1.5, out) < 0
    assert L.ov_minimax_coeffs(4, 0.01, None) < 0
    assert L.ov_poly_delta_n(0, 0.01) < 0
    assert L.ov_poly_delta_n(10, 0.0) < 0
    assert L.ov_adaptive_degree(None, 1e-6) == 0
    assert L.ov_selftest_bounded_wait(None, None) == 1
    assert L.ov_sync(None, None) == 1


def test_multimass_solve_checks_its_arguments_on_the_host(ovl):
    """solve_overlap_multimass: the mass list and tolerance are checked before the state check,
    and no device work starts on a rejected call."""
    L = ovl.lib()
    h = _raw_ctx(ovl)
    a, b = ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000)
    st = (ovl._ovl._SolveStats * 4)()

    def call(masses, n=None, tol=1e-10, ctx=h):
        arr = (ctypes.c_double * max(len(masses), 1))(*masses)
        return L.solve_overlap_multimass(ctx, len(masses) if n is None else n, arr, None, a, b, 1, tol, st, None)

    assert call([0.1], ctx=None) == 1
    assert call([], n=0) == 1
    assert b"n_mass" in L.ov_last_error(h)
    assert call([0.1] * 33) == 1  # more than OV_MAX_MASSES
    assert call([0.1, float("nan")]) == 1
    assert call([0.1, 2.0]) == 1  # |m| < 2: the shift m^2 / (1 - m^2/4) must be finite
    assert call([0.1, -2.5]) == 1
    assert call([0.1, 0.2], tol=0.0) == 1
    assert call([0.1, 0.2]) == 9  # valid masses: the missing gauge field is reported
    ctx = ovl.Context(ovl.Params(dims=(4, 4, 4, 4), eps=0.01, poly_degree=8, max_nrhs=1))
    with pytest.raises(ValueError):
        ovl.solve_overlap_multimass(ctx, None, None, [])  # the binding needs at least one mass
    ctx.close()
    assert b"gauge" in L.ov_last_error(h)
    arr = (ctypes.c_double * 2)(0.1, 0.2)
    assert L.solve_overlap_multimass(h, 2, arr, None, a, a, 1, 1e-10, st, None) == 9  # state first
    L.ov_destroy(h)


def test_error_codes_for_invalid_arguments(ovl):
    L = ovl.lib()
    h = _raw_ctx(ovl)
    a = ctypes.c_void_p(0x1000)
    # eigensolver and deflate argument checks happen before any device work
    lam = (ctypes.c_double * 4)()
    assert L.ov_eigensolve_Q(h, 0.0, 4, 1e-8, 10, None, lam, 1, None) == 9  # no gauge yet
    assert L.deflate(h, 0.0, a, None, 3, 0, None) == 1  # lambda missing
    assert L.deflate(h, float("nan"), a, lam, 1, 0, None) == 1
    assert L.deflate(h, 0.0, a, lam, 1, 7, None) == 1  # bad dtype
    L.ov_destroy(h)
    # a context that cannot be made reports through ov_last_error(NULL)
    p = ovl._ovl._Params()
    p.dims[:] = [4, 4, 4, 4]
    p.eps = 0.5
    p.poly_degree = 8
    p.max_nrhs = 0
    hh = ctypes.c_void_p()
    assert L.ov_create(ctypes.byref(p), ctypes.byref(hh)) == 1
    assert b"max_nrhs" in L.ov_last_error(None)


def test_noalloc_rejects_oversize_without_a_gpu(ovl):
    L = ovl.lib()
    d = (ctypes.c_int * 4)(32, 32, 32, 32)
    bc = (ctypes.c_int * 4)(0, 0, 0, 1)
    rc = L.apply_wilson_noalloc(d, bc, -1.5, ctypes.c_void_p(16), ctypes.c_void_p(32), ctypes.c_void_p(64), 1, None, 1,
                                None)
    assert rc == ovl.OV_ERR_ARG and b"scratch" in L.ov_last_error(None)


@pytest.mark.parametrize("dims", [(2**31 - 1, 2**31 - 1, 2**31 - 1, 2**31 - 1), (2, 2**31 - 1, 2**30, 4),
                                  (65536, 65536, 65536, 65536)])
def test_extents_near_int_max_are_rejected_without_overflow(ovl, dims):
    """Extents whose product overflows 64 bits (or wraps to a small value) are rejected on the host."""
    L = ovl.lib()
    d = (ctypes.c_int * 4)(*dims)
    bc = (ctypes.c_int * 4)(0, 0, 0, 1)
    rc = L.apply_wilson_noalloc(d, bc, -1.5, ctypes.c_void_p(16), ctypes.c_void_p(32), ctypes.c_void_p(64), 1, None, 1,
                                None)
    assert rc == ovl.OV_ERR_ARG and b"scratch" in L.ov_last_error(None)
    with pytest.raises(ovl.OvlError) as e:
        ovl.Context(ovl.Params(dims=dims))
    assert e.value.code == ovl.OV_ERR_ARG
