"""ctypes binding of libovl (see include/ovl.h for the contract of each call)."""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(HERE, "libovl.so")

OV_OK = 0
(OV_ERR_ARG, OV_ERR_CUDA, OV_ERR_OOM, OV_ERR_NOT_CONVERGED, OV_ERR_BREAKDOWN, OV_ERR_NAN, OV_ERR_TIMEOUT,
 OV_ERR_NO_BANK, OV_ERR_STATE) = range(1, 10)
OV_BC_PERIODIC, OV_BC_ANTIPERIODIC, OV_BC_DIRICHLET = 0, 1, 2
OV_PREC_F64, OV_PREC_F32, OV_PREC_F16, OV_PREC_BF16 = 0, 1, 2, 3
OV_C128, OV_C64 = 0, 1
ERROR_NAMES = {1: "ARG", 2: "CUDA", 3: "OOM", 4: "NOT_CONVERGED", 5: "BREAKDOWN", 6: "NAN", 7: "TIMEOUT",
               8: "NO_BANK", 9: "STATE"}


class OvlError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"libovl error {code} ({ERROR_NAMES.get(code, '?')}): {message}")
        self.code = code


class _Params(C.Structure):
    _fields_ = [
        ("dims", C.c_int * 4),
        ("bc", C.c_int * 4),
        ("m0", C.c_double),
        ("hw_norm", C.c_double),
        ("eps", C.c_double),
        ("poly_degree", C.c_int),
        ("coeffs", C.POINTER(C.c_double)),
        ("precision", C.c_int),
        ("inner_precision", C.c_int),
        ("max_nrhs", C.c_int),
        ("max_iter", C.c_int),
        ("inner_tol", C.c_double),
        ("launch_shape", C.c_int),
        ("poly_kind", C.c_int),
        ("adaptive_order", C.c_int),
    ]


class _SolveStats(C.Structure):
    _fields_ = [
        ("status", C.c_int),
        ("outer_iters", C.c_int),
        ("inner_iters", C.c_int),
        ("sign_applies", C.c_longlong),
        ("dslash_calls", C.c_longlong),
        ("true_residual", C.c_double),
        ("seconds", C.c_double),
    ]


class _Profile(C.Structure):
    _fields_ = [
        ("clenshaw_ms", C.c_double),
        ("clenshaw_regions", C.c_longlong),
        ("clenshaw_launches", C.c_longlong),
        ("clenshaw_bytes", C.c_double),
        ("kernel_launches", C.c_longlong),
    ]


_VP, _DP, _I, _D = C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_double

_SIGNATURES = {
    "ov_create": (_I, [C.POINTER(_Params), C.POINTER(_VP)]),
    "ov_destroy": (_I, [_VP]),
    "ov_last_error": (C.c_char_p, [_VP]),
    "ov_last_info": (C.c_char_p, [_VP]),
    "ov_tune_info": (C.c_char_p, [_VP]),
    "ov_sync": (_I, [_VP, _VP]),
    "ov_selftest_bounded_wait": (_I, [_VP, _VP]),
    "ov_eigensolve_overlap": (_I, [_VP, _D, _I, _I, _I, _D, _I, _DP, _DP, _VP]),
    "ov_clear_overlap_deflation": (_I, [_VP, _D, _I]),
    "ov_volume": (C.c_longlong, [_VP]),
    "ov_hw_norm": (_D, [_VP]),
    "ov_poly_delta": (_D, [_VP]),
    "ov_poly_delta_n": (_D, [_I, _D]),
    "ov_minimax_coeffs": (_D, [_I, _D, _DP]),
    "ov_adaptive_degree": (_I, [_VP, _D]),
    "ov_set_gauge": (_I, [_VP, _VP, _I, _VP]),
    "ov_set_profiling": (_I, [_VP, _I]),
    "ov_read_profile": (_I, [_VP, _I, C.POINTER(_Profile)]),
    "ov_launch_count": (C.c_longlong, []),
    "ov_chebyshev_coeffs": (_I, [_I, _D, _DP]),
    "ov_host_eigh": (_I, [_I, _DP, _DP, _DP]),
    "apply_wilson": (_I, [_VP, _VP, _VP, _I, _DP, _I, _VP]),
    "apply_sign_Hw": (_I, [_VP, _VP, _VP, _I, _DP, _VP]),
    "apply_overlap": (_I, [_VP, _VP, _VP, _I, _D, _DP, _VP]),
    "apply_wilson_noalloc": (_I, [C.POINTER(C.c_int), C.POINTER(C.c_int), _D, _VP, _VP, _VP, _I, _DP, _I, _VP]),
    "ov_project_small": (_I, [_VP, _D, _VP, _VP, _VP, _I, _VP]),
    "ov_set_projection": (_I, [_VP, _I]),
    "ov_set_eigensolver_memory": (_I, [_VP, C.c_longlong]),
    "deflate": (_I, [_VP, _D, _VP, _DP, _I, _I, _VP]),
    "ov_eigensolve_Q": (_I, [_VP, _D, _I, _D, _I, _VP, _DP, _I, _VP]),
    "ov_set_inner_precision": (_I, [_VP, _I]),
    "solve_overlap": (_I, [_VP, _D, _DP, _VP, _VP, _I, _D, C.POINTER(_SolveStats), _VP]),
    "solve_overlap_multimass": (_I, [_VP, _I, _DP, _DP, _VP, _VP, _I, _D, C.POINTER(_SolveStats), _VP]),
    "ov_apply_dHdphi": (_I, [_VP, _VP, _VP, _I, _DP, _VP]),
    "ov_apply_dDdphi": (_I, [_VP, _VP, _VP, _I, _D, _DP, _VP]),
    "ov_correlator": (_I, [_VP, _VP, _I, _DP, _VP]),
    "ov_dcorr_dE": (_I, [_VP, _D, _D, _D, _VP, _VP, _I, _D, _DP, _VP]),
    "ov_timeslice_scale": (_I, [_VP, _VP, _VP, _I, _DP, _I, _VP]),
    "ov_inner": (_I, [_VP, _VP, _VP, _I, _I, _DP, _VP]),
}

_lib = None


def library_path():
    return _LIB_PATH


def lib():
    """The loaded libovl.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libovl.so is not built ({_LIB_PATH}); run paper_1111_6288_gb300.build.build()")
        L = C.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc, ctx_handle=None):
    if rc != OV_OK:
        msg = lib().ov_last_error(ctx_handle)
        raise OvlError(rc, msg.decode() if msg else "")


def _darr(values):
    if values is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(values, dtype=np.float64))
    return a, a.ctypes.data_as(_DP)


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


@dataclass
class Params:
    """Mirror of ``ov_params`` (include/ovl.h)."""

    dims: Sequence[int]
    bc: Sequence[int] = (OV_BC_PERIODIC, OV_BC_PERIODIC, OV_BC_PERIODIC, OV_BC_ANTIPERIODIC)
    m0: float = -1.5
    hw_norm: float = 0.0
    eps: float = 0.01
    poly_degree: int = 200
    coeffs: Optional[Sequence[float]] = None
    precision: int = OV_PREC_F64
    inner_precision: int = OV_PREC_F64
    max_nrhs: int = 12
    max_iter: int = 0
    inner_tol: float = 0.0
    launch_shape: int = 0
    poly_kind: int = 0
    adaptive_order: int = 0


@dataclass
class SolveStats:
    status: int = 0
    outer_iters: int = 0
    inner_iters: int = 0
    sign_applies: int = 0
    dslash_calls: int = 0
    true_residual: float = 0.0
    seconds: float = 0.0


class Context:
    """An ``ov_ctx``: one lattice geometry and operator parameter set."""

    def __init__(self, params: Params):
        p = _Params()
        p.dims[:] = list(params.dims)
        p.bc[:] = list(params.bc)
        p.m0 = params.m0
        p.hw_norm = params.hw_norm
        p.eps = params.eps
        p.poly_degree = params.poly_degree
        self._coeffs, cptr = _darr(params.coeffs)
        p.coeffs = cptr
        p.precision = params.precision
        p.inner_precision = params.inner_precision
        p.max_nrhs = params.max_nrhs
        p.max_iter = params.max_iter
        p.inner_tol = params.inner_tol
        p.launch_shape = params.launch_shape
        p.poly_kind = params.poly_kind
        p.adaptive_order = params.adaptive_order
        h = C.c_void_p()
        rc = lib().ov_create(C.byref(p), C.byref(h))
        _check(rc, None)
        self.handle = h
        self.params = params
        self.dims = tuple(int(d) for d in params.dims)

    def close(self):
        if getattr(self, "handle", None):
            lib().ov_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def last_info(self):
        """Summary of the last solve (cycles, degrees, iterations) or eigensolver call on this context."""
        return lib().ov_last_info(self.handle).decode()

    @property
    def tune_info(self):
        """Timings of the Wilson-kernel right-hand-side blocks tried so far."""
        return lib().ov_tune_info(self.handle).decode()

    @property
    def volume(self):
        return int(lib().ov_volume(self.handle))

    @property
    def hw_norm(self):
        return float(lib().ov_hw_norm(self.handle))

    @property
    def delta(self):
        """Error |1 - sqrt(x) P(x)| of the polynomial in use, maximised over [eps, 1]."""
        return float(lib().ov_poly_delta(self.handle))

    def adaptive_degree(self, delta_target):
        """Degree the adaptive order picks for a polynomial error target (host; no GPU)."""
        return int(lib().ov_adaptive_degree(self.handle, float(delta_target)))

    @property
    def site_shape(self):
        lx, ly, lz, lt = self.dims
        return (lt, lz, ly, lx)

    def spinor_dtype(self):
        import torch

        return torch.complex128 if self.params.precision == OV_PREC_F64 else torch.complex64

    def _check_spinor(self, t, name, dtype=None):
        import torch

        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        want = dtype or self.spinor_dtype()
        if t.dtype != want:
            raise TypeError(f"{name} has dtype {t.dtype}, expected {want}")
        if tuple(t.shape[1:]) != self.site_shape + (4, 3):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected (nrhs,) + {self.site_shape + (4, 3)}")
        return t.shape[0]

    def set_inner_precision(self, precision):
        """Inner-CG precision of later solves (OV_PREC_F64, OV_PREC_F32, or the context's 16-bit format)."""
        _check(lib().ov_set_inner_precision(self.handle, int(precision)), self.handle)
        self.params.inner_precision = int(precision)

    def set_projection(self, method):
        """FP32 small-space projections of 8+ vectors: 0 timed choice, 1 CUDA cores, 2 tensor cores."""
        _check(lib().ov_set_projection(self.handle, int(method)), self.handle)

    def set_eigensolver_memory(self, nbytes):
        """Working-set budget (bytes) of the eigensolver's chunked filter and residual passes."""
        _check(lib().ov_set_eigensolver_memory(self.handle, int(nbytes)), self.handle)

    def set_profiling(self, on=True):
        """Record CUDA events around every polynomial (Clenshaw) loop."""
        _check(lib().ov_set_profiling(self.handle, int(on)), self.handle)

    def read_profile(self, precision=OV_PREC_F32):
        """Summed event time, launches and algorithmic bytes of the recorded loops of one
        precision (resets them)."""
        p = _Profile()
        _check(lib().ov_read_profile(self.handle, int(precision), C.byref(p)), self.handle)
        return dict(clenshaw_ms=p.clenshaw_ms, clenshaw_regions=p.clenshaw_regions,
                    clenshaw_launches=p.clenshaw_launches, clenshaw_bytes=p.clenshaw_bytes,
                    kernel_launches=p.kernel_launches)

    def set_gauge(self, U, stream=None):
        import torch

        if not (isinstance(U, torch.Tensor) and U.is_cuda and U.is_contiguous()):
            raise TypeError("U must be a contiguous CUDA tensor")
        if tuple(U.shape) != (4,) + self.site_shape + (3, 3):
            raise ValueError(f"U has shape {tuple(U.shape)}")
        dt = {torch.complex128: OV_C128, torch.complex64: OV_C64}.get(U.dtype)
        if dt is None:
            raise TypeError("U must be complex128 or complex64")
        _check(lib().ov_set_gauge(self.handle, C.c_void_p(U.data_ptr()), dt, _stream(stream)), self.handle)


def _phase_ptr(phase, nrhs):
    if phase is None:
        return None, None
    if np.isscalar(phase):
        phase = [float(phase)] * nrhs
    if len(phase) != nrhs:
        raise ValueError("phase must have one entry per right-hand side")
    return _darr(phase)


def apply_wilson(ctx: Context, x, out, phase=None, hermitian=False, stream=None):
    """out = D_w x (or H_w x = gamma5 D_w x if hermitian)."""
    n = ctx._check_spinor(x, "x")
    ctx._check_spinor(out, "out")
    keep, ph = _phase_ptr(phase, n)
    rc = lib().apply_wilson(ctx.handle, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), n, ph, int(hermitian),
                            _stream(stream))
    _check(rc, ctx.handle)
    return out


def eigensolve_overlap(ctx: Context, n_ev, chirality=1, phase=0.0, krylov=0, tol=1e-4, max_restarts=50, stream=None):
    """Low modes of D_ov in one chiral sector for the solver's deflated CG (registered on ctx);
    returns (Ritz values of P_s D_ov^+ D_ov P_s, residual norms) as numpy arrays."""
    theta = np.zeros(n_ev)
    res = np.zeros(n_ev)
    _check(lib().ov_eigensolve_overlap(ctx.handle, float(phase), int(chirality), int(n_ev), int(krylov), float(tol),
                                       int(max_restarts), theta.ctypes.data_as(_DP), res.ctypes.data_as(_DP),
                                       _stream(stream)), ctx.handle)
    return theta, res


def clear_overlap_deflation(ctx: Context, phase=0.0, chirality=0):
    """Drop the D_ov deflation spaces of a phase (chirality 0: both sectors)."""
    _check(lib().ov_clear_overlap_deflation(ctx.handle, float(phase), int(chirality)), ctx.handle)


def selftest_bounded_wait(ctx: Context, stream=None):
    """Make one bounded device wait run out (about 1 ms); the next sync() raises OV_ERR_TIMEOUT."""
    _check(lib().ov_selftest_bounded_wait(ctx.handle, _stream(stream)), ctx.handle)


def sync(ctx: Context, stream=None):
    """Synchronise the stream; raises OvlError (OV_ERR_TIMEOUT) if a bounded device wait ran out."""
    _check(lib().ov_sync(ctx.handle, _stream(stream)), ctx.handle)


def apply_sign_Hw(ctx: Context, x, out, phase=None, stream=None):
    """out = sign(H_w) x with the registered small space."""
    n = ctx._check_spinor(x, "x")
    ctx._check_spinor(out, "out")
    keep, ph = _phase_ptr(phase, n)
    _check(lib().apply_sign_Hw(ctx.handle, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), n, ph,
                               _stream(stream)), ctx.handle)
    return out


def apply_overlap(ctx: Context, x, out, mass=0.0, phase=None, stream=None):
    """out = D(m) x = (1 - m/2)(x + gamma5 sign(H_w) x) + m x."""
    n = ctx._check_spinor(x, "x")
    ctx._check_spinor(out, "out")
    keep, ph = _phase_ptr(phase, n)
    _check(lib().apply_overlap(ctx.handle, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), n, float(mass), ph,
                               _stream(stream)), ctx.handle)
    return out


def project_small(ctx: Context, x, ys, xperp, phase=0.0, stream=None):
    """ys = V diag(s) V^+ x and xperp = x - V V^+ x with the bank registered for phase."""
    n = ctx._check_spinor(x, "x")
    ctx._check_spinor(ys, "ys")
    ctx._check_spinor(xperp, "xperp")
    _check(lib().ov_project_small(ctx.handle, float(phase), C.c_void_p(x.data_ptr()), C.c_void_p(ys.data_ptr()),
                                  C.c_void_p(xperp.data_ptr()), n, _stream(stream)), ctx.handle)
    return ys, xperp


def deflate(ctx: Context, V, lam, phase=0.0, stream=None):
    """Register the small-space bank (V: [n_ev, ...site..., 4, 3] CUDA tensor, lam: n_ev eigenvalues of Q)."""
    import torch

    lam_a, lam_p = _darr(lam)
    n_ev = 0 if lam_a is None else len(lam_a)
    if n_ev == 0:
        _check(lib().deflate(ctx.handle, float(phase), None, None, 0, OV_C128, _stream(stream)), ctx.handle)
        return
    dt = {torch.complex128: OV_C128, torch.complex64: OV_C64}.get(V.dtype)
    if dt is None or not V.is_cuda or not V.is_contiguous() or V.shape[0] != n_ev:
        raise TypeError("V must be a contiguous CUDA complex tensor with one vector per eigenvalue")
    ctx._check_spinor(V, "V", dtype=V.dtype)
    _check(lib().deflate(ctx.handle, float(phase), C.c_void_p(V.data_ptr()), lam_p, n_ev, dt, _stream(stream)),
           ctx.handle)


def eigensolve_Q(ctx: Context, n_ev, phase=0.0, tol=1e-10, max_iter=100, register=True, want_vectors=False,
                 stream=None):
    """Lowest-|lambda| eigenpairs of Q (FP64); returns (lambda, V or None)."""
    import torch

    lam = np.zeros(n_ev)
    V = None
    vptr = None
    if want_vectors:
        V = torch.empty((n_ev,) + ctx.site_shape + (4, 3), dtype=torch.complex128, device="cuda")
        vptr = C.c_void_p(V.data_ptr())
    rc = lib().ov_eigensolve_Q(ctx.handle, float(phase), int(n_ev), float(tol), int(max_iter), vptr,
                               lam.ctypes.data_as(_DP), int(register), _stream(stream))
    _check(rc, ctx.handle)
    return lam, V


def solve_overlap(ctx: Context, b, x, mass, tol=1e-10, phase=None, stream=None, raise_on_error=True):
    """Solve D(m) x = b (x: initial guess in, solution out); returns SolveStats."""
    import torch

    n = ctx._check_spinor(b, "b", dtype=torch.complex128)
    ctx._check_spinor(x, "x", dtype=torch.complex128)
    keep, ph = _phase_ptr(phase, n)
    st = _SolveStats()
    rc = lib().solve_overlap(ctx.handle, float(mass), ph, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), n,
                             float(tol), C.byref(st), _stream(stream))
    stats = SolveStats(st.status, st.outer_iters, st.inner_iters, st.sign_applies, st.dslash_calls, st.true_residual,
                       st.seconds)
    if raise_on_error:
        _check(rc, ctx.handle)
    return stats


def solve_overlap_multimass(ctx: Context, b, x, masses, tol=1e-10, phase=None, stream=None, raise_on_error=True):
    """Solve D(m_i) x[i] = b for every mass (the multi-mass CG: one shared first cycle, then each
    mass on its own).  b: [nrhs, ...sites, 4, 3] complex128; x: [n_mass, nrhs, ...] complex128,
    output only.  Returns one SolveStats per mass (the shared cycle's work in the first)."""
    import torch

    masses = [float(m) for m in masses]
    nm = len(masses)
    if nm < 1:
        raise ValueError("at least one mass")
    n = ctx._check_spinor(b, "b", dtype=torch.complex128)
    if not isinstance(x, torch.Tensor) or x.dim() < 2 or x.shape[0] != nm:
        raise ValueError(f"x must have shape (n_mass = {nm}, nrhs, ...)")
    if ctx._check_spinor(x[0], "x[0]", dtype=torch.complex128) != n or not x.is_contiguous():
        raise ValueError("x[i] must match b's shape and x must be contiguous")
    keep, ph = _phase_ptr(phase, n)
    marr = np.ascontiguousarray(masses, dtype=np.float64)
    st = (_SolveStats * max(nm, 1))()
    rc = lib().solve_overlap_multimass(ctx.handle, nm, marr.ctypes.data_as(_DP), ph, C.c_void_p(b.data_ptr()),
                                       C.c_void_p(x.data_ptr()), n, float(tol), st, _stream(stream))
    stats = [SolveStats(s.status, s.outer_iters, s.inner_iters, s.sign_applies, s.dslash_calls, s.true_residual,
                        s.seconds) for s in st[:nm]]
    if raise_on_error:
        _check(rc, ctx.handle)
    return stats


def launch_count():
    """Kernels the library has launched so far in this process."""
    return int(lib().ov_launch_count())


def chebyshev_coeffs(n, eps):
    """The library's Chebyshev coefficients of x^{-1/2} on [eps, 1] (host; no GPU)."""
    out = np.zeros(n + 1)
    _check(lib().ov_chebyshev_coeffs(int(n), float(eps), out.ctypes.data_as(_DP)))
    return out


def minimax_coeffs(n, eps):
    """The library's minimax coefficients (least relative error for x^{-1/2} on [eps, 1], host);
    returns (coefficients, delta)."""
    out = np.zeros(n + 1)
    d = float(lib().ov_minimax_coeffs(int(n), float(eps), out.ctypes.data_as(_DP)))
    if d < 0:
        raise OvlError(1, "ov_minimax_coeffs: invalid arguments")
    return out, d


def poly_delta(n, eps):
    """delta = max over [eps, 1] of |1 - sqrt(x) P(x)| of the library's degree-n interpolant (host)."""
    v = float(lib().ov_poly_delta_n(int(n), float(eps)))
    if v < 0:
        raise OvlError(1, "ov_poly_delta_n: invalid arguments")
    return v


def host_eigh(A):
    """The library's host Hermitian eigensolver (no GPU); returns (w ascending, Z)."""
    A = np.asfortranarray(np.asarray(A, dtype=np.complex128)).copy(order="F")
    n = A.shape[0]
    w = np.zeros(n)
    Z = np.zeros((n, n), dtype=np.complex128, order="F")
    _check(lib().ov_host_eigh(n, A.ctypes.data_as(_DP), w.ctypes.data_as(_DP), Z.ctypes.data_as(_DP)))
    return w, Z


# ---------------------------------------------------------------------------
# field derivatives and the pion correlator (Sec. 4)
# ---------------------------------------------------------------------------

def apply_dHdphi(ctx: Context, x, out, phase=None, stream=None):
    """out = dH_w/dphi x (complex128)."""
    import torch

    n = ctx._check_spinor(x, "x", dtype=torch.complex128)
    ctx._check_spinor(out, "out", dtype=torch.complex128)
    keep, ph = _phase_ptr(phase, n)
    _check(lib().ov_apply_dHdphi(ctx.handle, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), n, ph,
                                 _stream(stream)), ctx.handle)
    return out


def apply_dDdphi(ctx: Context, x, out, mass, phase=None, stream=None):
    """out = dD(m)/dphi x (complex128), through the small space and the polynomial."""
    import torch

    n = ctx._check_spinor(x, "x", dtype=torch.complex128)
    ctx._check_spinor(out, "out", dtype=torch.complex128)
    keep, ph = _phase_ptr(phase, n)
    _check(lib().ov_apply_dDdphi(ctx.handle, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), n, float(mass),
                                 ph, _stream(stream)), ctx.handle)
    return out


def correlator(ctx: Context, S, stream=None):
    """C(t) = sum over right-hand sides, space, spin and colour of |S|^2 (numpy [Lt])."""
    import torch

    n = ctx._check_spinor(S, "S", dtype=torch.complex128)
    out = np.zeros(ctx.dims[3])
    _check(lib().ov_correlator(ctx.handle, C.c_void_p(S.data_ptr()), n, out.ctypes.data_as(_DP), _stream(stream)),
           ctx.handle)
    return out


def timeslice_scale(ctx: Context, x, out, w, gamma5=False, stream=None):
    """out(t) = w(t) (gamma5) x(t)."""
    import torch

    n = ctx._check_spinor(x, "x", dtype=torch.complex128)
    ctx._check_spinor(out, "out", dtype=torch.complex128)
    wa, wp = _darr(w)
    _check(lib().ov_timeslice_scale(ctx.handle, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), n, wp,
                                    int(gamma5), _stream(stream)), ctx.handle)
    return out


def inner(ctx: Context, a, b, per_timeslice=False, stream=None):
    """<a_j, b_j> per right-hand side (numpy complex [nrhs]) or per (rhs, t) ([nrhs, Lt])."""
    import torch

    n = ctx._check_spinor(a, "a", dtype=torch.complex128)
    ctx._check_spinor(b, "b", dtype=torch.complex128)
    m = n * (ctx.dims[3] if per_timeslice else 1)
    out = np.zeros(2 * m)
    _check(lib().ov_inner(ctx.handle, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), n, int(per_timeslice),
                          out.ctypes.data_as(_DP), _stream(stream)), ctx.handle)
    z = out[0::2] + 1j * out[1::2]
    return z.reshape(n, ctx.dims[3]) if per_timeslice else z


def _solve_columns(ctx, b, mass, phase, tol):
    import torch

    x = torch.zeros_like(b)
    solve_overlap(ctx, b, x, mass, tol=tol, phase=[phase] * b.shape[0])
    return x


def dcorr_dE(ctx: Context, S, mass, charge, E, lam=None, tol=1e-12, stream=None):
    """ov_dcorr_dE: without lam, dC(t)/dE (numpy [Lt]) of C(t) = sum |S|^2_t through the tangent
    solve; with lam (the adjoint solution), the adjoint form's per-timeslice terms.  Returns
    (per-timeslice values [Lt], their sum)."""
    import torch

    n = ctx._check_spinor(S, "S", dtype=torch.complex128)
    lptr = None
    if lam is not None:
        if ctx._check_spinor(lam, "lam", dtype=torch.complex128) != n:
            raise ValueError("lam must have as many columns as S")
        lptr = C.c_void_p(lam.data_ptr())
    out = np.zeros(ctx.dims[3] + 1)
    _check(lib().ov_dcorr_dE(ctx.handle, float(mass), float(charge), float(E), C.c_void_p(S.data_ptr()), lptr, n,
                             float(tol), out.ctypes.data_as(_DP), _stream(stream)), ctx.handle)
    return out[:-1], float(out[-1])


def correlator_jacobian(ctx: Context, sources, E, charge, mass, tol=1e-12):
    """C(t) and dC(t)/dE at field E (phase charge * E), the derivative by the tangent of the solve
    (ov_dcorr_dE).  Returns numpy arrays [Lt]."""
    phase = charge * float(E)
    S = _solve_columns(ctx, sources, mass, phase, tol)
    return correlator(ctx, S), dcorr_dE(ctx, S, mass, charge, E, tol=tol)[0]


def _make_correlator_function():
    import torch

    class PionCorrelator(torch.autograd.Function):
        """C(t; E) of the point-source propagators at field E, phase phi = charge * E.

        forward: one solve per source and the correlator.  backward: the adjoint solve
        lam = D^-+ (g o S) = gamma5 D^-1 gamma5 (g o S), then dL/dE from ov_dcorr_dE.
        """

        @staticmethod
        def forward(fctx, E, ctx, sources, charge, mass, tol):
            phase = charge * float(E)
            S = _solve_columns(ctx, sources, mass, phase, tol)
            fctx.ovl = (ctx, S, charge, mass, tol, phase, float(E))
            return torch.from_numpy(correlator(ctx, S)).to(E.dtype)

        @staticmethod
        def backward(fctx, gC):
            ctx, S, charge, mass, tol, phase, E = fctx.ovl
            g = gC.detach().cpu().double().numpy()
            w = torch.empty_like(S)
            timeslice_scale(ctx, S, w, g, gamma5=True)        # gamma5 (g o S)
            y = _solve_columns(ctx, w, mass, phase, tol)
            lam = torch.empty_like(S)
            timeslice_scale(ctx, y, lam, np.ones(ctx.dims[3]), gamma5=True)
            _, gE = dcorr_dE(ctx, S, mass, charge, E, lam=lam)
            return torch.tensor(gE, dtype=gC.dtype), None, None, None, None, None

    return PionCorrelator


_PION = None


def pion_correlator(E, ctx: Context, sources, charge, mass, tol=1e-12):
    """Differentiable C(t; E) (torch.autograd): E is a 0-d float64 tensor."""
    global _PION
    if _PION is None:
        _PION = _make_correlator_function()
    return _PION.apply(E, ctx, sources, charge, mass, tol)
