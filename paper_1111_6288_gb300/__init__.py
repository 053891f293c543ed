"""GB300 (sm_103a) overlap Dirac operator library -- Python binding.

Thin ctypes wrapper around ``libovl.so`` (the C ABI declared in
``include/ovl.h``).  Every operation runs in the library's CUDA kernels; this
module only checks and marshals arguments.  PyTorch provides device memory and
streams.  There is no CPU fallback: if the library is not built, importing the
operations raises.

Method: Lujan, Alexandru, Lee, "Electric polarizability of hadrons with
overlap fermions on multi-GPUs" (Lattice 2011): D_ov = 1 + gamma5 sign(H_w)
(Sec. 2, eq. 1), sign(H_w) ~ Q P(Q^2) with an exact small space (Sec. 2),
CG for the propagator (Sec. 3.2), background electric field as a U(1) phase
on the links (Sec. 4).
"""
from ._ovl import (  # noqa: F401
    OV_BC_ANTIPERIODIC,
    OV_BC_DIRICHLET,
    OV_BC_PERIODIC,
    OV_ERR_ARG,
    OV_ERR_BREAKDOWN,
    OV_ERR_CUDA,
    OV_ERR_NAN,
    OV_ERR_NO_BANK,
    OV_ERR_NOT_CONVERGED,
    OV_ERR_OOM,
    OV_ERR_STATE,
    OV_ERR_TIMEOUT,
    OV_OK,
    OV_PREC_BF16,
    OV_PREC_F16,
    OV_PREC_F32,
    OV_PREC_F64,
    Context,
    OvlError,
    Params,
    SolveStats,
    apply_dDdphi,
    apply_dHdphi,
    apply_overlap,
    apply_sign_Hw,
    apply_wilson,
    chebyshev_coeffs,
    correlator,
    correlator_jacobian,
    dcorr_dE,
    clear_overlap_deflation,
    deflate,
    eigensolve_Q,
    eigensolve_overlap,
    host_eigh,
    inner,
    launch_count,
    lib,
    minimax_coeffs,
    library_path,
    pion_correlator,
    poly_delta,
    project_small,
    selftest_bounded_wait,
    solve_overlap,
    solve_overlap_multimass,
    sync,
    timeslice_scale,
)
