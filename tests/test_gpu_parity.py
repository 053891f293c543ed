"""CUDA path against the CPU oracle, element by element, through the C ABI.

FP64 results must agree with the oracle to 1e-12 relative per operator
application (max |difference| / max |oracle|).  FP32 results are held to a
bound derived from single-precision rounding (see ``F32_TOL``).  Lattices
span several 128-site thread blocks with ragged tails, plus the 2^4 case in
which forward and backward neighbours coincide.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from oracle import dense, dirac
from oracle import overlap as ov

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
# One Wilson application sums 9 terms of O(1) per component in FP32: a few ulps (6e-8) each.
F32_WILSON_TOL = 2e-6
M0 = -1.5


def relerr(got, want):
    return float(np.abs(got - want).max() / np.abs(want).max())


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1111_6288_gb300 as P

    return P


def to_dev(a, dtype=None):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


def make_ctx(P, dims, bc=(0, 0, 0, 1), precision=0, inner=0, eps=0.01, degree=30, hw_norm=0.0, max_nrhs=8,
             inner_tol=0.0):
    return P.Context(P.Params(dims=dims, bc=bc, m0=M0, hw_norm=hw_norm, eps=eps, poly_degree=degree,
                              precision=precision, inner_precision=inner, max_nrhs=max_nrhs, inner_tol=inner_tol))


BC_NUM = {0: 1.0, 1: -1.0, 2: 0.0}


def oracle_bc(bc):
    return tuple(BC_NUM[b] for b in bc)


def gpu_apply(P, ctx, fn, x, **kw):
    import torch

    xd = to_dev(x, ctx.spinor_dtype())
    out = torch.empty_like(xd)
    fn(ctx, xd, out, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy()


# ---------------------------------------------------------------------------
# Wilson operator
# ---------------------------------------------------------------------------

WILSON_CASES = [
    ((2, 2, 2, 2), (0, 0, 0, 1), [0.0]),
    ((4, 4, 4, 4), (0, 0, 0, 1), [0.0, 0.3]),
    ((6, 4, 3, 6), (2, 0, 0, 2), [0.4, -0.2, 0.0]),  # 432 sites: 3 blocks + a ragged tail
    ((5, 3, 4, 7), (1, 2, 0, 0), [1.3]),
]


@pytest.mark.parametrize("dims,bc,phases", WILSON_CASES)
@pytest.mark.parametrize("hermitian", [False, True])
def test_wilson_f64_matches_oracle(P, dims, bc, phases, hermitian):
    U = synth.random_su3_field(dims, 0.4, 11)
    x = synth.gaussian_spinor(dims, len(phases), 12)
    ctx = make_ctx(P, dims, bc)
    ctx.set_gauge(to_dev(U))
    got = gpu_apply(P, ctx, P.apply_wilson, x, phase=phases, hermitian=hermitian)
    f = dirac.hermitian_wilson if hermitian else dirac.wilson
    want = np.stack([f(U, x[j], M0, oracle_bc(bc), phases[j]) for j in range(len(phases))])
    assert relerr(got, want) < F64_TOL
    ctx.close()


@pytest.mark.parametrize("dims,bc,phases", WILSON_CASES[1:3])
def test_wilson_f32_matches_oracle(P, dims, bc, phases):
    U = synth.random_su3_field(dims, 0.4, 11)
    x = synth.gaussian_spinor(dims, len(phases), 12)
    ctx = make_ctx(P, dims, bc, precision=1)
    ctx.set_gauge(to_dev(U))
    got = gpu_apply(P, ctx, P.apply_wilson, x, phase=phases, hermitian=True)
    want = np.stack([dirac.hermitian_wilson(U, x[j], M0, oracle_bc(bc), phases[j]) for j in range(len(phases))])
    assert relerr(got, want) < F32_WILSON_TOL
    ctx.close()


def test_wilson_batched_equals_one_by_one(P):
    import torch

    dims = (4, 4, 4, 6)
    U = synth.random_su3_field(dims, 0.3, 2)
    x = synth.gaussian_spinor(dims, 4, 3)
    ctx = make_ctx(P, dims)
    ctx.set_gauge(to_dev(U))
    phases = [0.0, 0.1, -0.3, 0.0]
    batched = gpu_apply(P, ctx, P.apply_wilson, x, phase=phases, hermitian=True)
    for j in range(4):
        one = gpu_apply(P, ctx, P.apply_wilson, x[j:j + 1], phase=[phases[j]], hermitian=True)
        assert np.array_equal(one[0], batched[j])
    ctx.close()


# ---------------------------------------------------------------------------
# sign function and overlap with an exact small space (4^4, degree 200)
# ---------------------------------------------------------------------------

# Q^2 interval for the 4^4 field below: its smallest |Q| is 0.050 (0.059 after removing 8
# modes), so [0.002, 1] holds the whole large-space spectrum and the Chebyshev recurrence
# stays inside [-1, 1].  (An interval that misses part of the spectrum evaluates T_k outside
# [-1, 1], where the recurrence amplifies rounding by cosh(k acosh|y|) and no two
# implementations agree to 1e-12.)
EPS4 = 0.002


@pytest.fixture(scope="module")
def lat4():
    """4^4, links eps = 0.3, seed 0: exact 8 lowest |lambda| eigenvectors of Q (dense)."""
    dims = (4, 4, 4, 4)
    bc = (0, 0, 0, 1)
    U = synth.random_su3_field(dims, 0.3, 0)
    hw = 6.5  # the bound |4 + m0| + 4 the library uses by default
    H = dense.hw_matrix(U, M0, oracle_bc(bc))
    lam, W, lam_all, W_all = dense.low_modes(H, hw, 8)
    V = dense.vectors_to_fields(W, synth.site_shape(dims))
    assert np.sort(np.abs(lam_all))[0] ** 2 > EPS4
    return dict(dims=dims, bc=bc, U=U, hw=hw, lam=lam, V=V, lam_all=lam_all)


def oracle_params(d, degree, eps):
    return ov.OverlapParams(m0=M0, hw_norm=d["hw"], eps=eps, degree=degree, bc=oracle_bc(d["bc"]))


@pytest.mark.parametrize("n_ev", [0, 8])
def test_sign_f64_matches_oracle(P, lat4, n_ev):
    d = lat4
    degree, eps = 200, EPS4
    ctx = make_ctx(P, d["dims"], d["bc"], degree=degree, eps=eps)
    ctx.set_gauge(to_dev(d["U"]))
    small = ov.SmallSpace.empty(synth.site_shape(d["dims"]))
    if n_ev:
        P.deflate(ctx, to_dev(d["V"][:n_ev]), d["lam"][:n_ev])
        small = ov.SmallSpace.from_eigenpairs(d["V"][:n_ev], d["lam"][:n_ev])
    x = synth.gaussian_spinor(d["dims"], 2, 5)
    got = gpu_apply(P, ctx, P.apply_sign_Hw, x)
    p = oracle_params(d, degree, eps)
    want = np.stack([ov.sign_hw(d["U"], x[j], p, small) for j in range(2)])
    assert relerr(got, want) < F64_TOL
    ctx.close()


def test_sign_f64_minimax_matches_oracle(P, lat4):
    """The minimax polynomial (poly_kind = 1): the library's Remez coefficients in the GPU
    recurrence against the oracle's sign function with the oracle's own Remez coefficients."""
    d = lat4
    degree, eps = 200, EPS4
    ctx = P.Context(P.Params(dims=d["dims"], bc=d["bc"], m0=M0, eps=eps, poly_degree=degree, poly_kind=1,
                             max_nrhs=2))
    ctx.set_gauge(to_dev(d["U"]))
    P.deflate(ctx, to_dev(d["V"]), d["lam"])
    x = synth.gaussian_spinor(d["dims"], 2, 5)
    got = gpu_apply(P, ctx, P.apply_sign_Hw, x)
    from oracle import chebyshev

    cm, _ = chebyshev.minimax_coeffs(degree, eps)
    p = ov.OverlapParams(m0=M0, hw_norm=d["hw"], eps=eps, degree=degree, bc=oracle_bc(d["bc"]), coeffs=cm)
    small = ov.SmallSpace.from_eigenpairs(d["V"], d["lam"])
    want = np.stack([ov.sign_hw(d["U"], x[j], p, small) for j in range(2)])
    assert relerr(got, want) < F64_TOL
    ctx.close()


@pytest.mark.parametrize("mass", [0.0, 0.1])
def test_overlap_f64_matches_oracle(P, lat4, mass):
    d = lat4
    degree, eps = 200, EPS4
    ctx = make_ctx(P, d["dims"], d["bc"], degree=degree, eps=eps)
    ctx.set_gauge(to_dev(d["U"]))
    P.deflate(ctx, to_dev(d["V"]), d["lam"])
    small = ov.SmallSpace.from_eigenpairs(d["V"], d["lam"])
    x = synth.gaussian_spinor(d["dims"], 1, 1)
    got = gpu_apply(P, ctx, P.apply_overlap, x, mass=mass)
    want = ov.overlap(d["U"], x[0], mass, oracle_params(d, degree, eps), small)
    assert relerr(got[0], want) < F64_TOL
    ctx.close()


def test_overlap_ragged_lattice_field_phases_random_banks(P):
    """6x4x3x6 (ragged), Dirichlet x and t, three right-hand sides at two field
    phases with a different (random orthonormal) small space for each phase."""
    dims, bc = (6, 4, 3, 6), (2, 0, 0, 2)
    U = synth.random_su3_field(dims, 0.3, 21)
    site = synth.site_shape(dims)
    rng = np.random.default_rng(22)
    banks = {}
    degree, eps, mass = 24, 0.02, 0.05
    ctx = make_ctx(P, dims, bc, degree=degree, eps=eps)
    ctx.set_gauge(to_dev(U))
    for phase, nev in [(0.0, 5), (0.25, 3)]:
        A = rng.standard_normal((12 * 432, nev)) + 1j * rng.standard_normal((12 * 432, nev))
        Qm, _ = np.linalg.qr(A)
        V = dense.vectors_to_fields(Qm, site)
        lam = rng.standard_normal(nev)
        banks[phase] = ov.SmallSpace.from_eigenpairs(V, lam)
        P.deflate(ctx, to_dev(V), lam, phase=phase)
    phases = [0.25, 0.0, 0.25]
    x = synth.gaussian_spinor(dims, 3, 23)
    got = gpu_apply(P, ctx, P.apply_overlap, x, mass=mass, phase=phases)
    p = ov.OverlapParams(m0=M0, hw_norm=6.5, eps=eps, degree=degree, bc=oracle_bc(bc))
    for j in range(3):
        want = ov.overlap(U, x[j], mass, p, banks[phases[j]], phases[j])
        assert relerr(got[j], want) < F64_TOL
    ctx.close()


def test_sign_f32_error_is_stated(P, lat4):
    """FP32 sign(H_w) against the FP64 oracle: degree-200 Clenshaw in single precision."""
    d = lat4
    ctx = make_ctx(P, d["dims"], d["bc"], degree=200, eps=EPS4, precision=1)
    ctx.set_gauge(to_dev(d["U"]))
    P.deflate(ctx, to_dev(d["V"]), d["lam"])
    x = synth.gaussian_spinor(d["dims"], 1, 5)
    got = gpu_apply(P, ctx, P.apply_sign_Hw, x)
    small = ov.SmallSpace.from_eigenpairs(d["V"], d["lam"])
    want = ov.sign_hw(d["U"], x[0], oracle_params(d, 200, EPS4), small)
    err = relerr(got[0], want)
    print(f"FP32 sign(H_w) relative error vs FP64 oracle at n = 200: {err:.3e}")
    assert err < 1e-4
    ctx.close()


def test_missing_bank_for_nonzero_phase_is_an_error(P, lat4):
    d = lat4
    ctx = make_ctx(P, d["dims"], d["bc"])
    ctx.set_gauge(to_dev(d["U"]))
    x = to_dev(synth.gaussian_spinor(d["dims"], 1, 5))
    import torch

    with pytest.raises(P.OvlError) as e:
        P.apply_sign_Hw(ctx, x, torch.empty_like(x), phase=[0.5])
    assert e.value.code == 8
    ctx.close()


# ---------------------------------------------------------------------------
# solver
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("inner", [0, 1])
def test_solve_reaches_tolerance_and_matches_oracle(P, lat4, inner):
    import torch

    d = lat4
    degree, eps, mass, tol = 200, EPS4, 0.1, 1e-10
    ctx = make_ctx(P, d["dims"], d["bc"], degree=degree, eps=eps, inner=inner)
    ctx.set_gauge(to_dev(d["U"]))
    P.deflate(ctx, to_dev(d["V"]), d["lam"])
    b = synth.point_sources(d["dims"], [(0, 1), (3, 2)])
    bd = to_dev(b)
    xd = torch.zeros_like(bd)
    st = P.solve_overlap(ctx, bd, xd, mass, tol=tol)
    x = xd.cpu().numpy()
    assert st.true_residual <= tol
    small = ov.SmallSpace.from_eigenpairs(d["V"], d["lam"])
    p = oracle_params(d, degree, eps)
    for j in range(2):
        r = b[j] - ov.overlap(d["U"], x[j], mass, p, small)
        assert np.linalg.norm(r) / np.linalg.norm(b[j]) <= 2 * tol  # oracle's own operator
    print(f"inner precision {inner}: outer {st.outer_iters}, inner {st.inner_iters}, residual {st.true_residual:.2e}")
    ctx.close()


@pytest.mark.parametrize("mass", [0.1, 0.02])
def test_adaptive_order_solve_matches_oracle(P, lat4, mass):
    """Mixed solve with the per-cycle polynomial degree (adaptive order): the true residual,
    always taken at the full degree, reaches the tolerance against the oracle's operator, and
    the inner cycles ran at lower degrees."""
    import torch

    d = lat4
    degree, eps, tol = 200, EPS4, 1e-10
    ctx = P.Context(P.Params(dims=d["dims"], bc=d["bc"], m0=M0, eps=eps, poly_degree=degree, precision=1,
                             inner_precision=1, max_nrhs=4, adaptive_order=1))
    ctx.set_gauge(to_dev(d["U"]))
    P.deflate(ctx, to_dev(d["V"]), d["lam"])
    b = synth.point_sources(d["dims"], [(0, 1), (3, 2)])
    bd = to_dev(b)
    xd = torch.zeros_like(bd)
    st = P.solve_overlap(ctx, bd, xd, mass, tol=tol)
    x = xd.cpu().numpy()
    assert st.true_residual <= tol
    small = ov.SmallSpace.from_eigenpairs(d["V"], d["lam"])
    p = oracle_params(d, degree, eps)
    for j in range(2):
        r = b[j] - ov.overlap(d["U"], x[j], mass, p, small)
        assert np.linalg.norm(r) / np.linalg.norm(b[j]) <= 2 * tol
    degrees = [int(t.split("n ")[1].split(",")[0]) for t in ctx.last_info.split("|")[1:]]
    print(f"adaptive order, m = {mass}: cycles at degrees {degrees}; {ctx.last_info}")
    assert min(degrees) < degree
    ctx.close()


def test_eigensolver_matches_dense(P, lat4):
    d = lat4
    ctx = make_ctx(P, d["dims"], d["bc"])
    ctx.set_gauge(to_dev(d["U"]))
    lam, V = P.eigensolve_Q(ctx, 8, tol=1e-11, max_iter=200, want_vectors=True)
    assert np.allclose(np.sort(lam), np.sort(d["lam"]), atol=1e-10)
    Vh = V.cpu().numpy()
    for i in range(8):
        r = dirac.hermitian_wilson(d["U"], Vh[i], M0, oracle_bc(d["bc"])) / d["hw"] - lam[i] * Vh[i]
        assert np.linalg.norm(r) < 1e-10
    ctx.close()


def test_eigensolver_in_column_chunks_matches_dense(P, lat4):
    """The same eigenpairs with a working-set budget that splits the filter and the residual pass
    into ragged chunks of the 24-column block: 5 columns at a time in FP32, 2 in FP64 (the
    recurrence acts on each column alone, so only rounding may differ)."""
    d = lat4
    ctx = make_ctx(P, d["dims"], d["bc"])
    ctx.set_gauge(to_dev(d["U"]))
    vb32 = 12 * int(np.prod(d["dims"])) * 8
    ctx.set_eigensolver_memory(3 * 5 * vb32)
    lam, V = P.eigensolve_Q(ctx, 8, tol=1e-11, max_iter=200, want_vectors=True)
    assert "block 24" in ctx.last_info
    assert np.allclose(np.sort(lam), np.sort(d["lam"]), atol=1e-10)
    Vh = V.cpu().numpy()
    for i in range(8):
        r = dirac.hermitian_wilson(d["U"], Vh[i], M0, oracle_bc(d["bc"])) / d["hw"] - lam[i] * Vh[i]
        assert np.linalg.norm(r) < 1e-10
    ctx.close()


def test_eigensolver_fp32_level_target_with_warm_start(P, lat4):
    """A target of 2e-6 keeps the whole iteration in FP32; the n_ev wanted vectors are widened to FP64
    and orthonormalised there.  A second field phase then starts from the first phase's bank.  Both
    in ragged chunks of 5 columns, against the oracle's dense spectrum and Wilson operator at that
    phase: eigenvalues to FP32 level, residuals within the target plus the FP64 re-orthonormalisation
    (FP32 rounding of the vectors, ~1e-7), and FP64-orthonormal vectors."""
    d = lat4
    ctx = make_ctx(P, d["dims"], d["bc"])
    ctx.set_gauge(to_dev(d["U"]))
    ctx.set_eigensolver_memory(3 * 5 * 12 * int(np.prod(d["dims"])) * 8)
    for phase in (0.0, 0.2):
        lam, V = P.eigensolve_Q(ctx, 8, phase=phase, tol=2e-6, max_iter=300, want_vectors=True)
        info = ctx.last_info
        assert "f64/" not in info, info
        assert ("warm start" in info) == (phase != 0.0), info
        H = dense.hw_matrix(d["U"], M0, oracle_bc(d["bc"]), phase)
        want, _, _, _ = dense.low_modes(H, d["hw"], 8)
        assert np.allclose(np.sort(lam), np.sort(want), atol=1e-6), (lam, want)
        Vh = V.cpu().numpy()
        G = np.array([[dirac.inner(Vh[i], Vh[j]) for j in range(8)] for i in range(8)])
        assert np.abs(G - np.eye(8)).max() < 1e-12
        for i in range(8):
            r = dirac.hermitian_wilson(d["U"], Vh[i], M0, oracle_bc(d["bc"]), phase) / d["hw"] - lam[i] * Vh[i]
            assert np.linalg.norm(r) < 3e-6, (phase, i, np.linalg.norm(r))
    ctx.close()


# ---------------------------------------------------------------------------
# sign function at the measured workload's polynomial (n = 527, sqrt(eps) = 0.02)
# ---------------------------------------------------------------------------

def test_sign_f64_at_the_bench_degree_matches_oracle(P):
    """FP64 sign(H_w) on 8^4 with the bench's polynomial (minimax, n = 527 on [4e-4, 1]) and
    boundary conditions, links exp(i 0.2 H) as in the 16^3 x 32 workload, and a 16-vector small
    space that is not an invariant subspace (random orthonormal vectors, mixed signs), so that the
    projection, the 1054 Wilson applications of the recurrence and the final Q all enter.  The
    lowest |Q| of such a near-free field (the doublers, ~0.08) lies inside the polynomial's
    interval, so the recurrence stays in [-1, 1] and the two implementations agree to 1e-12."""
    from oracle import chebyshev

    dims, bc, degree, eps, n_ev = (8, 8, 8, 8), (0, 0, 0, 1), 527, 0.02 ** 2, 16
    U = synth.random_su3_field(dims, 0.2, 0)
    rng = np.random.default_rng(21)
    site = synth.site_shape(dims) + (4, 3)
    A = rng.standard_normal((n_ev, int(np.prod(site)))) + 1j * rng.standard_normal((n_ev, int(np.prod(site))))
    Qm, _ = np.linalg.qr(A.T)
    V = np.ascontiguousarray(Qm.T.reshape((n_ev,) + site))
    lam = np.where(np.arange(n_ev) % 3 == 0, -1.0, 1.0) * (0.05 + 0.001 * np.arange(n_ev))
    ctx = P.Context(P.Params(dims=dims, bc=bc, m0=M0, eps=eps, poly_degree=degree, poly_kind=1, max_nrhs=1))
    ctx.set_gauge(to_dev(U))
    P.deflate(ctx, to_dev(V), lam)
    x = synth.gaussian_spinor(dims, 1, 5)
    got = gpu_apply(P, ctx, P.apply_sign_Hw, x)
    cm, _ = chebyshev.minimax_coeffs(degree, eps)
    p = ov.OverlapParams(m0=M0, hw_norm=ctx.hw_norm, eps=eps, degree=degree, bc=oracle_bc(bc), coeffs=cm)
    want = ov.sign_hw(U, x[0], p, ov.SmallSpace.from_eigenpairs(V, lam))
    assert relerr(got[0], want) < F64_TOL
    ctx.close()
