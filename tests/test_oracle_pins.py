"""Pins of the CPU oracle against things other than itself.

Each check compares the oracle with a closed form, an invariant, a library
routine, a brute-force construction or a number the paper prints, so that a
plausible mistake (a dropped term, a wrong sign or index, a transposed or
missing dagger) fails at least one of them.  ``test_oracle_mutations.py``
plants such mistakes in the oracle and checks that these pins catch them.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import chebyshev, dense, dirac, solver
from oracle import overlap as ov

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
M0 = -1.5


def _chiral_gammas():
    """The chosen convention written independently of the oracle: gamma_k =
    [[0, -i sigma_k], [i sigma_k, 0]] (k = x, y, z), gamma_t = [[0, 1], [1, 0]]."""
    sig = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    g = []
    for s in sig:
        m = np.zeros((4, 4), np.complex128)
        m[:2, 2:] = -1j * s
        m[2:, :2] = 1j * s
        g.append(m)
    m = np.zeros((4, 4), np.complex128)
    m[:2, 2:] = m[2:, :2] = np.eye(2)
    g.append(m)
    return np.array(g)


TEST_GAMMA = _chiral_gammas()


# --------------------------------------------------------------------------
# helpers shared with the mutation tests
# --------------------------------------------------------------------------

def plane_wave(dims, p, u):
    """psi(n) = exp(i p.n) u for n = (x, y, z, t); u a 4x3 spin-colour vector."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return ph[..., None, None] * u


def free_wilson_symbol(p, m0):
    """D_w(p) = m0 + sum(1 - cos p) + i sum gamma_mu sin p_mu (4x4 spin matrix)."""
    M = m0 + sum(1.0 - math.cos(q) for q in p)
    return M * np.eye(4) + 1j * sum(math.sin(q) * TEST_GAMMA[mu] for mu, q in enumerate(p))


def free_plane_wave_error(dims, bc, momenta, seed=3):
    """max relative error of the oracle's D_w on plane waves against the closed form."""
    rng = np.random.default_rng(seed)
    U = synth.unit_gauge(dims)
    worst = 0.0
    for p in momenta:
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = plane_wave(dims, p, u)
        got = dirac.wilson(U, psi, M0, bc)
        want = plane_wave(dims, p, free_wilson_symbol(p, M0) @ u)
        worst = max(worst, np.abs(got - want).max() / np.abs(want).max())
    return worst


def lattice_momenta(dims, antiperiodic_t, count, seed=5):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        k = [rng.integers(0, L) for L in dims]
        p = [2 * math.pi * k[mu] / dims[mu] for mu in range(3)]
        p.append(((2 * k[3] + 1) if antiperiodic_t else 2 * k[3]) * math.pi / dims[3])
        out.append(p)
    return out


def gauge_covariance_error(dims, bc, phase, seed=0):
    """|| D[U^g] (g psi) - g D[U] psi || / || D[U] psi ||, U^g_mu(n) = g(n) U_mu(n) g(n+mu)^+."""
    U = synth.random_su3_field(dims, 0.5, seed)
    g = synth.random_gauge_transform(dims, seed + 11)
    psi = synth.gaussian_spinor(dims, 1, seed + 2)[0]
    Ug = np.empty_like(U)
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=3 - mu)
        Ug[mu] = g @ U[mu] @ np.conj(np.swapaxes(g_fwd, -1, -2))
    lhs = dirac.wilson(Ug, dirac.colour_mult(g, psi), M0, bc, phase)
    rhs = dirac.colour_mult(g, dirac.wilson(U, psi, M0, bc, phase))
    return np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs)


def hermiticity_error(dims, bc, phase, seed=0):
    """|<a, H_w b> - <H_w a, b>| / (|a| |H_w b|)."""
    U = synth.random_su3_field(dims, 0.4, seed)
    a, b = synth.gaussian_spinor(dims, 2, seed + 1)
    ha = dirac.hermitian_wilson(U, a, M0, bc, phase)
    hb = dirac.hermitian_wilson(U, b, M0, bc, phase)
    return abs(dirac.inner(a, hb) - dirac.inner(ha, b)) / (dirac.norm(a) * dirac.norm(hb))


def brute_wilson_matrix(U, m0, bcf, phase):
    """D_w written out block by block with explicit site loops (no array shifts)."""
    lt, lz, ly, lx = U.shape[1:5]
    L = (lx, ly, lz, lt)
    nsite = lx * ly * lz * lt

    def idx(c):
        x, y, z, t = c
        return ((t * lz + z) * ly + y) * lx + x

    D = np.zeros((12 * nsite, 12 * nsite), dtype=np.complex128)
    I4 = np.eye(4)
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    n = (x, y, z, t)
                    i = idx(n)
                    D[12 * i:12 * i + 12, 12 * i:12 * i + 12] += (4 + m0) * np.eye(12)
                    for mu in range(4):
                        f = list(n)
                        f[mu] += 1
                        fac = 1.0
                        if f[mu] == L[mu]:
                            f[mu], fac = 0, bcf[mu]
                        u = U[mu, t, z, y, x]
                        if mu == 0:
                            u = u * np.exp(1j * phase * t)
                        j = idx(f)
                        D[12 * i:12 * i + 12, 12 * j:12 * j + 12] += -0.5 * fac * np.kron(I4 - TEST_GAMMA[mu], u)
                        b = list(n)
                        b[mu] -= 1
                        fac = 1.0
                        if b[mu] < 0:
                            b[mu], fac = L[mu] - 1, bcf[mu]
                        xb, yb, zb, tb = b
                        ub = U[mu, tb, zb, yb, xb]
                        if mu == 0:
                            ub = ub * np.exp(1j * phase * tb)
                        j = idx(b)
                        D[12 * i:12 * i + 12, 12 * j:12 * j + 12] += -0.5 * fac * np.kron(I4 + TEST_GAMMA[mu], ub.conj().T)
    return D


def brute_force_error(dims, bc, phase, seed=4):
    U = synth.random_su3_field(dims, 0.6, seed)
    site = synth.site_shape(dims)
    A = dense.operator_matrix(lambda v: dirac.wilson(U, v, M0, bc, phase), site + (4, 3))
    B = brute_wilson_matrix(U, M0, dirac.bc_factors(bc), phase)
    return np.abs(A - B).max()


def small_lattice_setup(dims=(2, 2, 2, 2), n_ev=8, bc=(1, 1, 1, -1), phase=0.0, seed=0, eps_field=0.3, degree=200):
    """Random field on a tiny lattice with its exact spectrum and an overlap parameter set
    whose interval [eps, 1] covers every eigenvalue outside the small space."""
    U = synth.random_su3_field(dims, eps_field, seed)
    H = dense.hw_matrix(U, M0, bc, phase)
    lam_all, W_all = np.linalg.eigh(H)
    hw_norm = float(np.abs(lam_all).max())
    lq = np.sort(np.abs(lam_all / hw_norm))
    eps = (0.9 * lq[n_ev]) ** 2
    params = ov.OverlapParams(m0=M0, hw_norm=hw_norm, eps=eps, degree=degree, bc=bc)
    lam, W, lam_q, W_all = dense.low_modes(H, hw_norm, n_ev)
    small = ov.SmallSpace.from_eigenpairs(dense.vectors_to_fields(W, synth.site_shape(dims)), lam)
    return U, params, small, lam_q, W_all, phase


def dense_split_error(setup, seed=9):
    """oracle sign(H_w) x against the exact spectral form of the same split operator."""
    U, params, small, lam_q, W_all, phase = setup
    dims = U.shape[1:5][::-1]
    x = synth.gaussian_spinor(dims, 1, seed)[0]
    got = ov.sign_hw(U, x, params, small, phase)
    F = dense.split_sign_matrix(lam_q, W_all, small.V.shape[0], params.coeffs, params.eps)
    want = (F @ x.ravel()).reshape(x.shape)
    return np.linalg.norm(got - want) / np.linalg.norm(want)


# --------------------------------------------------------------------------
# gamma matrices
# --------------------------------------------------------------------------

def test_gamma_clifford_algebra_and_gamma5():
    assert np.array_equal(dirac.GAMMA, TEST_GAMMA)
    g = dirac.GAMMA
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T)
        for b in range(4):
            assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2.0 * (a == b) * np.eye(4), atol=1e-15)
        assert np.allclose(g[a] @ dirac.GAMMA5 + dirac.GAMMA5 @ g[a], 0.0)
    assert np.allclose(dirac.GAMMA5, np.diag([1, 1, -1, -1]))


# --------------------------------------------------------------------------
# Wilson operator
# --------------------------------------------------------------------------

@pytest.mark.parametrize("antiperiodic_t", [False, True])
def test_free_field_plane_waves_are_eigenvectors(antiperiodic_t):
    dims = (4, 6, 2, 8)
    bc = (1, 1, 1, -1 if antiperiodic_t else 1)
    err = free_plane_wave_error(dims, bc, lattice_momenta(dims, antiperiodic_t, 12))
    assert err < 1e-13


def test_free_field_spectrum_2x4_closed_form():
    """Free field, periodic 2^4: momenta are 0 or pi, so H_w(p) = gamma5 M with
    M = m0 + 2 (#pi components); ||H_w|| = 6.5 and the smallest |eigenvalue| 0.5."""
    dims = (2, 2, 2, 2)
    H = dense.hw_matrix(synth.unit_gauge(dims), M0)
    got = np.sort(np.abs(np.linalg.eigvalsh(H)))
    want = []
    for k in range(5):
        want += [abs(M0 + 2 * k)] * (math.comb(4, k) * 12)
    assert np.allclose(got, np.sort(want), atol=1e-13)
    assert got[-1] == pytest.approx(6.5) and got[0] == pytest.approx(0.5)


@pytest.mark.parametrize("bc,phase", [((1, 1, 1, 1), 0.0), ((1, 1, 1, -1), 0.3), ((0, 1, 1, 0), -0.7)])
def test_gauge_covariance(bc, phase):
    assert gauge_covariance_error((4, 2, 6, 4), bc, phase) < 1e-13


@pytest.mark.parametrize("bc,phase", [((1, 1, 1, -1), 0.0), ((0, 1, 1, 0), 0.25), ((-1, 1, 0, 1), -1.1)])
def test_hw_is_hermitian(bc, phase):
    assert hermiticity_error((4, 4, 2, 6), bc, phase) < 1e-14


@pytest.mark.parametrize("dims,bc,phase", [((2, 2, 2, 2), (1, 1, 1, -1), 0.0),
                                           ((2, 2, 2, 4), (0, 1, -1, 0), 0.4),
                                           ((3, 2, 2, 2), (1, 0, 1, 1), -0.9)])
def test_wilson_matches_brute_force_blocks(dims, bc, phase):
    """Tiny lattices, including 2^4 where forward and backward neighbours coincide."""
    assert brute_force_error(dims, bc, phase) < 1e-14


def test_dirichlet_blocks_boundary_hops():
    dims = (4, 4, 4, 6)
    U = synth.random_su3_field(dims, 0.3, 2)
    psi = np.zeros(synth.site_shape(dims) + (4, 3), np.complex128)
    psi[0] = synth.gaussian_spinor(dims, 1, 3)[0][0]  # supported on t = 0 only
    out_d = dirac.wilson(U, psi, M0, (1, 1, 1, 0))
    out_p = dirac.wilson(U, psi, M0, (1, 1, 1, 1))
    assert np.abs(out_d[-1]).max() == 0.0  # nothing hops from t = 0 back to t = Lt - 1
    assert np.abs(out_p[-1]).max() > 0.1 * np.abs(psi).max()
    assert np.allclose(out_d[:2], out_p[:2], atol=1e-15)


# --------------------------------------------------------------------------
# polynomial and the error law (eq. 2)
# --------------------------------------------------------------------------

def test_paper_error_law_values():
    dl = GOLD["delta_law"]
    assert (chebyshev.DELTA_A, chebyshev.DELTA_B) == (dl["A"], dl["b"])
    o = GOLD["order_without_small_space"]
    n = chebyshev.order_for_delta(o["delta"], o["sqrt_eps"])
    assert 0.5 * o["order"] < n < 2 * o["order"]  # "~1e5"
    f1 = GOLD["figure1_example"]
    d = chebyshev.delta_law(f1["n"], f1["sqrt_eps"])
    assert round(d, 1) == f1["delta"]  # 0.08 rounds to the caption's 0.1
    # orders of the synthetic workloads at delta = 1e-10 (derived from eq. 2)
    assert round(chebyshev.order_for_delta(1e-10, 0.02)) == 527
    assert round(chebyshev.order_for_delta(1e-10, 0.01)) == 1054


def test_vectors_per_gpu_arithmetic():
    """Sec. 3: 36 FP64 spin-colour vectors on 24^3 x 64 fill a 6 GB GPU."""
    v = GOLD["vectors_per_gpu"]
    sites = int(np.prod(v["lattice"]))
    nbytes = v["vectors"] * sites * 12 * 16
    assert 0.9 * v["gpu_gb"] * 1e9 < nbytes < 1.1 * v["gpu_gb"] * 1e9


@pytest.mark.parametrize("n,eps", [(13, 0.06 ** 2), (64, 0.01), (200, 4e-4), (527, 4e-4)])
def test_coeffs_match_numpy_chebinterpolate(n, eps):
    c = chebyshev.chebyshev_coeffs(n, eps)

    def g(y):
        return 1.0 / np.sqrt(((1 - eps) * y + 1 + eps) / 2)

    ref = np.polynomial.chebyshev.chebinterpolate(g, n)
    assert np.abs(c - ref).max() < 1e-12 * np.abs(ref).max()


def test_eval_poly_matches_numpy_chebval():
    c = chebyshev.chebyshev_coeffs(77, 0.003)
    x = np.linspace(0.003, 1.0, 997)
    ref = np.polynomial.chebyshev.chebval(chebyshev.to_y(x, 0.003), c)
    assert np.abs(chebyshev.eval_poly(c, 0.003, x) - ref).max() < 1e-12 * np.abs(ref).max()


def test_error_law_shape():
    """Measured delta of the interpolant follows eq. 2: same decay rate (b within
    [1.9, 2.2]) and a prefactor within 3x of the paper's A."""
    se = 0.02
    ns = np.arange(100, 501, 50)
    deltas = np.array([chebyshev.approximation_error(chebyshev.chebyshev_coeffs(int(n), se * se), se * se) for n in ns])
    slope, icpt = np.polyfit(ns * se, np.log(deltas), 1)
    assert 1.9 <= -slope <= 2.2
    for n, d in zip(ns, deltas):
        assert 1.0 / 3.0 <= d / chebyshev.delta_law(n, se) <= 3.0
    f1 = GOLD["figure1_example"]
    c = chebyshev.chebyshev_coeffs(f1["n"], f1["sqrt_eps"] ** 2)
    d13 = chebyshev.approximation_error(c, f1["sqrt_eps"] ** 2)
    assert f1["delta"] / 3 < d13 < f1["delta"] * 3


# --------------------------------------------------------------------------
# sign function and overlap on tiny lattices (dense references)
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def setup_2x4():
    return small_lattice_setup()


@pytest.fixture(scope="module")
def setup_2x4_field():
    """Dirichlet x and t with a background-field phase (the E != 0 operators)."""
    return small_lattice_setup(bc=(0, 1, 1, 0), phase=0.37, seed=5)


@pytest.mark.parametrize("which", ["setup_2x4", "setup_2x4_field"])
def test_sign_matches_dense_split_operator(which, request):
    assert dense_split_error(request.getfixturevalue(which)) < 1e-12


def test_sign_close_to_exact_sign_and_squares_to_one(setup_2x4):
    U, params, small, lam_q, W_all, _ = setup_2x4
    delta = chebyshev.approximation_error(params.coeffs, params.eps)
    x = synth.gaussian_spinor((2, 2, 2, 2), 1, 21)[0]
    s = ov.sign_hw(U, x, params, small)
    exact = (dense.exact_sign_matrix(lam_q, W_all) @ x.ravel()).reshape(x.shape)
    assert np.linalg.norm(s - exact) <= 2 * delta + 1e-13
    ss = ov.sign_hw(U, s, params, small)
    assert np.linalg.norm(ss - x) <= 3 * delta + 1e-13


def test_sign_dag_is_adjoint_for_any_orthonormal_set():
    """With a random orthonormal V (not eigenvectors) sign_hw is not Hermitian;
    sign_hw_dag must still be its exact adjoint."""
    dims = (2, 2, 2, 4)
    U = synth.random_su3_field(dims, 0.3, 3)
    site = synth.site_shape(dims)
    rng = np.random.default_rng(4)
    A = rng.standard_normal((12 * 32, 5)) + 1j * rng.standard_normal((12 * 32, 5))
    Qm, _ = np.linalg.qr(A)
    small = ov.SmallSpace(dense.vectors_to_fields(Qm, site), np.array([1, -1, -1, 1, 1.0]))
    p = ov.OverlapParams(m0=M0, hw_norm=6.0, eps=0.01, degree=40, bc=(1, 1, 1, -1))
    a, b = synth.gaussian_spinor(dims, 2, 8)
    lhs = dirac.inner(a, ov.sign_hw(U, b, p, small))
    rhs = dirac.inner(ov.sign_hw_dag(U, a, p, small), b)
    assert abs(lhs - rhs) < 1e-13
    herm_gap = abs(lhs - dirac.inner(ov.sign_hw(U, a, p, small), b))
    assert herm_gap > 1e-6  # the non-Hermitian case really is exercised


def test_overlap_ginsparg_wilson_gamma5_hermiticity_normality(setup_2x4):
    U, params, small, lam_q, W_all, _ = setup_2x4
    delta = chebyshev.approximation_error(params.coeffs, params.eps)
    x = synth.gaussian_spinor((2, 2, 2, 2), 1, 31)[0]
    g5 = dirac.gamma5

    def D(v):
        return ov.overlap(U, v, 0.0, params, small)

    def Dd(v):
        return ov.overlap_dag(U, v, 0.0, params, small)

    gw = g5(D(x)) + D(g5(x)) - D(g5(D(x)))
    assert np.linalg.norm(gw) <= 4 * delta + 1e-12
    assert np.linalg.norm(Dd(x) - g5(D(g5(x)))) < 1e-12
    assert np.linalg.norm(D(Dd(x)) - Dd(D(x))) <= 4 * delta + 1e-12


def test_overlap_spectrum_on_unit_circle(setup_2x4):
    U, params, small, _, _, _ = setup_2x4
    site = synth.site_shape((2, 2, 2, 2))
    Dm = dense.operator_matrix(lambda v: ov.overlap(U, v, 0.0, params, small), site + (4, 3))
    ev = np.linalg.eigvals(Dm)
    assert np.abs(np.abs(ev - 1.0) - 1.0).max() < 1e-10


def test_massive_overlap_normalisation(setup_2x4):
    """D(m) = (1 - m/2) D_ov + m: D(m=2) is 2 times the identity for any sign function."""
    U, params, small, _, _, _ = setup_2x4
    x = synth.gaussian_spinor((2, 2, 2, 2), 1, 41)[0]
    assert np.linalg.norm(ov.overlap(U, x, 2.0, params, small) - 2.0 * x) < 1e-14


@pytest.mark.parametrize("mass", [0.02, 0.3, -0.1, 1.5])
def test_massive_normal_operator_is_a_shifted_family(setup_2x4, mass):
    """With sign^2 = 1 and sign Hermitian, D(m) D(m)^+ = (1 - m^2/4) D_ov D_ov^+ + m^2, and on a
    chiral sector P_s D(m) D(m)^+ P_s = k (A0 + (m^2 / k) P_s), A0 = 2 P_s (1 + s sign) P_s,
    k = 1 - m^2/4: one operator shifted by a constant per mass, the form that the chiral-sector
    CG and the multi-mass CG solve.  Exact with the exact sign; within a few delta with the
    oracle's polynomial D(m) and D(m)^+."""
    U, params, small, lam_q, W_all, _ = setup_2x4
    n = W_all.shape[0]
    G5 = np.kron(np.eye(n // 12), np.kron(dirac.GAMMA5, np.eye(3)))
    S = dense.exact_sign_matrix(lam_q, W_all)
    I = np.eye(n)
    Dov = I + G5 @ S
    Dm = (1 - mass / 2) * Dov + mass * I
    k = 1 - mass * mass / 4
    assert np.abs(Dm @ Dm.conj().T - (k * Dov @ Dov.conj().T + mass * mass * I)).max() < 1e-12
    for s in (1, -1):
        Ps = (I + s * G5) / 2
        A0 = Ps @ (2 * (I + s * S)) @ Ps
        assert np.abs(Ps @ Dm @ Dm.conj().T @ Ps - k * (A0 + (mass * mass / k) * Ps)).max() < 1e-12
    delta = chebyshev.approximation_error(params.coeffs, params.eps)
    assert shifted_family_error(setup_2x4, mass) <= 8 * delta + 1e-12


def shifted_family_error(setup, mass):
    """max over chiral sectors s of |P_s D(m) D(m)^+ x_s - [(1 - m^2/4) 2 (x_s + s P_s sign x_s) + m^2 x_s]|
    / |x_s| for the oracle's polynomial D(m), D(m)^+ and sign (x_s = P_s x, x Gaussian)."""
    U, params, small, _, W_all, _ = setup
    n = W_all.shape[0]
    G5 = np.kron(np.eye(n // 12), np.kron(dirac.GAMMA5, np.eye(3)))
    I = np.eye(n)
    k = 1 - mass * mass / 4
    x = synth.gaussian_spinor((2, 2, 2, 2), 1, 61)[0]
    worst = 0.0
    for s in (1, -1):
        Ps = (I + s * G5) / 2
        xs = (Ps @ x.ravel()).reshape(x.shape)
        y = ov.overlap(U, ov.overlap_dag(U, xs, mass, params, small), mass, params, small)
        sx = ov.sign_hw(U, xs, params, small)
        want = k * 2 * (xs + s * (Ps @ sx.ravel()).reshape(x.shape)) + mass * mass * xs
        got = (Ps @ y.ravel()).reshape(x.shape)
        worst = max(worst, np.linalg.norm(got - want) / np.linalg.norm(xs))
    return worst


def test_free_field_overlap_closed_form():
    """Free field, periodic 4^4: D_ov(p) = 1 + D_w(p) / sqrt(M^2 + sum sin^2 p)."""
    dims = (4, 4, 4, 4)
    U = synth.unit_gauge(dims)
    # |H_w| spans [0.5, 6.5] here; sqrt(eps) = 0.07 < 0.5 / 6.5
    params = ov.OverlapParams(m0=M0, hw_norm=6.5, eps=0.005, degree=240)
    small = ov.SmallSpace.empty(synth.site_shape(dims))
    rng = np.random.default_rng(6)
    for p in lattice_momenta(dims, False, 6, seed=8):
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = plane_wave(dims, p, u)
        Dp = free_wilson_symbol(p, M0)
        omega = math.sqrt(np.real(np.trace(Dp.conj().T @ Dp)) / 4)
        want = plane_wave(dims, p, (np.eye(4) + Dp / omega) @ u)
        got = ov.overlap(U, psi, 0.0, params, small)
        assert np.abs(got - want).max() < 1e-11


# --------------------------------------------------------------------------
# solver
# --------------------------------------------------------------------------

def test_cgne_matches_dense_solve(setup_2x4):
    U, params, small, _, _, _ = setup_2x4
    mass = 0.1
    site = synth.site_shape((2, 2, 2, 2))
    b = synth.gaussian_spinor((2, 2, 2, 2), 1, 51)[0]
    x, iters, res = solver.cgne(lambda v: ov.overlap(U, v, mass, params, small),
                                lambda v: ov.overlap_dag(U, v, mass, params, small), b, tol=1e-11)
    assert res <= 1e-11 and iters > 5
    Dm = dense.operator_matrix(lambda v: ov.overlap(U, v, mass, params, small), site + (4, 3))
    x_ref = np.linalg.solve(Dm, b.ravel()).reshape(b.shape)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-9
