"""The multi-mass solve (Sec. 3.2, the multi-mass CG) against the oracle and single-mass solves.

On a 4^4 lattice with a field phase and the oracle's exact small space (8 H_w modes), every
mass's solution must reach the tolerance against the oracle's D(m), agree with the library's
own single-mass solve, and (without D_ov deflation, where the shared first cycle replaces one
cycle per mass) cost fewer sign applications than the single-mass solves together.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from oracle import dense
from oracle import overlap as ov

pytestmark = pytest.mark.gpu

M0 = -1.5
HW = 6.5
EPS4 = 0.002  # covers the 4^4 field's large-space spectrum once 8 modes are exact
DEGREE = 200
PHASE = 0.2
TOL = 1e-10
MASSES = [0.02, 0.05, 0.1, 0.4]


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
def lat():
    dims, bc = (4, 4, 4, 4), (0, 0, 0, 1)
    U = synth.random_su3_field(dims, 0.3, 0)
    H = dense.hw_matrix(U, M0, (1.0, 1.0, 1.0, -1.0), PHASE)
    lam, W, lam_all, _ = dense.low_modes(H, HW, 8)
    assert np.sort(np.abs(lam_all))[8] ** 2 > EPS4
    V = dense.vectors_to_fields(W, synth.site_shape(dims))
    return dict(dims=dims, bc=bc, U=U, lam=lam, V=V)


def make_ctx(P, d, adaptive):
    ctx = P.Context(P.Params(dims=d["dims"], bc=d["bc"], m0=M0, eps=EPS4, poly_degree=DEGREE, precision=1,
                             inner_precision=1, max_nrhs=2, adaptive_order=adaptive))
    ctx.set_gauge(dev(d["U"]))
    P.deflate(ctx, dev(d["V"]), d["lam"], phase=PHASE)
    return ctx


@pytest.mark.parametrize("deflated,adaptive", [(False, 0), (True, 1)])
def test_multimass_matches_oracle_and_single_mass_solves(P, lat, deflated, adaptive):
    import torch

    d = lat
    b = synth.point_sources(d["dims"], [(0, 1), (3, 2)])
    phases = [PHASE, PHASE]
    ctx = make_ctx(P, d, adaptive)
    if deflated:
        for chi in (1, -1):
            P.eigensolve_overlap(ctx, 16, chirality=chi, phase=PHASE)
    X = torch.full((len(MASSES),) + b.shape, float("nan"), dtype=torch.complex128, device="cuda")  # output only
    sts = P.solve_overlap_multimass(ctx, dev(b), X, MASSES, tol=TOL, phase=phases)
    print(f"deflated {deflated}: {ctx.last_info}")
    for st in sts:
        assert st.status == 0 and st.true_residual <= TOL
    single = 0
    for i, m in enumerate(MASSES):
        x1 = torch.zeros_like(dev(b))
        st1 = P.solve_overlap(ctx, dev(b), x1, m, tol=TOL, phase=phases)
        single += st1.sign_applies
        rel = float((X[i] - x1).norm() / x1.norm())
        assert rel < 1e-7, (m, rel)
    multi = sum(st.sign_applies for st in sts)
    print(f"sign applications: multi-mass {multi}, single-mass solves {single}")
    if not deflated:
        assert multi < single
    ctx.close()
    small = ov.SmallSpace.from_eigenpairs(d["V"], d["lam"])
    p = ov.OverlapParams(m0=M0, hw_norm=HW, eps=EPS4, degree=DEGREE, bc=(1.0, 1.0, 1.0, -1.0))
    Xh = X.cpu().numpy()
    for i in (0, len(MASSES) - 1):
        for j in range(2):
            r = b[j] - ov.overlap(d["U"], Xh[i, j], MASSES[i], p, small, PHASE)
            assert np.linalg.norm(r) / np.linalg.norm(b[j]) <= 2 * TOL


def test_multimass_zero_source_repeated_and_negative_masses(P, lat):
    """A zero right-hand side gives exact zeros for every mass; repeated masses and a negative
    mass (the shift depends on m^2, the correction D(m)^+ on m itself) solve like the others."""
    import torch

    d = lat
    b = np.concatenate([synth.point_sources(d["dims"], [(1, 0)]), np.zeros_like(synth.point_sources(d["dims"], [(0, 0)]))])
    masses = [0.3, -0.1, 0.3]
    ctx = make_ctx(P, d, 0)
    X = torch.empty((len(masses),) + b.shape, dtype=torch.complex128, device="cuda")
    sts = P.solve_overlap_multimass(ctx, dev(b), X, masses, tol=TOL, phase=[PHASE, PHASE])
    assert all(st.status == 0 and st.true_residual <= TOL for st in sts)
    assert float(X[:, 1].abs().max()) == 0.0
    assert float((X[0] - X[2]).abs().max()) <= 1e-9 * float(X[0].abs().max())
    small = ov.SmallSpace.from_eigenpairs(d["V"], d["lam"])
    p = ov.OverlapParams(m0=M0, hw_norm=HW, eps=EPS4, degree=DEGREE, bc=(1.0, 1.0, 1.0, -1.0))
    r = b[0] - ov.overlap(d["U"], X[1, 0].cpu().numpy(), -0.1, p, small, PHASE)
    assert np.linalg.norm(r) / np.linalg.norm(b[0]) <= 2 * TOL
    ctx.close()
