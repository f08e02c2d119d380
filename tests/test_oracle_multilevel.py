"""Pins of the oracle's multilevel recursion (the two-level method applied to its own coarse
system, Sec. 3 and Sec. 6.4): the generic stencil level against the pinned fine classes and against
dense matrices, and the nested iteration matrix of the three-level V-cycle."""
import numpy as np
import pytest

from oracle.aggregation import Aggregation
from oracle.coarse import CoarseOperator
from oracle.dirac import DiracOperator, gamma5_field
from oracle.mg import Params, TwoLevel
from oracle.multilevel import (MultiLevel, StencilAggregation, StencilCoarse, StencilOperator, StencilSAP,
                               StencilTwoLevel, _block_sum)
from oracle.sap import SAP
from paper_1303_1377_gb300 import synth

DIMS = (4, 4, 4, 4)
# level 0: 4^4 fine sites, aggregates 2x2x2x1 -> level 1: 2x2x2x4 sites of 2N0 = 4 components;
# level-1 aggregates 1x1x1x2 -> level 2: 2^4 sites of 2N1 = 4 components
P0 = dict(N=2, agg_block=(2, 2, 2, 1), sap_block=(2, 2, 2, 2), nu=2)
P1 = dict(N=2, agg_block=(1, 1, 1, 2), sap_block=(1, 1, 1, 2), nu=2)
DIMS1 = (2, 2, 2, 4)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def dense_sap(Ad, blk, n, nu):
    """M_SAP^(nu) = sum_{k<nu} (I - K A)^k K with K = B_black (I - A B_red) + B_red and exact
    inverses of A restricted to every block (Sec. 2.3)."""
    m = Ad.shape[0]
    B = []
    for colour in (0, 1):
        Bc = np.zeros((m, m), dtype=np.complex128)
        for b in np.nonzero(blk.colour == colour)[0]:
            idx = (blk.sites[b][:, None] * n + np.arange(n)[None, :]).ravel()
            Bc[np.ix_(idx, idx)] = np.linalg.inv(Ad[np.ix_(idx, idx)])
        B.append(Bc)
    I = np.eye(m)
    K = B[1] @ (I - Ad @ B[0]) + B[0]
    M = np.zeros_like(K)
    Ek = I
    for _ in range(nu):
        M = M + Ek @ K
        Ek = (I - K @ Ad) @ Ek
    return M


def gamma5_dense(V, n):
    return np.diag(np.tile(np.r_[np.ones(n // 2), -np.ones(n // 2)], V)).astype(np.complex128)


@pytest.fixture(scope="module")
def op():
    return DiracOperator(synth.gauge_field(DIMS, 0.4, seed=71), DIMS, 0.1, 1.0)


@pytest.fixture(scope="module")
def dense0(op):
    return op.dense()


def _hierarchy(op, inner="vcycle", inner_tol=5e-2, coarse_tol=1e-14, nu1=P1["nu"]):
    p1 = dict(P1, nu=nu1)
    ml = MultiLevel(op, [Params(coarse_tol=coarse_tol, coarse_maxiter=5000, **P0),
                         Params(coarse_tol=coarse_tol, coarse_maxiter=5000, **p1)],
                    inner=inner, inner_tol=inner_tol)
    v0 = synth.random_test_vectors(DIMS, 2, seed=72)
    v1 = synth.gaussian_coarse(int(np.prod(DIMS1)), 4, 2, seed=73)
    ml.build([v0, v1])
    return ml


@pytest.fixture(scope="module")
def three(op):
    return _hierarchy(op)


def test_fine_operator_as_stencil(op):
    """D written as nine 12 x 12 blocks per site is D; its Gamma5 is that of the chiral basis."""
    A = StencilOperator.from_dirac(op)
    x = synth.gaussian_spinors(DIMS, 1, seed=74)[0]
    assert rel(A.apply(x.reshape(op.V, 12)), op.apply(x).reshape(op.V, 12)) < 1e-14
    assert np.array_equal(A.gamma5(x.reshape(op.V, 12)), gamma5_field(x).reshape(op.V, 12))


def test_generic_level_reproduces_fine_classes(op):
    """The stencil-level aggregation, Galerkin stencil and SAP applied to the fine D give the pinned
    fine-level P, D_c and M_SAP (a second implementation of each, checked against the first)."""
    A = StencilOperator.from_dirac(op)
    v = synth.random_test_vectors(DIMS, 3, seed=75)
    fagg = Aggregation(op.lat, (2, 2, 2, 2), v)
    sagg = StencilAggregation(op.lat, (2, 2, 2, 2), v.reshape(3, op.V, 12))
    assert np.allclose(sagg.P, fagg.P, rtol=0, atol=1e-13)
    x = synth.gaussian_spinors(DIMS, 1, seed=76)[0]
    assert rel(sagg.restrict(x.reshape(op.V, 12)), fagg.restrict(x)) < 1e-14
    e = synth.gaussian_coarse(fagg.blk.nblocks, fagg.nc, 1, seed=77)[0]
    assert rel(sagg.prolong(e), fagg.prolong(e).reshape(op.V, 12)) < 1e-14
    Bs = StencilCoarse(A, sagg).B
    Bf = CoarseOperator(op, fagg).B
    assert np.max(np.abs(Bs - Bf)) < 1e-13 * np.max(np.abs(Bf))
    b = synth.gaussian_spinors(DIMS, 1, seed=78)[0]
    ref = SAP(op, (2, 2, 2, 2), mr_steps=4).apply(b, 2).reshape(op.V, 12)
    assert rel(StencilSAP(A, (2, 2, 2, 2), mr_steps=4).apply(b.reshape(op.V, 12), 2), ref) < 1e-13


def test_level_operator_is_the_dense_galerkin_product(three, dense0):
    """D_1 = P_0^H D P_0 as a dense matrix, and Gamma5^c D_1 is hermitian (Sec. 3.2)."""
    P = three.levels[0].agg.dense()
    D1 = three.levels[1].D
    D1d = D1.dense()
    assert rel(D1d, P.conj().T @ dense0 @ P) < 1e-13
    G = gamma5_dense(D1.V, D1.n)
    assert np.max(np.abs(G @ D1d - (G @ D1d).conj().T)) < 1e-13 * np.max(np.abs(D1d))


def test_level_aggregation_properties(three):
    """On level 1: P^H P = I, Gamma5_1 P = P Gamma5_2 (Gamma5 compatibility, with Gamma5^c in the
    role of Gamma5), and every level-1 test vector lies in range(P) (Sec. 3.1-3.2)."""
    lv = three.levels[1]
    P = lv.agg.dense()
    assert np.max(np.abs(P.conj().T @ P - np.eye(P.shape[1]))) < 1e-13
    G1 = gamma5_dense(lv.D.V, lv.D.n)
    G2 = gamma5_dense(lv.agg.blk.nblocks, lv.agg.nc)
    assert np.max(np.abs(G1 @ P - P @ G2)) < 1e-14
    for v in lv.vectors:
        vf = v.ravel()
        assert np.linalg.norm(vf - P @ (P.conj().T @ vf)) < 1e-12 * np.linalg.norm(vf)


def test_level_galerkin_stencil_dense_gamma5_and_mass_shift(three):
    """D_2 assembled as a stencil equals the dense P_1^H D_1 P_1; Gamma5^c D_2 is hermitian; adding
    delta I to D_1 adds exactly delta I to D_2 (P^H P = I)."""
    lv = three.levels[1]
    D1d = lv.D.dense()
    P = lv.agg.dense()
    D2d = lv.Dc.dense()
    assert rel(D2d, P.conj().T @ D1d @ P) < 1e-13
    G2 = gamma5_dense(lv.Dc.V, lv.Dc.n)
    assert np.max(np.abs(G2 @ D2d - (G2 @ D2d).conj().T)) < 1e-13 * np.max(np.abs(D2d))
    delta = 0.37
    B = lv.D.B.copy()
    B[:, 0] += delta * np.eye(lv.D.n)
    shifted = StencilCoarse(StencilOperator(lv.D.lat, B), lv.agg)
    diff = shifted.B - lv.Dc.B
    assert np.max(np.abs(diff[:, 0] - delta * np.eye(lv.Dc.n))) < 1e-14
    assert np.max(np.abs(diff[:, 1:])) < 1e-14


def test_level_sap_exact_blocks_equal_dense_sum(three):
    """Level-1 SAP with exact block solves: nu = 1 and nu = 3 against the dense sum over
    (I - K D_1)^k K (Sec. 2.3)."""
    lv = three.levels[1]
    sap = StencilSAP(lv.D, P1["sap_block"], block_solver="exact")
    D1d = lv.D.dense()
    b = synth.gaussian_coarse(lv.D.V, lv.D.n, 1, seed=79)[0]
    for nu in (1, 3):
        M = dense_sap(D1d, sap.blk, lv.D.n, nu)
        assert rel(sap.apply(b, nu), M @ b.ravel()) < 1e-12


def test_level_mr_converges_and_orthogonality(three):
    """Level-1 odd-even MR: many steps reach the exact block solve; each step leaves the new residual
    orthogonal to S rho on every block."""
    lv = three.levels[1]
    sap = StencilSAP(lv.D, P1["sap_block"], mr_steps=4)
    r = synth.gaussian_coarse(lv.D.V, lv.D.n, 1, seed=80)[0]
    for colour in (0, 1):
        exact = sap.exact_block_solve(r, colour)
        assert rel(sap.mr_block_solve(r, colour, steps=200), exact) < 1e-11
    hist = []
    sap.mr_block_solve(r, 1, history=hist)
    bos, nb = sap.blk.block_of_site, sap.blk.nblocks
    for t, rho_new in hist:
        ip = _block_sum(np.sum(np.conj(t) * rho_new, axis=1), bos, nb)
        nt = _block_sum(np.sum(np.abs(t) ** 2, axis=1), bos, nb).real
        nr = _block_sum(np.sum(np.abs(rho_new) ** 2, axis=1), bos, nb).real
        assert np.all(np.abs(ip) <= 1e-12 * np.sqrt(nt * nr) + 1e-300)


def test_three_level_vcycle_equals_nested_iteration_matrix(op, dense0):
    """inner = "vcycle", exact block solves on both smoothing levels, coarsest solve to 1e-14:
    C_0 = M_0 (I - D P_0 C_1 P_0^H) + P_0 C_1 P_0^H with
    C_1 = M_1 (I - D_1 P_1 D_2^{-1} P_1^H) + P_1 D_2^{-1} P_1^H (Sec. 4.2, applied at each level)."""
    ml = _hierarchy(op, nu1=1)  # one level-1 sweep, so that C_1 stays visibly different from D_1^{-1}
    l0, l1 = ml.levels
    l0.sap.block_solver, l0.sap._dense = "exact", dense0
    l1.sap.block_solver = "exact"
    P0d, P1d = l0.agg.dense(), l1.agg.dense()
    D1d = l1.D.dense()
    D2d = P1d.conj().T @ D1d @ P1d
    M0 = dense_sap(dense0, l0.sap.blk, 12, P0["nu"])
    M1 = dense_sap(D1d, l1.sap.blk, l1.D.n, 1)
    CGC1 = P1d @ np.linalg.solve(D2d, P1d.conj().T)
    C1 = M1 @ (np.eye(D1d.shape[0]) - D1d @ CGC1) + CGC1
    T = P0d @ C1 @ P0d.conj().T
    C0 = M0 @ (np.eye(dense0.shape[0]) - dense0 @ T) + T
    r = synth.gaussian_spinors(DIMS, 1, seed=81)[0]
    err = rel(ml.vcycle(r), C0 @ r.ravel())
    # the recursion is not the two-level V-cycle (C_1 differs from D_1^{-1}), by far more than err
    two = P0d @ np.linalg.solve(D1d, P0d.conj().T)
    C2 = M0 @ (np.eye(dense0.shape[0]) - dense0 @ two) + two
    assert err < 1e-10 and rel(C0 @ r.ravel(), C2 @ r.ravel()) > 1e3 * err


def test_tight_inner_fgmres_gives_the_two_level_vcycle(op, dense0):
    """inner = "fgmres" to 1e-13: the level-1 solve is exact to rounding, so the three-level V-cycle
    is the two-level one with an exact coarse solve, M_0 (I - D P_0 D_1^{-1} P_0^H) + P_0 D_1^{-1} P_0^H."""
    ml = _hierarchy(op, inner="fgmres", inner_tol=1e-13, coarse_tol=5e-2)
    l0 = ml.levels[0]
    l0.sap.block_solver, l0.sap._dense = "exact", dense0
    P0d = l0.agg.dense()
    D1d = ml.levels[1].D.dense()
    M0 = dense_sap(dense0, l0.sap.blk, 12, P0["nu"])
    T = P0d @ np.linalg.solve(D1d, P0d.conj().T)
    C = M0 @ (np.eye(dense0.shape[0]) - dense0 @ T) + T
    r = synth.gaussian_spinors(DIMS, 1, seed=82)[0]
    assert rel(ml.vcycle(r), C @ r.ravel()) < 1e-9
    assert ml.levels[0].cs.last_iters > 1


def test_level_setup_update_against_dense_iteration_matrix(three):
    """The Algorithm 2 update on level 1, v + C_1 (v - D_1 v), with exact block and coarse solves,
    against the dense C_1; and Algorithm 1's C_1 v."""
    lv = three.levels[1]
    D1d = lv.D.dense()
    saved = lv.sap.block_solver
    lv.sap.block_solver = "exact"
    try:
        P = lv.agg.dense()
        CGC = P @ np.linalg.solve(P.conj().T @ D1d @ P, P.conj().T)
        M1 = dense_sap(D1d, lv.sap.blk, lv.D.n, P1["nu"])
        C = M1 @ (np.eye(D1d.shape[0]) - D1d @ CGC) + CGC
        v = synth.gaussian_coarse(lv.D.V, lv.D.n, 1, seed=83)[0]
        vf = v.ravel()
        u2 = lv.setup_update(v)
        lv.p.setup_update = "idsetup"
        u1 = lv.setup_update(v)
    finally:
        lv.p.setup_update = "ddalpha"
        lv.sap.block_solver = saved
    assert rel(u2, C @ vf + vf - C @ (D1d @ vf)) < 1e-9
    assert rel(u1, C @ vf) < 1e-9


def test_multilevel_setup_runs_two_level_setups_finest_first(op):
    """ML5: the level-0 stage of the multilevel setup is the two-level setup itself (same vectors);
    level 1 then starts from the supplied random vectors on D_1 and ends orthonormalisable."""
    p0 = Params(n_inv=1, **P0)
    p1 = Params(n_inv=1, **P1)
    v0 = synth.random_test_vectors(DIMS, 2, seed=84)
    drawn = []

    def initial(l, V, n, N):
        drawn.append((l, V, n, N))
        return synth.gaussian_coarse(V, n, N, seed=85 + l)

    ml = MultiLevel(op, [p0, p1])
    vecs = ml.setup(v0, initial)
    ref = TwoLevel(op, Params(n_inv=1, **P0)).setup(v0)
    assert rel(vecs[0], ref) < 1e-13
    assert drawn == [(1, int(np.prod(DIMS1)), 4, 2)]
    assert vecs[1].shape == (2, int(np.prod(DIMS1)), 4)
    assert isinstance(ml.levels[1], StencilTwoLevel)
    assert ml.levels[1].D.V == int(np.prod(DIMS1))


def test_three_level_solve_matches_dense_lu(op, dense0):
    """Whole method with three levels (MR smoothers, coarse solves to 5e-2, the default inner FGMRES):
    true residual <= 1e-10 and agreement with a dense LU."""
    ml = _hierarchy(op, inner="fgmres", inner_tol=5e-2, coarse_tol=5e-2)
    b = synth.gaussian_spinors(DIMS, 1, seed=86)[0]
    z, info = ml.solve(b)
    assert np.linalg.norm(b - op.apply(z)) <= 1e-10 * np.linalg.norm(b)
    ref = np.linalg.solve(dense0, b.ravel())
    assert rel(z, ref) < 1e-8
    # every level-0 V-cycle runs at least one level-1 V-cycle inside its FGMRES; the coarsest GMRES runs
    assert info["vcycles_per_level"][1] >= info["vcycles_per_level"][0] > 0 and info["coarsest_iters"] > 0


def test_four_level_solve():
    """Four levels on 4^4 (aggregates 2x2x2x1, then 1x1x1x2, then single sites): the solve still
    reaches a true residual of 1e-10 and the coarsest odd-even GMRES is reached through the recursion."""
    D = DiracOperator(synth.gauge_field(DIMS, 0.4, seed=87), DIMS, 0.05, 1.0)
    p2 = Params(N=1, agg_block=(1, 1, 1, 1), sap_block=(1, 1, 1, 1), nu=2)
    ml = MultiLevel(D, [Params(**P0), Params(**P1), p2])
    ml.build([synth.random_test_vectors(DIMS, 2, seed=88), synth.gaussian_coarse(int(np.prod(DIMS1)), 4, 2, seed=89),
              synth.gaussian_coarse(16, 4, 1, seed=90)])
    assert ml.n_levels == 4 and ml.levels[2].Dc.n == 2
    b = synth.gaussian_spinors(DIMS, 1, seed=91)[0]
    z, info = ml.solve(b)
    assert np.linalg.norm(b - D.apply(z)) <= 1e-10 * np.linalg.norm(b)
    assert info["coarsest_iters"] > 0
