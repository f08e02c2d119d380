"""Pins of the oracle's V-cycle (Sec. 4.2), setup (Algorithms 1-2) and FGMRES solve (Sec. 5)."""
import json
import os

import numpy as np
import pytest

from oracle.dirac import DiracOperator
from oracle.mg import Params, TwoLevel
from paper_1303_1377_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_default_parameters_are_table1():
    t = json.load(open(os.path.join(GOLDEN, "table1_defaults.json")))
    p = Params()
    for k in ("n_inv", "N", "coarse_tol", "n_kv", "tol", "nu", "mr_steps", "coarse_restart"):
        assert getattr(p, k) == t[k], k
    assert tuple(p.agg_block) == tuple(t["agg_block"]) and tuple(p.sap_block) == tuple(t["sap_block"])


@pytest.fixture(scope="module")
def small():
    dims = (4, 4, 4, 4)
    D = DiracOperator(synth.gauge_field(dims, 0.4, seed=41), dims, 0.15, 1.0)
    p = Params(N=2, agg_block=(2, 2, 2, 2), sap_block=(2, 2, 2, 2), nu=2, coarse_tol=1e-14, coarse_maxiter=5000)
    mg = TwoLevel(D, p, vectors=synth.random_test_vectors(dims, 2, seed=42))
    mg.sap.block_solver = "exact"
    Dd = D.dense()
    mg.sap._dense = Dd
    return D, mg, Dd


def _dense_operators(mg, Dd):
    """Dense P D_c^{-1} P^H and M_SAP^(nu) built from exact block inverses (Sec. 2.3)."""
    n = Dd.shape[0]
    P = mg.agg.dense()
    Dc = P.conj().T @ Dd @ P
    CGC = P @ np.linalg.solve(Dc, P.conj().T)
    B = []
    for colour in (0, 1):
        Bc = np.zeros((n, n), dtype=np.complex128)
        for blk in np.nonzero(mg.sap.blk.colour == colour)[0]:
            idx = (mg.sap.blk.sites[blk][:, None] * 12 + np.arange(12)[None, :]).ravel()
            Bc[np.ix_(idx, idx)] = np.linalg.inv(Dd[np.ix_(idx, idx)])
        B.append(Bc)
    I = np.eye(n)
    K = B[1] @ (I - Dd @ B[0]) + B[0]
    E = I - K @ Dd
    Msap = np.zeros_like(K)
    Ek = I
    for _ in range(mg.p.nu):
        Msap = Msap + Ek @ K
        Ek = E @ Ek
    return P, CGC, Msap


def test_vcycle_equals_dense_iteration_matrix(small):
    """C^(nu) = M_SAP^(nu) (I - D P D_c^{-1} P^H) + P D_c^{-1} P^H (Eq. iterationmatrix),
    with exact coarse and block solves; and pi_R = I - P D_c^{-1} P^H D is a projection with pi_R P = 0."""
    D, mg, Dd = small
    n = Dd.shape[0]
    P, CGC, Msap = _dense_operators(mg, Dd)
    C = Msap @ (np.eye(n) - Dd @ CGC) + CGC
    r = synth.gaussian_spinors(D.lat.dims, 1, seed=43)[0]
    assert np.linalg.norm(mg.vcycle(r).ravel() - C @ r.ravel()) < 1e-9 * np.linalg.norm(C @ r.ravel())
    piR = np.eye(n) - CGC @ Dd
    assert np.allclose(piR @ piR, piR, atol=1e-9)
    assert np.allclose(piR @ P, 0, atol=1e-9)
    # setup update of Algorithm 2: v + C (v - D v) = C v + (I - C D) v
    v = synth.gaussian_spinors(D.lat.dims, 1, seed=44)[0]
    upd = v + mg.vcycle(v - D.apply(v))
    assert np.linalg.norm(upd.ravel() - (C @ v.ravel() + (np.eye(n) - C @ Dd) @ v.ravel())) < 1e-9 * np.linalg.norm(upd)


def test_setup_updates_against_dense_iteration_matrix(small):
    """The two setup updates against the dense C^(nu) (exact coarse and block solves):
    Algorithm 1 (inexact deflation) v <- C v; Algorithm 2 v <- C v + (I - C D) v."""
    D, mg, Dd = small
    n = Dd.shape[0]
    P, CGC, Msap = _dense_operators(mg, Dd)
    C = Msap @ (np.eye(n) - Dd @ CGC) + CGC
    v = synth.gaussian_spinors(D.lat.dims, 1, seed=45)[0]
    Cv = C @ v.ravel()
    try:
        mg.p.setup_update = "idsetup"
        u1 = mg.setup_update(v).ravel()
        mg.p.setup_update = "ddalpha"
        u2 = mg.setup_update(v).ravel()
    finally:
        mg.p.setup_update = "ddalpha"
    assert np.linalg.norm(u1 - Cv) < 1e-9 * np.linalg.norm(Cv)
    assert np.linalg.norm(u2 - (Cv + v.ravel() - C @ (Dd @ v.ravel()))) < 1e-9 * np.linalg.norm(u2)
    # the two differ by the V-cycle error propagator applied to v, which is not zero here
    assert np.linalg.norm(u2 - u1) > 1e-3 * np.linalg.norm(u2)


def test_full_solve_2x2x2x2_dense_lu():
    """Whole method on a 2^4 lattice (SAP blocks and aggregates of one site): the FGMRES solution
    agrees with a dense LU and its true residual is below 1e-10."""
    dims = (2, 2, 2, 2)
    D = DiracOperator(synth.gauge_field(dims, 0.5, seed=51), dims, 0.05, 1.0)
    p = Params(N=3, agg_block=(1, 1, 1, 1), sap_block=(1, 1, 1, 1), n_inv=2, nu=2)
    mg = TwoLevel(D, p)
    mg.setup(synth.random_test_vectors(dims, 3, seed=52))
    b = synth.gaussian_spinors(dims, 1, seed=53)[0]
    z, info = mg.solve(b)
    Dd = D.dense()
    ref = np.linalg.solve(Dd, b.ravel())
    assert info["resid"] <= 1e-10
    assert np.linalg.norm(b.ravel() - Dd @ z.ravel()) <= 1e-10 * np.linalg.norm(b)
    kappa = np.linalg.cond(Dd)
    assert np.linalg.norm(z.ravel() - ref) <= kappa * 1e-10 * np.linalg.norm(ref)


def test_full_solve_4x4x4x4_default_blocks_of_two():
    dims = (4, 4, 4, 4)
    D = DiracOperator(synth.gauge_field(dims, 0.4, seed=61), dims, 0.02, 1.0)
    p = Params(N=4, agg_block=(2, 2, 2, 2), sap_block=(2, 2, 2, 2), n_inv=2, nu=2)
    mg = TwoLevel(D, p)
    mg.setup(synth.random_test_vectors(dims, 4, seed=62))
    b = synth.gaussian_spinors(dims, 1, seed=63)[0]
    z, info = mg.solve(b)
    assert np.linalg.norm(b - D.apply(z)) <= 1e-10 * np.linalg.norm(b)
    ref = np.linalg.solve(D.dense(), b.ravel())
    assert np.linalg.norm(z.ravel() - ref) < 1e-7 * np.linalg.norm(ref)
