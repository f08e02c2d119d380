"""Pins of the oracle's aggregation P (Sec. 3.1-3.2) and coarse operator D_c = P^H D P."""
import numpy as np
import pytest

from oracle.aggregation import Aggregation
from oracle.coarse import CoarseOperator, CoarseSolver
from oracle.dirac import DiracOperator, gamma5_field
from paper_1303_1377_gb300 import synth

CASES = [
    # (lattice, aggregate block, N): coarse 2^4 (forward = backward neighbour), and coarse 2x2x2x4
    ((4, 4, 4, 4), (2, 2, 2, 2), 3),
    ((2, 2, 2, 8), (1, 1, 1, 2), 4),
]


def _setup(dims, bdims, N, m0=-0.1, seed=31):
    U = synth.gauge_field(dims, 0.5, seed=seed)
    D = DiracOperator(U, dims, m0, 1.0)
    v = synth.random_test_vectors(dims, N, seed=seed + 1)
    agg = Aggregation(D.lat, bdims, v)
    return D, agg, v


@pytest.mark.parametrize("dims,bdims,N", CASES)
def test_P_orthonormal_gamma5_compatible_and_spans_vectors(dims, bdims, N):
    D, agg, v = _setup(dims, bdims, N)
    P = agg.dense()
    assert np.allclose(P.conj().T @ P, np.eye(P.shape[1]), atol=1e-13)  # P^H P = I (Sec. 3.1)
    # Gamma5 P = P Gamma5^c (Eq. commute_with_g5)
    g5P = np.stack([gamma5_field(P[:, c].reshape(-1, 4, 3)).ravel() for c in range(P.shape[1])], axis=1)
    Pg5c = np.stack([agg.prolong(agg.gamma5_coarse(np.eye(P.shape[1])[c].reshape(-1, agg.nc))).ravel() for c in range(P.shape[1])], axis=1)
    assert np.allclose(g5P, Pg5c, atol=1e-14)
    # every test vector lies in range(P) (Sec. 3.1)
    for j in range(N):
        vj = v[j].ravel()
        assert np.linalg.norm(vj - P @ (P.conj().T @ vj)) < 1e-12 * np.linalg.norm(vj)


def test_local_orthonormalisation_is_ordered_qr():
    """The basis on each aggregate is the Q factor of the ordered QR with positive real diagonal:
    P_a^H v_j|_a vanishes for basis index > j and is positive real on the diagonal."""
    D, agg, v = _setup((4, 4, 4, 4), (2, 2, 2, 2), 3)
    R = np.stack([agg.restrict(v[j]) for j in range(3)], axis=-1)  # [nb, 2N, N]
    for h in range(2):
        Rh = R[:, h * 3:(h + 1) * 3, :]
        for i in range(3):
            for j in range(3):
                if i > j:
                    assert np.all(np.abs(Rh[:, i, j]) < 1e-12)
                if i == j:
                    assert np.all(Rh[:, i, j].real > 0) and np.all(np.abs(Rh[:, i, j].imag) < 1e-12)


@pytest.mark.parametrize("dims,bdims,N", CASES)
def test_assembled_stencil_equals_dense_PHDP(dims, bdims, N):
    D, agg, _ = _setup(dims, bdims, N)
    Dc = CoarseOperator(D, agg)
    P = agg.dense()
    ref = P.conj().T @ D.dense() @ P
    assert np.allclose(Dc.dense(), ref, atol=1e-12)


@pytest.mark.parametrize("dims,bdims,N", CASES)
def test_coarse_gamma5_symmetry_and_mass_shift(dims, bdims, N):
    D, agg, _ = _setup(dims, bdims, N)
    Dc = CoarseOperator(D, agg).dense()
    nc = agg.nc
    g5c = np.tile(np.r_[np.ones(N), -np.ones(N)], Dc.shape[0] // nc)
    PG = g5c[:, None] * Dc  # Gamma5^c D_c = D_c^PG is hermitian (Lemma 3.x (i), (iii))
    assert np.allclose(PG, PG.conj().T, atol=1e-12)
    D2 = DiracOperator(D.U, dims, D.m0 + 0.3, D.c_sw)
    Dc2 = CoarseOperator(D2, agg).dense()
    assert np.allclose(Dc2 - Dc, 0.3 * np.eye(Dc.shape[0]), atol=1e-12)  # P^H P = I


def test_coarse_field_of_values_inside_fine():
    """F(D_c) subset of F(D) (Lemma 3.x (iv)): Rayleigh quotients of D_c are those of D at P x."""
    D, agg, _ = _setup((4, 4, 4, 4), (2, 2, 2, 2), 3)
    Dc = CoarseOperator(D, agg)
    x = synth.gaussian_coarse(Dc.B.shape[0], agg.nc, 1, seed=5)[0]
    x = x / np.linalg.norm(x)
    Px = agg.prolong(x)
    assert abs(np.vdot(x, Dc.apply(x)) - np.vdot(Px.ravel(), D.apply(Px).ravel())) < 1e-12
    assert abs(np.linalg.norm(Px) - 1.0) < 1e-13


@pytest.mark.parametrize("dims,bdims,N", CASES)
def test_odd_even_coarse_solve_matches_dense(dims, bdims, N):
    D, agg, _ = _setup(dims, bdims, N, m0=0.3)
    Dc = CoarseOperator(D, agg)
    cs = CoarseSolver(Dc, restart=30, tol=1e-13, maxiter=5000)
    b = synth.gaussian_coarse(Dc.B.shape[0], agg.nc, 1, seed=7)[0]
    x = cs.solve(b)
    ref = np.linalg.solve(Dc.dense(), b.ravel())
    assert np.linalg.norm(x.ravel() - ref) < 1e-10 * np.linalg.norm(ref)
