"""Pins of the oracle's SAP smoother (Sec. 2.3) and its local MR solver (Sec. 6)."""
import numpy as np
import pytest

from oracle.dirac import DiracOperator
from oracle.sap import SAP, _block_sum
from paper_1303_1377_gb300 import synth

DIMS = (4, 4, 4, 4)


@pytest.fixture(scope="module")
def op():
    U = synth.gauge_field(DIMS, 0.4, seed=21)
    return DiracOperator(U, DIMS, 0.2, 1.0)


@pytest.fixture(scope="module")
def dense(op):
    return op.dense()


def _block_inverse_dense(sap, Dd, colour):
    """B_colour as a dense matrix: block-diagonal inverse of D restricted to the blocks of one colour."""
    n = Dd.shape[0]
    B = np.zeros((n, n), dtype=np.complex128)
    for b in np.nonzero(sap.blk.colour == colour)[0]:
        idx = (sap.blk.sites[b][:, None] * 12 + np.arange(12)[None, :]).ravel()
        B[np.ix_(idx, idx)] = np.linalg.inv(Dd[np.ix_(idx, idx)])
    return B


def test_mr_converges_to_dense_block_solve(op):
    """Odd-even reduction + MR + back-substitution solves D_i e_i = r_i once MR has converged."""
    sap = SAP(op, (2, 2, 2, 2), mr_steps=4)
    r = synth.gaussian_spinors(DIMS, 1, seed=22)[0]
    for colour in (0, 1):
        exact = sap.exact_block_solve(r, colour)
        mr = sap.mr_block_solve(r, colour, steps=150)
        assert np.linalg.norm(mr - exact) < 1e-11 * np.linalg.norm(exact)


def test_mr_residual_orthogonality(op):
    """Each MR step makes the new residual orthogonal to S rho on every block."""
    sap = SAP(op, (2, 2, 2, 2), mr_steps=4)
    r = synth.gaussian_spinors(DIMS, 1, seed=23)[0]
    hist = []
    sap.mr_block_solve(r, 0, history=hist)
    assert len(hist) == 4
    for t, rho_new in hist:
        ip = _block_sum(np.sum(np.conj(t) * rho_new, axis=(1, 2)), sap.blk.block_of_site, sap.blk.nblocks)
        nt = _block_sum(np.sum(np.abs(t) ** 2, axis=(1, 2)), sap.blk.block_of_site, sap.blk.nblocks).real
        nr = _block_sum(np.sum(np.abs(rho_new) ** 2, axis=(1, 2)), sap.blk.block_of_site, sap.blk.nblocks).real
        assert np.all(np.abs(ip) <= 1e-12 * np.sqrt(nt * nr) + 1e-300)


def test_mr_residual_decreases(op):
    """MR minimises ||rho - alpha S rho||, so block residual norms never grow."""
    sap = SAP(op, (2, 2, 2, 2), mr_steps=6)
    r = synth.gaussian_spinors(DIMS, 1, seed=24)[0]
    hist = []
    sap.mr_block_solve(r, 1, history=hist)
    norms = [np.linalg.norm(h[1]) for h in hist]
    assert all(b <= a * (1 + 1e-14) for a, b in zip(norms, norms[1:]))


def test_exact_sap_equals_dense_K(op, dense):
    """With exact block solves: M_SAP^(1) b = K b, K = B_black (I - D B_red) + B_red (Eq. SAP_1step);
    the error propagator is (I - B_black D)(I - B_red D); M_SAP^(nu) = sum_k (I-KD)^k K."""
    sap = SAP(op, (2, 2, 2, 2), block_solver="exact")
    sap._dense = dense
    n = dense.shape[0]
    Br = _block_inverse_dense(sap, dense, 0)
    Bb = _block_inverse_dense(sap, dense, 1)
    I = np.eye(n)
    K = Bb @ (I - dense @ Br) + Br
    assert np.allclose(I - K @ dense, (I - Bb @ dense) @ (I - Br @ dense), atol=1e-10)
    b = synth.gaussian_spinors(DIMS, 1, seed=25)[0]
    bf = b.ravel()
    assert np.allclose(sap.apply(b, 1).ravel(), K @ bf, atol=1e-11)
    E = I - K @ dense
    M3 = (I + E + E @ E) @ K
    assert np.allclose(sap.apply(b, 3).ravel(), M3 @ bf, atol=1e-10)


def test_sap_reduces_large_eigen_components():
    """Smoothing property (Sec. 2.3, Fig. errSAP): near the critical mass ||E v||/||v|| stays close
    to one for the eigenvectors of smallest |lambda| and is much smaller for the largest (qualitative)."""
    op = DiracOperator(synth.gauge_field(DIMS, 0.4, seed=21), DIMS, -0.6, 1.0)
    dense = op.dense()
    sap = SAP(op, (2, 2, 2, 2), block_solver="exact")
    n = dense.shape[0]
    Br = _block_inverse_dense(sap, dense, 0)
    Bb = _block_inverse_dense(sap, dense, 1)
    E = (np.eye(n) - Bb @ dense) @ (np.eye(n) - Br @ dense)
    lam, vecs = np.linalg.eig(dense)
    order = np.argsort(np.abs(lam))
    ratio = np.linalg.norm(E @ vecs[:, order], axis=0) / np.linalg.norm(vecs[:, order], axis=0)
    assert np.mean(ratio[:4]) > 0.9
    assert np.mean(ratio[:4]) > 2 * np.mean(ratio[-n // 20:])
