"""Pins of the oracle's GMRES / FGMRES against the textbook least-squares characterisation."""
import numpy as np

from oracle.krylov import fgmres, gmres


def _matrix(n=40, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return A / np.sqrt(n) + 2.5 * np.eye(n)


def test_gmres_k_steps_is_krylov_least_squares():
    A = _matrix()
    b = np.random.default_rng(1).standard_normal(40) + 0j
    for k in (1, 3, 7, 12):
        x, info = gmres(lambda v: A @ v, b, restart=30, tol=0.0, maxiter=k)
        assert info["iters"] == k
        K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        y = np.linalg.lstsq(A @ Q, b, rcond=None)[0]
        assert np.linalg.norm(x - Q @ y) < 1e-10 * np.linalg.norm(x)


def test_restarted_gmres_converges_to_dense_solution():
    A = _matrix(60, seed=2)
    b = np.random.default_rng(3).standard_normal(60) + 1j
    x, info = gmres(lambda v: A @ v, b, restart=5, tol=1e-12, maxiter=2000)
    assert info["restarts"] > 0
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) < 1e-10 * np.linalg.norm(ref)


def test_fgmres_exact_preconditioner_one_step():
    A = _matrix(30, seed=4)
    Ainv = np.linalg.inv(A)
    b = np.random.default_rng(5).standard_normal(30) + 0j
    x, info = fgmres(lambda v: A @ v, lambda v: Ainv @ v, b, n_kv=25, tol=1e-12)
    assert info["iters"] == 1
    assert np.linalg.norm(A @ x - b) < 1e-12 * np.linalg.norm(b)


def test_fgmres_identity_preconditioner_equals_gmres():
    A = _matrix(50, seed=6)
    b = np.random.default_rng(7).standard_normal(50) + 0j
    x1, i1 = fgmres(lambda v: A @ v, lambda v: v, b, n_kv=8, tol=1e-11)
    x2, i2 = gmres(lambda v: A @ v, b, restart=8, tol=1e-11, maxiter=1000)
    assert np.linalg.norm(A @ x1 - b) <= 1e-11 * np.linalg.norm(b)
    assert np.linalg.norm(x1 - x2) < 1e-9 * np.linalg.norm(x2)
