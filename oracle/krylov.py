"""Restarted GMRES and flexible GMRES (oracle; test infrastructure only).

Textbook forms (Saad, Iterative Methods for Sparse Linear Systems, Alg. 6.9 and
9.6), as used by the paper: restarted GMRES(30) for the odd-even reduced coarse
system (Sec. 6) and right-preconditioned FGMRES(n_kv) around one V-cycle for the
fine system (Sec. 5, Table 1).  Arnoldi uses modified Gram-Schmidt, the
Hessenberg least-squares problem is solved with complex Givens rotations, and
the iteration stops when the Arnoldi residual estimate |g_{k+1}| drops to
tol * ||b||.  At every restart the residual is recomputed as b - A x.  FGMRES
accepts convergence only once the recomputed (true) residual meets the tolerance.

Inner product <u, v> = u^H v throughout.

Pins (tests/test_oracle_krylov.py): after k steps without restart GMRES returns
the dense least-squares minimiser over the Krylov space; FGMRES with the exact
inverse as preconditioner converges in one step; solutions agree with a dense LU.
"""
from __future__ import annotations

import numpy as np


def _norm(v: np.ndarray) -> float:
    return float(np.sqrt(np.sum(np.abs(v) ** 2)))


def _dot(u: np.ndarray, v: np.ndarray) -> complex:
    return complex(np.vdot(u.ravel(), v.ravel()))


def _givens(a: complex, b: float):
    """Rotation (c real, s complex) with [c s; -conj(s) c] [a; b] = [r; 0]."""
    denom = np.hypot(abs(a), abs(b))
    if denom == 0.0:
        return 1.0, 0.0 + 0.0j
    if abs(a) == 0.0:
        return 0.0, 1.0 + 0.0j
    c = abs(a) / denom
    s = (a / abs(a)) * np.conj(b) / denom
    return c, s


def _arnoldi_cycle(A, M, r, beta, m, tol_abs, budget):
    """One restart cycle; returns (update, steps, estimate)."""
    V = [r / beta]
    Z = []
    H = np.zeros((m + 1, m), dtype=np.complex128)
    cs = np.zeros(m)
    sn = np.zeros(m, dtype=np.complex128)
    g = np.zeros(m + 1, dtype=np.complex128)
    g[0] = beta
    k_last = -1
    est = beta
    for k in range(min(m, budget)):
        z = V[k] if M is None else M(V[k])
        Z.append(z)
        w = A(z)
        for i in range(k + 1):
            H[i, k] = _dot(V[i], w)
            w = w - H[i, k] * V[i]
        hk = _norm(w)
        H[k + 1, k] = hk
        V.append(w / hk if hk > 0 else np.zeros_like(w))
        for i in range(k):
            t0 = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
            t1 = -np.conj(sn[i]) * H[i, k] + cs[i] * H[i + 1, k]
            H[i, k], H[i + 1, k] = t0, t1
        c, s = _givens(H[k, k], hk)
        cs[k], sn[k] = c, s
        H[k, k] = c * H[k, k] + s * hk
        H[k + 1, k] = 0.0
        g[k + 1] = -np.conj(s) * g[k]
        g[k] = c * g[k]
        est = abs(g[k + 1])
        k_last = k
        if est <= tol_abs:
            break
    n = k_last + 1
    y = np.zeros(n, dtype=np.complex128)
    for i in range(n - 1, -1, -1):
        y[i] = (g[i] - np.dot(H[i, i + 1:n], y[i + 1:n])) / H[i, i]
    upd = np.zeros_like(r)
    for i in range(n):
        upd = upd + y[i] * Z[i]
    return upd, n, est


def gmres(A, b, x0=None, restart=30, tol=1e-10, maxiter=1000):
    """Restarted GMRES(restart) for A x = b; stops when the estimate <= tol ||b||."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, copy=True)
    bnorm = _norm(b)
    info = {"iters": 0, "restarts": 0, "resid": 0.0}
    if bnorm == 0.0:
        return x, info
    r = b - A(x) if x0 is not None else np.array(b, copy=True)
    beta = _norm(r)
    while beta > tol * bnorm and info["iters"] < maxiter:
        upd, n, est = _arnoldi_cycle(A, None, r, beta, restart, tol * bnorm, maxiter - info["iters"])
        x = x + upd
        info["iters"] += n
        if est <= tol * bnorm or info["iters"] >= maxiter:
            beta = est
            break
        info["restarts"] += 1
        r = b - A(x)
        beta = _norm(r)
    info["resid"] = beta / bnorm
    return x, info


def fgmres(A, M, b, x0=None, n_kv=25, tol=1e-10, maxiter=10000):
    """Right-preconditioned flexible GMRES(n_kv); converged when ||b - A x|| <= tol ||b||."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, copy=True)
    bnorm = _norm(b)
    info = {"iters": 0, "restarts": 0, "resid": 0.0, "history": []}
    if bnorm == 0.0:
        return x, info
    r = b - A(x)
    beta = _norm(r)
    while beta > tol * bnorm and info["iters"] < maxiter:
        upd, n, est = _arnoldi_cycle(A, M, r, beta, n_kv, tol * bnorm, maxiter - info["iters"])
        x = x + upd
        info["iters"] += n
        r = b - A(x)
        beta = _norm(r)
        info["history"].append(beta / bnorm)
        info["restarts"] += 1
    info["resid"] = beta / bnorm
    return x, info
