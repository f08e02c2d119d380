"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the oracle.

This module holds no arithmetic of the solver itself: it only draws random numbers
and shapes them into the objects the method consumes (gauge links, right-hand
sides, test vectors, gauge transformations).  Every generator uses numpy's
counter-based Philox bit generator keyed by the seed, so a given (shape, seed)
always yields the same array on any machine.

Layouts (all complex128, lexicographic site order with x0 = time slowest and x3
fastest, the ordering of Sec. 2.2):
  gauge field   U[site, mu, a, b]        (U_mu(x) in SU(3), Sec. 2.2)
  spinor        psi[site, spin, colour]  (12 components per site, colour fastest, Sec. 2.1)
"""
from __future__ import annotations

import numpy as np


def volume(dims) -> int:
    d = tuple(int(v) for v in dims)
    if len(d) != 4:
        raise ValueError("lattice dims must have 4 entries (L0, L1, L2, L3)")
    return int(np.prod(d))


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream)]))


def _traceless_hermitian(g: np.random.Generator, n: int) -> np.ndarray:
    a = g.standard_normal((n, 3, 3)) + 1j * g.standard_normal((n, 3, 3))
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)
    return h


def _expi(h: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*H) for hermitian H via its eigendecomposition."""
    lam, q = np.linalg.eigh(h)
    ph = np.exp(1j * eps * lam)
    return np.einsum("nab,nb,ncb->nac", q, ph, np.conj(q))


def gauge_field(dims, eps: float, seed: int, chunk: int = 1 << 18) -> np.ndarray:
    """Links U_mu(x) = exp(i*eps*H_mu(x)), H traceless hermitian with Gaussian entries.

    H = (A + A^H)/2 - tr(.)/3, A i.i.d. complex N(0,1) per real/imaginary part.
    Returns complex128 [V, 4, 3, 3].
    """
    V = volume(dims)
    g = _rng(seed, 1)
    out = np.empty((V * 4, 3, 3), dtype=np.complex128)
    n = V * 4
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        out[s:e] = _expi(_traceless_hermitian(g, e - s), eps)
    return out.reshape(V, 4, 3, 3)


def unit_gauge(dims) -> np.ndarray:
    V = volume(dims)
    u = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u


def random_su3(n: int, seed: int) -> np.ndarray:
    """n Haar-ish random SU(3) matrices (QR of a complex Gaussian, phase-fixed)."""
    g = _rng(seed, 2)
    a = g.standard_normal((n, 3, 3)) + 1j * g.standard_normal((n, 3, 3))
    q, r = np.linalg.qr(a)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q = q / (det ** (1.0 / 3.0))[:, None, None]
    return q


def gaussian_spinors(dims, nrhs: int, seed: int) -> np.ndarray:
    """i.i.d. complex Gaussian spinors, N(0,1) per real/imaginary part: [nrhs, V, 4, 3]."""
    V = volume(dims)
    g = _rng(seed, 3)
    return g.standard_normal((nrhs, V, 4, 3)) + 1j * g.standard_normal((nrhs, V, 4, 3))


def point_sources(dims, site: int = 0) -> np.ndarray:
    """The 12 point sources e_{x, sigma, c} at one site: [12, V, 4, 3]."""
    V = volume(dims)
    b = np.zeros((12, V, 4, 3), dtype=np.complex128)
    for k in range(12):
        b[k, site, k // 3, k % 3] = 1.0
    return b


def random_test_vectors(dims, n: int, seed: int) -> np.ndarray:
    """Initial random test vectors for the adaptive setup: [n, V, 4, 3] complex Gaussian."""
    V = volume(dims)
    g = _rng(seed, 4)
    return g.standard_normal((n, V, 4, 3)) + 1j * g.standard_normal((n, V, 4, 3))


def gaussian_coarse(nc_sites: int, ncomp: int, nrhs: int, seed: int) -> np.ndarray:
    """Random coarse vectors [nrhs, nc_sites, ncomp] (complex Gaussian)."""
    g = _rng(seed, 5)
    return g.standard_normal((nrhs, nc_sites, ncomp)) + 1j * g.standard_normal((nrhs, nc_sites, ncomp))
