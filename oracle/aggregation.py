"""Aggregation-based interpolation P and restriction P^H (Sec. 3.1-3.2).

Standard aggregation (Sec. 3.2, Definition): for every lattice-block L_j the two
aggregates A_j0 = L_j x {spins 0,1} x C and A_j1 = L_j x {spins 2,3} x C.
P e_(j,h,k) is the k-th vector of an orthonormal basis of
span(I_A v_1, ..., I_A v_N) on aggregate A = A_jh (Sec. 3.1, local
orthonormalisation, giving P^H P = I).  The basis is produced by modified
Gram-Schmidt in the order v_1, ..., v_N, i.e. the Q factor of the thin QR
factorisation with a positive real diagonal of R.

Coarse vectors are [nblocks, 2N] with component index h*N + k (h = 0 for spins
0,1 and h = 1 for spins 2,3), blocks numbered lexicographically by block coords.

Pins (tests/test_oracle_coarse.py): P^H P = I; Gamma5 P = P Gamma5^c (Eq.
commute_with_g5); every test vector lies in range(P); the QR factorisation
reproduces the restricted test vectors.
"""
from __future__ import annotations

import numpy as np

from .lattice import Blocking, Lattice


def modified_gram_schmidt(M: np.ndarray, rank_tol: float = 1e-12) -> np.ndarray:
    """Orthonormalise the columns of M[..., n, N] in order (modified Gram-Schmidt)."""
    Q = np.array(M, dtype=np.complex128, copy=True)
    N = Q.shape[-1]
    for j in range(N):
        for i in range(j):
            h = np.sum(np.conj(Q[..., :, i]) * Q[..., :, j], axis=-1)
            Q[..., :, j] -= h[..., None] * Q[..., :, i]
        nrm = np.sqrt(np.sum(np.abs(Q[..., :, j]) ** 2, axis=-1))
        ref = np.sqrt(np.sum(np.abs(M[..., :, j]) ** 2, axis=-1))
        if np.any(nrm <= rank_tol * np.maximum(ref, 1e-300)):
            raise np.linalg.LinAlgError("test vectors are linearly dependent on an aggregate")
        Q[..., :, j] /= nrm[..., None]
    return Q


class Aggregation:
    def __init__(self, lat: Lattice, block_dims, vectors: np.ndarray):
        """vectors: [N, V, 4, 3] test vectors v_1..v_N."""
        self.lat = lat
        self.blk = Blocking(lat, block_dims)
        v = np.asarray(vectors, dtype=np.complex128)
        self.N = v.shape[0]
        nb, bv = self.blk.nblocks, self.blk.bvol
        vb = np.moveaxis(v, 0, -1)[self.blk.sites]  # [nb, bvol, 4, 3, N]
        M = np.stack([vb[:, :, 0:2].reshape(nb, bv * 6, self.N), vb[:, :, 2:4].reshape(nb, bv * 6, self.N)], axis=1)
        self.P = modified_gram_schmidt(M)  # [nb, 2, bvol*6, N]

    @property
    def nc(self) -> int:
        return 2 * self.N

    def _split(self, r: np.ndarray) -> np.ndarray:
        nb, bv = self.blk.nblocks, self.blk.bvol
        rb = r[self.blk.sites]  # [nb, bvol, 4, 3]
        return np.stack([rb[:, :, 0:2].reshape(nb, bv * 6), rb[:, :, 2:4].reshape(nb, bv * 6)], axis=1)

    def restrict(self, r: np.ndarray) -> np.ndarray:
        """P^H r: [V,4,3] -> [nblocks, 2N]."""
        rh = self._split(r)
        e = np.einsum("bhkj,bhk->bhj", np.conj(self.P), rh)
        return e.reshape(self.blk.nblocks, self.nc)

    def prolong(self, e: np.ndarray) -> np.ndarray:
        """P e: [nblocks, 2N] -> [V,4,3]."""
        nb, bv = self.blk.nblocks, self.blk.bvol
        eh = e.reshape(nb, 2, self.N)
        rh = np.einsum("bhkj,bhj->bhk", self.P, eh).reshape(nb, 2, bv, 2, 3)
        out = np.zeros((self.lat.V, 4, 3), dtype=np.complex128)
        out[self.blk.sites] = np.concatenate([rh[:, 0], rh[:, 1]], axis=2)
        return out

    def dense(self) -> np.ndarray:
        """P as an n x (nblocks*2N) matrix."""
        ncols = self.blk.nblocks * self.nc
        out = np.zeros((self.lat.V * 12, ncols), dtype=np.complex128)
        for c in range(ncols):
            e = np.zeros(ncols, dtype=np.complex128)
            e[c] = 1.0
            out[:, c] = self.prolong(e.reshape(self.blk.nblocks, self.nc)).ravel()
        return out

    def gamma5_coarse(self, e: np.ndarray) -> np.ndarray:
        """Gamma5^c: +1 on the spin-0,1 aggregates, -1 on the spin-2,3 aggregates."""
        out = np.array(e, copy=True)
        out[..., self.N:] *= -1.0
        return out
