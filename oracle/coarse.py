"""Coarse operator D_c = P^H D P (Sec. 3.2) and its odd-even preconditioned solve (Sec. 6).

With the standard aggregation D_c is a nearest-neighbour coupling on the
periodic coarse lattice of blocks: (D_c x)_a = sum_d B_d(a) x_{a+d}, the nine
2N x 2N blocks being d = 0 (self) and d = +-mu.  Block B_d(a) = P_a^H D_{a,a+d} P_{a+d}
collects every coupling of D between a site of block a and a site of block a+d:
B_0 holds the site term and every hop that stays inside the block, B_{+mu}
(B_{-mu}) the hops in direction +mu (-mu) that leave it.  Blocks are kept per
direction, so on a coarse extent of two (where a+mu = a-mu) both are summed.

Direction index d: 0 = self, 1 + 2 mu = +mu, 2 + 2 mu = -mu.

The coarse solve (Sec. 6): restarted GMRES(30) on the odd-site Schur complement
S = D_oo - D_oe D_ee^{-1} D_eo of D_c (coarse parity = parity of the coarse
coordinate sum), zero initial guess, stopping when the residual of that reduced
system has dropped by the tolerance (5e-2, Table 1); the even part is
recovered as x_e = D_ee^{-1}(b_e - D_eo x_o).

Pins (tests/test_oracle_coarse.py): assembled stencil equals the dense P^H D P
(including coarse extent two); Gamma5^c D_c hermitian (Lemma 3.x (iii));
D_c(m0 + delta) - D_c(m0) = delta I; a tight coarse solve equals the dense solve.
"""
from __future__ import annotations

import numpy as np

from .aggregation import Aggregation
from .dirac import DiracOperator
from .krylov import gmres
from .lattice import Lattice


def direction_index(mu: int, sign: int) -> int:
    return 1 + 2 * mu + (0 if sign > 0 else 1)


class CoarseOperator:
    def __init__(self, D: DiracOperator, agg: Aggregation):
        self.D = D
        self.agg = agg
        blk = agg.blk
        nb, nc, N = blk.nblocks, agg.nc, agg.N
        self.clat = Lattice(blk.nb_dims)
        self.nc = nc
        same = {(mu, s): blk.same_block(mu, s) for mu in range(4) for s in (+1, -1)}
        B = np.zeros((nb, 9, nc, nc), dtype=np.complex128)
        for col in range(nc):
            e = np.zeros((nb, nc), dtype=np.complex128)
            e[:, col] = 1.0
            W = agg.prolong(e)  # column `col` of P on every block at once
            B[:, 0, :, col] = agg.restrict(D.apply(W, hop_mask=lambda mu, s: same[(mu, s)]))
            for mu in range(4):
                for s in (+1, -1):
                    T = D.hop(W, mu, s) * (~same[(mu, s)])[:, None, None]
                    B[:, direction_index(mu, s), :, col] = agg.restrict(T)
        self.B = B

    def shift(self, x: np.ndarray, mu: int, sign: int) -> np.ndarray:
        return self.clat.shift(x, mu, sign)

    def apply_hops(self, x: np.ndarray) -> np.ndarray:
        y = np.zeros_like(x)
        for mu in range(4):
            for s in (+1, -1):
                y = y + np.einsum("aij,aj->ai", self.B[:, direction_index(mu, s)], self.shift(x, mu, s))
        return y

    def apply(self, x: np.ndarray) -> np.ndarray:
        """D_c x for x [nblocks, 2N]."""
        return np.einsum("aij,aj->ai", self.B[:, 0], x) + self.apply_hops(x)

    def dense(self) -> np.ndarray:
        n = self.B.shape[0] * self.nc
        out = np.zeros((n, n), dtype=np.complex128)
        for c in range(n):
            e = np.zeros(n, dtype=np.complex128)
            e[c] = 1.0
            out[:, c] = self.apply(e.reshape(-1, self.nc)).ravel()
        return out


class CoarseSolver:
    def __init__(self, Dc: CoarseOperator, restart: int = 30, tol: float = 5e-2, maxiter: int = 1000):
        self.Dc = Dc
        for n in Dc.clat.dims:
            if n % 2:
                raise ValueError("odd-even coarse solve needs even coarse extents")
        self.restart, self.tol, self.maxiter = int(restart), float(tol), int(maxiter)
        self.even = Dc.clat.parity == 0
        self.odd = ~self.even
        self.Dee_inv = np.zeros_like(Dc.B[:, 0])
        self.Dee_inv[self.even] = np.linalg.inv(Dc.B[self.even, 0])
        self.last_iters = 0

    def _m(self, x, m):
        return x * m[:, None]

    def apply_Dee_inv(self, x):
        return np.einsum("aij,aj->ai", self.Dee_inv, self._m(x, self.even))

    def schur(self, x_o: np.ndarray) -> np.ndarray:
        x_o = self._m(x_o, self.odd)
        d_oo = self._m(np.einsum("aij,aj->ai", self.Dc.B[:, 0], x_o), self.odd)
        return d_oo - self._m(self.Dc.apply_hops(self.apply_Dee_inv(self.Dc.apply_hops(x_o))), self.odd)

    def reduced_rhs(self, b: np.ndarray) -> np.ndarray:
        return self._m(b, self.odd) - self._m(self.Dc.apply_hops(self.apply_Dee_inv(b)), self.odd)

    def back_substitute(self, b: np.ndarray, x_o: np.ndarray) -> np.ndarray:
        x_o = self._m(x_o, self.odd)
        return x_o + self.apply_Dee_inv(b - self.Dc.apply_hops(x_o))

    def solve(self, b: np.ndarray, tol=None, maxiter=None, fixed_iters=None) -> np.ndarray:
        """Approximate D_c^{-1} b.  fixed_iters runs exactly that many GMRES steps (no tolerance)."""
        bo = self.reduced_rhs(b)
        tol = self.tol if tol is None else tol
        maxiter = self.maxiter if maxiter is None else maxiter
        if fixed_iters is not None:
            tol, maxiter = 0.0, int(fixed_iters)
        x_o, info = gmres(self.schur, bo, restart=self.restart, tol=tol, maxiter=maxiter)
        self.last_iters = info["iters"]
        return self.back_substitute(b, x_o)
