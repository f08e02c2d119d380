"""Red-black multiplicative Schwarz (SAP) of Sec. 2.3 with the local solver of Sec. 6.

One SAP iteration (Sec. 2.3, Eq. SAP_1step):  z <- (I - K D) z + K b,
K = B_black (I - D B_red) + B_red,  B_colour = sum_{i in colour} I_i D_i^{-1} I_i^T,
D_i = I_i^T D I_i the restriction of D to the variables of lattice-block i.
Applied literally: first the red blocks solve D_i e_i = (b - D z)|_i and z += e,
then the residual is recomputed and the black blocks do the same.
M_SAP^(nu) b is nu such iterations from z = 0.

Local solver (Sec. 6, Table 1): a fixed number (4) of minimal-residual steps on
the odd-even reduced block system (Schur complement on the block's odd sites,
the same choice of odd sites as the global odd-even preconditioning in Sec. 6),
initial guess 0, followed by back-substitution on the even sites.  The MR step
is restarted GMRES with restart length one:
    alpha = <S rho, rho> / <S rho, S rho>,  x += alpha rho,  rho -= alpha S rho.

Pins (tests/test_oracle_sap.py): many MR steps converge to the dense block
solve; with exact block solves one iteration equals the dense K b and nu
iterations equal sum_k (I-KD)^k K b; the MR residual is orthogonal to S rho.
"""
from __future__ import annotations

import numpy as np

from .dirac import DiracOperator
from .lattice import Blocking


def _block_sum(values: np.ndarray, block_of_site: np.ndarray, nblocks: int) -> np.ndarray:
    """Sum a per-site complex quantity over each block."""
    re = np.bincount(block_of_site, weights=values.real, minlength=nblocks)
    im = np.bincount(block_of_site, weights=values.imag, minlength=nblocks)
    return re + 1j * im


class SAP:
    def __init__(self, D: DiracOperator, block_dims, mr_steps: int = 4, block_solver: str = "mr"):
        self.D = D
        self.blk = Blocking(D.lat, block_dims)
        for n in self.blk.nb_dims:
            if n % 2:
                raise ValueError("red-black SAP needs an even number of blocks in every direction")
        self.mr_steps = int(mr_steps)
        self.block_solver = block_solver
        self.same = {(mu, s): self.blk.same_block(mu, s) for mu in range(4) for s in (+1, -1)}
        self.site_colour = self.blk.colour[self.blk.block_of_site]
        self.even = D.lat.parity == 0
        self.odd = ~self.even
        self.Ainv = np.linalg.inv(D.A)
        self._dense = None

    # -- block-restricted pieces ------------------------------------------------
    def _mask(self, f: np.ndarray, m: np.ndarray) -> np.ndarray:
        return f * m.reshape((-1,) + (1,) * (f.ndim - 1))

    def block_hops(self, psi: np.ndarray) -> np.ndarray:
        """Hopping part of D with every coupling that leaves its block removed."""
        return self.D.apply(psi, hop_mask=lambda mu, s: self.same[(mu, s)], with_site=False)

    def apply_Ainv(self, psi: np.ndarray) -> np.ndarray:
        p = psi.reshape(self.D.V, 12)
        return np.einsum("xij,xj->xi", self.Ainv, p).reshape(psi.shape)

    def schur(self, rho: np.ndarray) -> np.ndarray:
        """S rho = A_oo rho - D_oe A_ee^{-1} D_eo rho on the odd sites of the blocks."""
        t_e = self._mask(self.block_hops(rho), self.even)
        t_o = self._mask(self.block_hops(self.apply_Ainv(t_e)), self.odd)
        return self._mask(self.D.apply_site(rho), self.odd) - t_o

    def mr_block_solve(self, r: np.ndarray, colour: int, steps=None, history=None) -> np.ndarray:
        """Approximate B_colour r by odd-even MR on every block of one colour."""
        steps = self.mr_steps if steps is None else steps
        sel = self.site_colour == colour
        E = sel & self.even
        O = sel & self.odd
        r_e = self._mask(r, E)
        r_o = self._mask(r, O)
        # reduced right-hand side b' = r_o - D_oe A_ee^{-1} r_e
        bprime = r_o - self._mask(self.block_hops(self.apply_Ainv(r_e)), O)
        x = np.zeros_like(r)
        rho = bprime
        for _ in range(steps):
            t = self._mask(self.schur(rho), O)
            num = _block_sum(np.sum(np.conj(t) * rho, axis=(1, 2)), self.blk.block_of_site, self.blk.nblocks)
            den = _block_sum(np.sum(np.abs(t) ** 2, axis=(1, 2)), self.blk.block_of_site, self.blk.nblocks).real
            ok = den > 1e-280  # a block whose reduced residual is already zero takes no step
            alpha = np.where(ok, num / np.where(ok, den, 1.0), 0.0)
            a_site = alpha[self.blk.block_of_site][:, None, None]
            x = x + a_site * rho
            rho_new = rho - a_site * t
            if history is not None:
                history.append((t, rho_new))
            rho = rho_new
        # back-substitution x_e = A_ee^{-1} (r_e - D_eo x_o)
        x_e = self.apply_Ainv(r_e - self._mask(self.block_hops(x), E))
        return self._mask(x, O) + self._mask(x_e, E)

    def exact_block_solve(self, r: np.ndarray, colour: int) -> np.ndarray:
        """B_colour r with dense solves of every D_i (tiny lattices only)."""
        if self._dense is None:
            self._dense = self.D.dense()
        Dd = self._dense
        rf = r.reshape(-1)
        out = np.zeros_like(rf)
        for b in np.nonzero(self.blk.colour == colour)[0]:
            idx = (self.blk.sites[b][:, None] * 12 + np.arange(12)[None, :]).ravel()
            out[idx] = np.linalg.solve(Dd[np.ix_(idx, idx)], rf[idx])
        return out.reshape(r.shape)

    def block_solve(self, r: np.ndarray, colour: int) -> np.ndarray:
        if self.block_solver == "exact":
            return self.exact_block_solve(r, colour)
        return self.mr_block_solve(r, colour)

    # -- the Schwarz iteration ----------------------------------------------------
    def iterate(self, z: np.ndarray, b: np.ndarray) -> np.ndarray:
        """One red-black iteration z <- (I - K D) z + K b."""
        for colour in (0, 1):
            r = b - self.D.apply(z)
            z = z + self.block_solve(r, colour)
        return z

    def apply(self, b: np.ndarray, nu: int) -> np.ndarray:
        """M_SAP^(nu) b: nu iterations from z = 0."""
        z = np.zeros_like(b)
        for _ in range(nu):
            z = self.iterate(z, b)
        return z
