"""Multilevel DD-alpha-AMG: the two-level method applied recursively to its own coarse system.

Test infrastructure only (the oracle): plain FP64 numpy, imported by tests alone.

Sec. 3 states that the coarse equation D_c e = P^H r can itself be solved by an algorithm of the
same two-level kind, recursively, until the operator is small enough to solve directly, and that
Gamma5-compatible aggregation (Sec. 3.2) is what keeps D_c fit for that recursion; Sec. 6.4 reports a
preliminary 2-, 3- and 4-level version.  The paper prints no algorithm for it, so this module fixes
the following readings (each is listed with the other readings of the paper):

  ML1  Level operators.  D_0 = D; D_{l+1} = P_l^H D_l P_l (Sec. 3.2).  Every D_l is a coupling of
       nearest neighbours on a periodic lattice, stored as nine blocks per site (self, +-mu), like
       D_c.  Its Gamma5 is +1 on the first half of a site's components and -1 on the second: the
       coarse Gamma5^c of Sec. 3.2 (aggregates of spins 0,1 first).  The fine D fits the same
       form (12 components, spins 0,1 first), so one class describes every level.
  ML2  Smoother on a level: red-black SAP over lattice blocks of that level's sites, each block
       solved by MR on its odd-site Schur complement with back-substitution (Sec. 2.3, Sec. 6),
       exactly as on the fine level; site parity and block colour as on the fine lattice.
  ML3  Aggregation on a level: lattice blocks x {Gamma5 = +1 components, Gamma5 = -1 components},
       local orthonormalisation of the level's test vectors in the order v_1..v_N (Sec. 3.1-3.2
       with Gamma5^c in place of Gamma5).
  ML4  Coarse-system solve on an intermediate level l+1 (not the coarsest): inner = "fgmres"
       (default) runs FGMRES(inner_kv) on D_{l+1}, right-preconditioned by the level-(l+1)
       V-cycle, from a zero guess until the relative residual drops to inner_tol (5e-2: the low
       accuracy the coarse solve needs, Sec. 4.2 and Table 1) -- the two-level solver of Sec. 5
       applied to the coarse system; inner = "vcycle" applies the level-(l+1) V-cycle once (the
       alternating smoother / coarse correction of Sec. 3, one sweep).  The coarsest system is
       solved by the odd-even GMRES(30) of Sec. 6 to coarse_tol, as in the two-level method.
  ML5  Setup, finest level first.  Level l runs the two-level setup (Algorithm 1 phase 1, then
       Algorithm 2 -- or Algorithm 1's update -- per its Params) on D_l, its coarse solves done by
       the odd-even GMRES on D_{l+1}; when it has finished, level l+1 starts the same setup from
       its own random test vectors.  The recursion of ML4 is switched on after the setup.

Fields on a level >= 1 are [V_l, n_l] complex arrays (n_l = 2 N_{l-1}); coarse vectors of the fine
two-level classes ([nblocks, 2N]) are exactly such fields.

Pins (tests/test_oracle_multilevel.py): the fine D written as a stencil equals D; the generic
level classes applied to the fine D reproduce the fine SAP, aggregation and D_c; on a coarse level
the aggregation is orthonormal, Gamma5-compatible and spans its vectors, the Galerkin stencil equals
the dense P^H D_l P, exact-block SAP equals the dense sum over (I - K D)^k K; the three-level V-cycle
equals the dense nested iteration matrix; with a tight inner solve it equals the two-level V-cycle
with an exact coarse solve; the three-level solve matches a dense LU.
"""
from __future__ import annotations

import numpy as np

from .aggregation import modified_gram_schmidt
from .coarse import CoarseSolver, direction_index
from .krylov import fgmres
from .lattice import Blocking, Lattice
from .mg import Params, TwoLevel

_DIRS = [(mu, s) for mu in range(4) for s in (+1, -1)]


class StencilOperator:
    """(A x)_a = B_0(a) x_a + sum_{mu, s} B_{s mu}(a) x_{a + s mu} on a periodic lattice (ML1).

    B: [V, 9, n, n] with the direction index of the coarse operator (0 = self, 1 + 2 mu = +mu,
    2 + 2 mu = -mu); both blocks are kept where an extent is two (a + mu = a - mu) and summed on
    apply.
    """

    def __init__(self, lat: Lattice, B: np.ndarray):
        self.lat = lat
        self.B = np.asarray(B, dtype=np.complex128)
        if self.B.shape[:2] != (lat.V, 9) or self.B.shape[2] != self.B.shape[3] or self.B.shape[2] % 2:
            raise ValueError("stencil blocks must be [V, 9, n, n] with n even")
        self.n = self.B.shape[2]

    # the coarse-solve interface (clat, nc, B, apply_hops) of the two-level coarse operator
    @property
    def clat(self) -> Lattice:
        return self.lat

    @property
    def nc(self) -> int:
        return self.n

    @property
    def V(self) -> int:
        return self.lat.V

    @classmethod
    def from_dirac(cls, D) -> "StencilOperator":
        """The fine Dirac operator as a stencil: B_0 = site term, B_{s mu} = the hop's 12 x 12 block,
        read off by applying each hop to a field that is the identity at every site."""
        V = D.V
        eye = np.broadcast_to(np.eye(12, dtype=np.complex128).reshape(1, 4, 3, 12), (V, 4, 3, 12))
        B = np.zeros((V, 9, 12, 12), dtype=np.complex128)
        B[:, 0] = D.A
        for mu, s in _DIRS:
            B[:, direction_index(mu, s)] = D.hop(eye, mu, s).reshape(V, 12, 12)
        return cls(D.lat, B)

    def hop(self, x: np.ndarray, mu: int, sign: int) -> np.ndarray:
        """The coupling to x + sign*mu: y_a = B_{sign mu}(a) x_{a + sign mu}."""
        return np.einsum("aij,aj->ai", self.B[:, direction_index(mu, sign)], self.lat.shift(x, mu, sign))

    def apply_site(self, x: np.ndarray) -> np.ndarray:
        return np.einsum("aij,aj->ai", self.B[:, 0], x)

    def apply_hops(self, x: np.ndarray, keep=None) -> np.ndarray:
        """Sum of the eight couplings; keep(mu, sign) -> bool[V] keeps a coupling only where True."""
        y = np.zeros_like(x)
        for mu, s in _DIRS:
            h = self.hop(x, mu, s)
            if keep is not None:
                h = h * keep(mu, s)[:, None]
            y = y + h
        return y

    def apply(self, x: np.ndarray, keep=None) -> np.ndarray:
        return self.apply_site(x) + self.apply_hops(x, keep)

    def gamma5(self, x: np.ndarray) -> np.ndarray:
        out = np.array(x, copy=True)
        out[..., self.n // 2:] *= -1.0
        return out

    def dense(self) -> np.ndarray:
        m = self.V * self.n
        eye = np.eye(m, dtype=np.complex128).reshape(self.V, self.n, m)
        out = np.zeros((m, m), dtype=np.complex128)
        for c in range(m):
            out[:, c] = self.apply(eye[:, :, c]).ravel()
        return out


def _block_sum(values: np.ndarray, block_of_site: np.ndarray, nblocks: int) -> np.ndarray:
    re = np.bincount(block_of_site, weights=values.real, minlength=nblocks)
    im = np.bincount(block_of_site, weights=values.imag, minlength=nblocks)
    return re + 1j * im


class StencilSAP:
    """Red-black SAP on a stencil level (ML2): one iteration z <- (I - K A) z + K b with
    K = B_black (I - A B_red) + B_red; the block solves by MR(mr_steps) on the odd-site Schur
    complement S = A_oo - A_oe A_ee^{-1} A_eo of the block (couplings that leave the block
    dropped), zero guess, then x_e = A_ee^{-1} (r_e - A_eo x_o).  A block whose sites are all
    even needs no MR step: its solve is the back-substitution alone."""

    def __init__(self, A: StencilOperator, block_dims, mr_steps: int = 4, block_solver: str = "mr"):
        self.A = A
        self.blk = Blocking(A.lat, block_dims)
        for nb in self.blk.nb_dims:
            if nb % 2:
                raise ValueError("red-black SAP needs an even number of blocks in every direction")
        self.mr_steps = int(mr_steps)
        self.block_solver = block_solver
        self.same = {(mu, s): self.blk.same_block(mu, s) for mu, s in _DIRS}
        self.site_colour = self.blk.colour[self.blk.block_of_site]
        self.even = A.lat.parity == 0
        self.odd = ~self.even
        self.Aee_inv = np.zeros_like(A.B[:, 0])
        self.Aee_inv[self.even] = np.linalg.inv(A.B[self.even, 0])
        self._dense = None

    def _mask(self, f: np.ndarray, m: np.ndarray) -> np.ndarray:
        return f * m[:, None]

    def block_hops(self, x: np.ndarray) -> np.ndarray:
        return self.A.apply_hops(x, keep=lambda mu, s: self.same[(mu, s)])

    def apply_Aee_inv(self, x: np.ndarray) -> np.ndarray:
        return np.einsum("aij,aj->ai", self.Aee_inv, self._mask(x, self.even))

    def schur(self, rho: np.ndarray) -> np.ndarray:
        rho = self._mask(rho, self.odd)
        t_e = self._mask(self.block_hops(rho), self.even)
        t_o = self._mask(self.block_hops(self.apply_Aee_inv(t_e)), self.odd)
        return self._mask(self.A.apply_site(rho), self.odd) - t_o

    def mr_block_solve(self, r: np.ndarray, colour: int, steps=None, history=None) -> np.ndarray:
        steps = self.mr_steps if steps is None else steps
        sel = self.site_colour == colour
        E, O = sel & self.even, sel & self.odd
        r_e, r_o = self._mask(r, E), self._mask(r, O)
        rho = r_o - self._mask(self.block_hops(self.apply_Aee_inv(r_e)), O)
        x = np.zeros_like(r)
        nb, bos = self.blk.nblocks, self.blk.block_of_site
        for _ in range(steps):
            t = self._mask(self.schur(rho), O)
            num = _block_sum(np.sum(np.conj(t) * rho, axis=1), bos, nb)
            den = _block_sum(np.sum(np.abs(t) ** 2, axis=1), bos, nb).real
            ok = den > 1e-280
            alpha = np.where(ok, num / np.where(ok, den, 1.0), 0.0)[bos][:, None]
            x = x + alpha * rho
            rho_new = rho - alpha * t
            if history is not None:
                history.append((t, rho_new))
            rho = rho_new
        x_e = self.apply_Aee_inv(r_e - self._mask(self.block_hops(x), E))
        return self._mask(x, O) + self._mask(x_e, E)

    def exact_block_solve(self, r: np.ndarray, colour: int) -> np.ndarray:
        if self._dense is None:
            self._dense = self.A.dense()
        n = self.A.n
        rf = r.reshape(-1)
        out = np.zeros_like(rf)
        for b in np.nonzero(self.blk.colour == colour)[0]:
            idx = (self.blk.sites[b][:, None] * n + np.arange(n)[None, :]).ravel()
            out[idx] = np.linalg.solve(self._dense[np.ix_(idx, idx)], rf[idx])
        return out.reshape(r.shape)

    def block_solve(self, r: np.ndarray, colour: int) -> np.ndarray:
        if self.block_solver == "exact":
            return self.exact_block_solve(r, colour)
        return self.mr_block_solve(r, colour)

    def iterate(self, z: np.ndarray, b: np.ndarray) -> np.ndarray:
        for colour in (0, 1):
            z = z + self.block_solve(b - self.A.apply(z), colour)
        return z

    def apply(self, b: np.ndarray, nu: int) -> np.ndarray:
        z = np.zeros_like(b)
        for _ in range(nu):
            z = self.iterate(z, b)
        return z


class StencilAggregation:
    """Gamma5-compatible aggregation on a stencil level (ML3): P restricted to aggregate
    (block j, half h) is the ordered orthonormal basis of the level's test vectors there."""

    def __init__(self, lat: Lattice, block_dims, vectors: np.ndarray):
        """vectors: [N, V, n] test vectors of the level."""
        self.lat = lat
        self.blk = Blocking(lat, block_dims)
        v = np.asarray(vectors, dtype=np.complex128)
        self.N, self.n = v.shape[0], v.shape[2]
        nb, bv, h = self.blk.nblocks, self.blk.bvol, v.shape[2] // 2
        vb = np.moveaxis(v, 0, -1)[self.blk.sites]  # [nb, bvol, n, N]
        M = np.stack([vb[:, :, :h].reshape(nb, bv * h, self.N), vb[:, :, h:].reshape(nb, bv * h, self.N)], axis=1)
        self.P = modified_gram_schmidt(M)  # [nb, 2, bvol*h, N]

    @property
    def nc(self) -> int:
        return 2 * self.N

    def restrict(self, r: np.ndarray) -> np.ndarray:
        nb, bv, h = self.blk.nblocks, self.blk.bvol, self.n // 2
        rb = r[self.blk.sites]  # [nb, bvol, n]
        rh = np.stack([rb[:, :, :h].reshape(nb, bv * h), rb[:, :, h:].reshape(nb, bv * h)], axis=1)
        return np.einsum("bhkj,bhk->bhj", np.conj(self.P), rh).reshape(nb, self.nc)

    def prolong(self, e: np.ndarray) -> np.ndarray:
        nb, bv, h = self.blk.nblocks, self.blk.bvol, self.n // 2
        rh = np.einsum("bhkj,bhj->bhk", self.P, e.reshape(nb, 2, self.N)).reshape(nb, 2, bv, h)
        out = np.zeros((self.lat.V, self.n), dtype=np.complex128)
        out[self.blk.sites] = np.concatenate([rh[:, 0], rh[:, 1]], axis=2)
        return out

    def dense(self) -> np.ndarray:
        ncols = self.blk.nblocks * self.nc
        out = np.zeros((self.lat.V * self.n, ncols), dtype=np.complex128)
        for c in range(ncols):
            e = np.zeros(ncols, dtype=np.complex128)
            e[c] = 1.0
            out[:, c] = self.prolong(e.reshape(self.blk.nblocks, self.nc)).ravel()
        return out


class StencilCoarse(StencilOperator):
    """D_{l+1} = P_l^H D_l P_l as a stencil on the lattice of aggregates (ML1): B_0(a) collects the
    site blocks and every coupling inside aggregate a, B_{s mu}(a) the couplings in direction s mu
    that leave it, each projected by P_a^H ... P_{a + s mu}."""

    def __init__(self, A: StencilOperator, agg: StencilAggregation):
        blk = agg.blk
        nb, nc = blk.nblocks, agg.nc
        same = {(mu, s): blk.same_block(mu, s) for mu, s in _DIRS}
        B = np.zeros((nb, 9, nc, nc), dtype=np.complex128)
        for col in range(nc):
            e = np.zeros((nb, nc), dtype=np.complex128)
            e[:, col] = 1.0
            W = agg.prolong(e)  # column `col` of P on every aggregate at once
            B[:, 0, :, col] = agg.restrict(A.apply(W, keep=lambda mu, s: same[(mu, s)]))
            for mu, s in _DIRS:
                T = A.hop(W, mu, s) * (~same[(mu, s)])[:, None]
                B[:, direction_index(mu, s), :, col] = agg.restrict(T)
        super().__init__(Lattice(blk.nb_dims), B)


class StencilTwoLevel(TwoLevel):
    """The two-level method (V-cycle, setup, FGMRES of Sec. 4-5) on a stencil level."""

    def __init__(self, A: StencilOperator, params: Params, vectors=None):
        self.D = A
        self.p = params
        self.sap = StencilSAP(A, params.sap_block, params.mr_steps)
        self.coarse_iters = 0
        self.vcycles = 0
        if vectors is not None:
            self.build(vectors)

    def build(self, vectors: np.ndarray):
        self.vectors = np.array(vectors, copy=True)
        self.agg = StencilAggregation(self.D.lat, self.p.agg_block, self.vectors)
        self.Dc = StencilCoarse(self.D, self.agg)
        self.cs = CoarseSolver(self.Dc, self.p.coarse_restart, self.p.coarse_tol, self.p.coarse_maxiter)


class RecursiveCoarseSolver:
    """Approximate D_{l+1}^{-1} b by the method of level l+1 (ML4)."""

    def __init__(self, level: TwoLevel, inner: str = "fgmres", n_kv: int = 10, tol: float = 5e-2, maxiter: int = 1000):
        if inner not in ("fgmres", "vcycle"):
            raise ValueError("inner must be 'fgmres' or 'vcycle'")
        self.level, self.inner = level, inner
        self.n_kv, self.tol, self.maxiter = int(n_kv), float(tol), int(maxiter)
        self.last_iters = 0

    def solve(self, b: np.ndarray, tol=None, maxiter=None, fixed_iters=None) -> np.ndarray:
        if self.inner == "vcycle":
            self.last_iters = 1
            return self.level.vcycle(b)
        tol = self.tol if tol is None else tol
        maxiter = self.maxiter if maxiter is None else maxiter
        if fixed_iters is not None:
            tol, maxiter = 0.0, int(fixed_iters)
        x, info = fgmres(self.level.D.apply, self.level.vcycle, b, n_kv=self.n_kv, tol=tol, maxiter=maxiter)
        self.last_iters = info["iters"]
        return x


class MultiLevel:
    """L-level DD-alpha-AMG (L = len(params) + 1): params[l] are the Table 1 style parameters of the
    pair (level l, level l+1) -- its aggregates, SAP blocks, N, nu, MR steps, setup -- and, for the
    last pair, the coarsest solve (odd-even GMRES, coarse_tol, coarse_restart).  params[0].n_kv,
    tol and max_outer are those of the outer FGMRES."""

    def __init__(self, D, params: list, inner: str = "fgmres", inner_kv: int = 10, inner_tol: float = 5e-2,
                 inner_maxiter: int = 1000):
        if len(params) < 1:
            raise ValueError("need at least one level pair")
        self.D = D
        self.params = list(params)
        self.inner, self.inner_kv, self.inner_tol, self.inner_maxiter = inner, inner_kv, inner_tol, inner_maxiter
        self.levels = [TwoLevel(D, self.params[0])]

    @property
    def n_levels(self) -> int:
        return len(self.params) + 1

    def _next(self, l: int) -> StencilTwoLevel:
        """Level l+1's two-level object on D_{l+1} = the coarse operator level l has just built."""
        Dc = self.levels[l].Dc
        A = Dc if isinstance(Dc, StencilOperator) else StencilOperator(Dc.clat, Dc.B)
        return StencilTwoLevel(A, self.params[l + 1])

    def _link(self):
        """Switch the coarse solves of all but the last pair to the recursion of ML4."""
        for l in range(len(self.levels) - 1):
            self.levels[l].cs = RecursiveCoarseSolver(self.levels[l + 1], self.inner, self.inner_kv, self.inner_tol,
                                                      self.inner_maxiter)

    def build(self, vectors: list):
        """The hierarchy from given test vectors: vectors[l] are level l's ([N, V, 4, 3] on level 0,
        [N, V_l, n_l] above)."""
        if len(vectors) != len(self.params):
            raise ValueError("one set of test vectors per level pair")
        self.levels = self.levels[:1]
        self.levels[0].build(vectors[0])
        for l in range(1, len(self.params)):
            self.levels.append(self._next(l - 1))
            self.levels[l].build(vectors[l])
        self._link()

    def setup(self, v0_fine: np.ndarray, initial_vectors):
        """ML5: initial_vectors(l, V_l, n_l, N_l) -> [N_l, V_l, n_l] supplies each coarser level's
        random start (the random numbers are inputs, not drawn here)."""
        self.levels = self.levels[:1]
        out = [self.levels[0].setup(v0_fine)]
        for l in range(1, len(self.params)):
            nxt = self._next(l - 1)
            self.levels.append(nxt)
            v0 = np.asarray(initial_vectors(l, nxt.D.V, nxt.D.n, self.params[l].N), dtype=np.complex128)
            out.append(nxt.setup(v0))
        self._link()
        return out

    def vcycle(self, r: np.ndarray) -> np.ndarray:
        return self.levels[0].vcycle(r)

    def solve(self, b: np.ndarray, x0=None, tol=None):
        p = self.params[0]
        tol = p.tol if tol is None else tol
        for lv in self.levels:
            lv.coarse_iters, lv.vcycles = 0, 0
        x, info = fgmres(self.D.apply, self.vcycle, b, x0=x0, n_kv=p.n_kv, tol=tol, maxiter=p.max_outer)
        info["vcycles_per_level"] = [lv.vcycles for lv in self.levels]
        info["coarsest_iters"] = self.levels[-1].coarse_iters
        return x, info
