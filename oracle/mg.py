"""Two-level DD-alpha-AMG: V-cycle, adaptive setup and FGMRES solve (Sec. 4.2, 4.3, 5).

V-cycle with no pre- and nu post-smoothing steps (Sec. 4.2, Eq. iterationmatrix):
    C^(nu) r = P D_c^{-1} P^H r + M_SAP^(nu) (r - D P D_c^{-1} P^H r)
             = M_SAP^(nu) pi_L r + P D_c^{-1} P^H r.
Evaluated as: e_c = D_c^{-1} P^H r (inexact, odd-even GMRES), x = P e_c,
r' = r - D x, x += M_SAP^(nu) r'.

Setup (the loop of Algorithm 1):
  v_1..v_N random;
  for eta = 1..3: for j: v_j <- M_SAP^(eta) v_j
  for eta = 1..n_inv: (re)build P, D_c from v; for j: v_j <- update(v_j); v_j <- v_j/||v_j||
  and, as the paper is silent on it, a final rebuild of P and D_c from the last vectors
  (flag rebuild_after_last).  The update is that of Algorithm 2 (the default,
  setup_update = "ddalpha"): v_j + C^(nu)(v_j - D v_j), one V-cycle iteration on D v = v_j
  started from v_j; or that of Algorithm 1 (setup_update = "idsetup", the inexact-deflation
  setup): C^(nu) v_j, the same iteration started from 0.

Solver: FGMRES(n_kv) right-preconditioned by one V-cycle (Sec. 5), tol 1e-10.
Defaults are Table 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .aggregation import Aggregation
from .coarse import CoarseOperator, CoarseSolver
from .dirac import DiracOperator
from .krylov import fgmres
from .sap import SAP


@dataclass
class Params:
    n_inv: int = 6
    N: int = 20
    agg_block: tuple = (4, 4, 4, 4)
    sap_block: tuple = (4, 4, 4, 4)
    coarse_tol: float = 5e-2
    coarse_restart: int = 30
    coarse_maxiter: int = 1000
    n_kv: int = 25
    tol: float = 1e-10
    nu: int = 2
    mr_steps: int = 4
    max_outer: int = 10000
    rebuild_after_last: bool = True
    setup_update: str = "ddalpha"  # "ddalpha" (Algorithm 2) or "idsetup" (Algorithm 1)
    stats: dict = field(default_factory=dict)


class TwoLevel:
    def __init__(self, D: DiracOperator, params: Params, vectors=None):
        self.D = D
        self.p = params
        self.sap = SAP(D, params.sap_block, params.mr_steps)
        self.coarse_iters = 0
        self.vcycles = 0
        if vectors is not None:
            self.build(vectors)

    def build(self, vectors: np.ndarray):
        self.vectors = np.array(vectors, copy=True)
        self.agg = Aggregation(self.D.lat, self.p.agg_block, self.vectors)
        self.Dc = CoarseOperator(self.D, self.agg)
        self.cs = CoarseSolver(self.Dc, self.p.coarse_restart, self.p.coarse_tol, self.p.coarse_maxiter)

    def vcycle(self, r: np.ndarray, coarse_fixed_iters=None) -> np.ndarray:
        ec = self.cs.solve(self.agg.restrict(r), fixed_iters=coarse_fixed_iters)
        self.coarse_iters += self.cs.last_iters
        self.vcycles += 1
        x = self.agg.prolong(ec)
        r2 = r - self.D.apply(x)
        return x + self.sap.apply(r2, self.p.nu)

    def setup_update(self, v: np.ndarray) -> np.ndarray:
        """The test-vector update of the setup's second phase, before normalisation."""
        if self.p.setup_update == "idsetup":
            return self.vcycle(v)  # Algorithm 1: C^(nu) v
        if self.p.setup_update != "ddalpha":
            raise ValueError("setup_update must be 'ddalpha' or 'idsetup'")
        return v + self.vcycle(v - self.D.apply(v))  # Algorithm 2: v + C^(nu) (v - D v)

    def setup(self, v0: np.ndarray):
        """Algorithm 2 (default) or Algorithm 1, per Params.setup_update."""
        v = np.array(v0, dtype=np.complex128, copy=True)
        for eta in (1, 2, 3):
            for j in range(v.shape[0]):
                v[j] = self.sap.apply(v[j], eta)
        for _ in range(self.p.n_inv):
            self.build(v)
            for j in range(v.shape[0]):
                v[j] = self.setup_update(v[j])
                v[j] = v[j] / np.sqrt(np.sum(np.abs(v[j]) ** 2))
        if self.p.rebuild_after_last or self.p.n_inv == 0:
            self.build(v)
        else:
            self.vectors = v
        return v

    def solve(self, b: np.ndarray, x0=None, tol=None):
        tol = self.p.tol if tol is None else tol
        self.coarse_iters = 0
        self.vcycles = 0
        x, info = fgmres(self.D.apply, self.vcycle, b, x0=x0, n_kv=self.p.n_kv, tol=tol, maxiter=self.p.max_outer)
        info["coarse_iters"] = self.coarse_iters
        return x, info
