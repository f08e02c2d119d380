"""Write oracle_spread.json: how far the oracle's own result moves when its inputs move by one
rounding unit.  Calls only oracle/ (and the seeded input generators).

Why: an iterated FP64 or FP32 quantity (SAP with MR steps, GMRES with a fixed step count, a
V-cycle) amplifies each rounding error by the conditioning of the steps that follow it, so a GPU
result can differ from the oracle's by more than one rounding unit without being wrong.  The GPU
parity tests therefore bound such quantities by a small multiple of the oracle's measured
sensitivity instead of by a hand-picked number.

Perturbation model, for a unit roundoff u (2^-53 for the FP64 path, 2^-24 for the FP32 path):
every real and imaginary part of the inputs the GPU rounds (the gauge links, from which the clover
term is rebuilt; the test vectors; the right-hand side; for the coarse solve the assembled D_c) is
multiplied by (1 + u*xi), xi uniform on [-1, 1].  The spread of a quantity is
max over TRIALS perturbations of max|f(perturbed) - f(exact)| / max|f(exact)|, the same error
measure the tests use.  The cases and seeds are those of tests/test_gpu_parity.py.

usage: python tests/golden/make_oracle_spread.py   (about a minute on one core)
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.aggregation import Aggregation  # noqa: E402
from oracle.coarse import CoarseOperator, CoarseSolver  # noqa: E402
from oracle.dirac import DiracOperator  # noqa: E402
from oracle.mg import Params as OParams  # noqa: E402
from oracle.mg import TwoLevel  # noqa: E402
from oracle.sap import SAP  # noqa: E402
from paper_1303_1377_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_spread.json")
CASES = {
    "4^4/2^4": ((4, 4, 4, 4), (2, 2, 2, 2), 4, 0.1),
    "8^4/4^4": ((8, 8, 8, 8), (4, 4, 4, 4), 6, 0.05),
    "4x4x4x12/2x2x2x6": ((4, 4, 4, 12), (2, 2, 2, 6), 3, 0.1),
}
CSW = 1.0
UNITS = {"64": 2.0 ** -53, "32": 2.0 ** -24}
TRIALS = 3


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


class Perturb:
    def __init__(self, seed):
        self.g = np.random.default_rng(seed)

    def __call__(self, a, u):
        a = np.asarray(a)
        re = a.real * (1 + u * self.g.uniform(-1, 1, a.shape))
        im = a.imag * (1 + u * self.g.uniform(-1, 1, a.shape))
        return (re + 1j * im).astype(np.complex128)


def spread(f, exact, trials=TRIALS):
    return max(rel(f(t), exact) for t in range(trials))


def case_spreads(name):
    dims, block, N, m0 = CASES[name]
    U = synth.gauge_field(dims, 0.5, seed=101)
    v = synth.random_test_vectors(dims, N, seed=102)
    D = DiracOperator(U, dims, m0, CSW)
    pert = Perturb(seed=7)
    out = {}
    # Dslash (FP32 path): links and input rounded
    x = synth.gaussian_spinors(dims, 6, seed=103)
    ref = np.stack([D.apply(x[r]) for r in range(6)])
    u = UNITS["32"]

    def dslash(_):
        Dp = DiracOperator(pert(U, u), dims, m0, CSW)
        xp = pert(x, u)
        return np.stack([Dp.apply(xp[r]) for r in range(6)])

    out["dslash_32"] = spread(dslash, ref)
    # SAP, nu = 1 and 3, MR(4)
    b = synth.gaussian_spinors(dims, 2, seed=104)
    for nu in (1, 3):
        ref = np.stack([SAP(D, block, mr_steps=4).apply(b[r], nu) for r in range(2)])
        for prec, u in UNITS.items():
            def sap(_, u=u, nu=nu):
                Dp = DiracOperator(pert(U, u), dims, m0, CSW)
                bp = pert(b, u)
                sp = SAP(Dp, block, mr_steps=4)
                return np.stack([sp.apply(bp[r], nu) for r in range(2)])
            out[f"sap_nu{nu}_{prec}"] = spread(sap, ref)
    # assembled D_c and its application (FP64 path): links and test vectors rounded
    agg = Aggregation(D.lat, block, v)
    Dc = CoarseOperator(D, agg)
    e = synth.gaussian_coarse(agg.blk.nblocks, agg.nc, 2, seed=106)
    refc = np.stack([Dc.apply(e[r]) for r in range(2)])
    u = UNITS["64"]
    stencils = []

    def stencil(_):
        Dp = DiracOperator(pert(U, u), dims, m0, CSW)
        Dcp = CoarseOperator(Dp, Aggregation(Dp.lat, block, pert(v, u)))
        stencils.append(Dcp)
        return Dcp.B

    out["stencil_64"] = spread(stencil, Dc.B)
    out["apply_Dc_64"] = max(rel(np.stack([Dcp.apply(pert(e[r], u)) for r in range(2)]), refc) for Dcp in stencils)
    # coarse odd-even GMRES with a fixed step count: D_c and the right-hand side rounded
    cs = CoarseSolver(Dc, restart=30, tol=5e-2)
    e = synth.gaussian_coarse(agg.blk.nblocks, agg.nc, 2, seed=107)
    for k in (3, 12, 35):
        ref = np.stack([cs.solve(e[r], fixed_iters=k) for r in range(2)])
        for prec, u in UNITS.items():
            def csolve(_, u=u, k=k):
                Dcp = CoarseOperator.__new__(CoarseOperator)
                Dcp.__dict__.update(Dc.__dict__)
                Dcp.B = pert(Dc.B, u)
                csp = CoarseSolver(Dcp, restart=30, tol=5e-2)
                ep = pert(e, u)
                return np.stack([csp.solve(ep[r], fixed_iters=k) for r in range(2)])
            out[f"coarse_solve_k{k}_{prec}"] = spread(csolve, ref)
    # V-cycle with 10 coarse steps: links, test vectors and right-hand side rounded
    r_in = synth.gaussian_spinors(dims, 2, seed=108)
    mg = TwoLevel(D, OParams(N=N, agg_block=block, sap_block=block, nu=2), vectors=v)
    ref = np.stack([mg.vcycle(r_in[q], coarse_fixed_iters=10) for q in range(2)])
    for prec, u in UNITS.items():
        def vcyc(_, u=u):
            Dp = DiracOperator(pert(U, u), dims, m0, CSW)
            mgp = TwoLevel(Dp, OParams(N=N, agg_block=block, sap_block=block, nu=2), vectors=pert(v, u))
            rp = pert(r_in, u)
            return np.stack([mgp.vcycle(rp[q], coarse_fixed_iters=10) for q in range(2)])
        out[f"vcycle_{prec}"] = spread(vcyc, ref)
    return out


def main():
    res = {"_about": "oracle sensitivity (see the docstring of make_oracle_spread.py): spread of each quantity under "
                     "relative input perturbations of one unit roundoff u (suffix _64: u = 2^-53, _32: u = 2^-24), "
                     f"max over {TRIALS} perturbations",
           "cases": {}}
    for name in CASES:
        res["cases"][name] = case_spreads(name)
        print(name, json.dumps(res["cases"][name]), flush=True)
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
