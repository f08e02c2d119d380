"""Two levels against three on one near-critical lattice: iteration counts and coarse-level work.

Test infrastructure only (the oracle).  Sec. 6.4 reports that going from two to three levels speeds
the solve up most near the critical mass, because the coarse system is the ill-conditioned part.
Timings of this FP64 numpy oracle say nothing about a GPU, so this script counts work instead:

  two levels   per solve: outer FGMRES iterations; odd-even GMRES steps on D_1 (each one
               application of the Schur complement of D_1, about one D_1 application);
  three levels per solve: outer FGMRES iterations; FGMRES steps on D_1 (one D_1 application and one
               level-1 V-cycle each); level-1 V-cycles; odd-even GMRES steps on D_2 (D_2 has
               1/prod(block1) of D_1's sites and N_1/N of its components per site).

Both hierarchies share the level-0 setup (the two-level Algorithm 2 run), so the comparison isolates
the coarse solve.  Writes paper_1303_1377_gb300/workloads.json["levels_study"] and prints it.

usage: python -m oracle.compare_levels [--N 8] [--N1 8] [--n-inv 3] [--workload lattice_8x8x8x8]
       [--dims 16,16,16,16 --m0 -0.93 --key levels_study_16x16x16x16]   (another volume or mass of
       the workload's ensemble parameters eps and seed)
       [--inner vcycle | --inner-tol 0.1]   (the level-1 solve inside the fine V-cycle, reading ML4)
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from paper_1303_1377_gb300 import synth

from .dirac import DiracOperator
from .mg import Params, TwoLevel
from .multilevel import MultiLevel

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1303_1377_gb300", "workloads.json")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=8)
    ap.add_argument("--N1", type=int, default=8)
    ap.add_argument("--n-inv", type=int, default=3)
    ap.add_argument("--workload", default="lattice_8x8x8x8")
    ap.add_argument("--dims", default=None)
    ap.add_argument("--m0", type=float, default=None)
    ap.add_argument("--key", default="levels_study")
    ap.add_argument("--inner", default="fgmres", choices=["fgmres", "vcycle"])
    ap.add_argument("--inner-tol", type=float, default=5e-2)
    a = ap.parse_args()
    rec = json.load(open(OUT))[a.workload]
    dims, eps, seed, m0 = tuple(rec["dims"]), rec["eps"], rec["seed"], rec["m0"]
    if a.dims:
        dims = tuple(int(d) for d in a.dims.split(","))
    if a.m0 is not None:
        m0 = a.m0
    D = DiracOperator(synth.gauge_field(dims, eps, seed), dims, m0, rec.get("c_sw", 1.0))
    blk = (2, 2, 2, 2)
    p0 = Params(N=a.N, agg_block=blk, sap_block=blk, n_inv=a.n_inv, nu=2)
    p1 = Params(N=a.N1, agg_block=blk, sap_block=blk, n_inv=a.n_inv, nu=2)
    t0 = time.perf_counter()
    two = TwoLevel(D, p0)
    two.setup(synth.random_test_vectors(dims, a.N, seed=seed + 7))
    b = synth.gaussian_spinors(dims, 1, seed=seed + 9)[0]
    # two levels: the coarse solve is the odd-even GMRES on D_1
    x2, info2 = two.solve(b)
    res2 = float(np.linalg.norm(b - D.apply(x2)) / np.linalg.norm(b))
    # three levels on the same level 0: level-1 setup, then FGMRES on D_1 with the level-1 V-cycle
    ml = MultiLevel(D, [p0, p1], inner=a.inner, inner_tol=a.inner_tol)
    ml.levels = [two]
    l1 = ml._next(0)
    ml.levels.append(l1)
    l1.setup(synth.gaussian_coarse(l1.D.V, l1.D.n, a.N1, seed=seed + 8))
    ml._link()
    t_setup = time.perf_counter() - t0
    out = {"workload": a.workload, "dims": list(dims), "m0": m0, "N": a.N, "N1": a.N1, "n_inv": a.n_inv, "blocks": list(blk),
           "level1_sites": int(l1.D.V), "level2_sites": int(l1.Dc.V), "seconds_setups_and_two_level_solve": t_setup}
    out["two_level"] = {"outer_iterations": int(info2["iters"]), "gmres_steps_D1": int(info2["coarse_iters"]), "rel_residual": res2}
    x3, info3 = ml.solve(b)
    res3 = float(np.linalg.norm(b - D.apply(x3)) / np.linalg.norm(b))
    out["three_level"] = {"outer_iterations": int(info3["iters"]), "fgmres_steps_D1": int(ml.levels[0].coarse_iters),
                          "level1_vcycles": int(info3["vcycles_per_level"][1]), "gmres_steps_D2": int(info3["coarsest_iters"]),
                          "rel_residual": res3}
    out["eps"], out["seed"], out["inner"], out["inner_tol"] = eps, seed, a.inner, a.inner_tol
    data = json.load(open(OUT))
    data[a.key] = out
    json.dump(data, open(OUT, "w"), indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
