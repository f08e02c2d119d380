"""FGMRES iterations per solve of the oracle's full method on a workload's 8^4 counterpart.

Test infrastructure only (the oracle): runs the adaptive setup (Algorithm 2, Table 1 defaults:
n_inv = 6, N = 20, nu = 2, 4^4 blocks) on the 8^4 lattice with the workload's eps, seed, c_sw
and m0, solves one point source to a relative residual of 1e-10 (Sec. 5) and records the
iteration count in paper_1303_1377_gb300/workloads.json under
"fgmres_iterations_8x8x8x8" -> <workload>. The benchmark's reference arm times the oracle per
FGMRES iteration on the host and multiplies by this count (and by the volume ratio), taking the
weak volume dependence of a multigrid iteration count as its assumption.

usage: python -m oracle.count_iterations --workload 32x32x32x64 --eps 0.5 --seed 3 --m0 -0.931885
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

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1303_1377_gb300", "workloads.json")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", required=True)
    ap.add_argument("--eps", type=float, required=True)
    ap.add_argument("--seed", type=int, required=True)
    ap.add_argument("--m0", type=float, required=True)
    ap.add_argument("--csw", type=float, default=1.0)
    a = ap.parse_args()
    dims = (8, 8, 8, 8)
    t0 = time.perf_counter()
    D = DiracOperator(synth.gauge_field(dims, a.eps, a.seed), dims, a.m0, a.csw)
    mg = TwoLevel(D, Params())
    mg.setup(synth.random_test_vectors(dims, mg.p.N, seed=a.seed + 7))
    t_setup = time.perf_counter() - t0
    b = np.zeros((D.V, 4, 3), dtype=np.complex128)
    b[0, 0, 0] = 1.0
    t1 = time.perf_counter()
    x, info = mg.solve(b)
    t_solve = time.perf_counter() - t1
    res = float(np.linalg.norm(b - D.apply(x)) / np.linalg.norm(b))
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data.setdefault("fgmres_iterations_8x8x8x8", {})[a.workload] = {
        "iterations": int(info["iters"]), "rel_residual": res, "eps": a.eps, "seed": a.seed, "m0": a.m0, "c_sw": a.csw,
        "setup_seconds": t_setup, "solve_seconds": t_solve, "params": "Table 1 defaults (n_inv=6, N=20, nu=2, 4^4 blocks)",
    }
    json.dump(data, open(OUT, "w"), indent=1)
    print(json.dumps(data["fgmres_iterations_8x8x8x8"][a.workload]))


if __name__ == "__main__":
    main()
