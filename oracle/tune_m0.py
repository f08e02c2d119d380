"""Choose the bare mass m0 of the synthetic workloads from the oracle's spectrum.

Test infrastructure: writes paper_1303_1377_gb300/workloads.json using only the
oracle.  For a gauge field U(eps, seed) the leftmost eigenvalue lambda_L of
D(m0 = 0) is found by implicitly restarted Arnoldi (scipy ARPACK, smallest real
part); since m0 enters D only as (m0 + 4) I (Sec. 2.2), D(m0) has its leftmost
eigenvalue at lambda_L + m0, and m0 = -Re(lambda_L) + gap puts the smallest
|eigenvalue| at about `gap` when lambda_L is real (Gamma5 pairing, Lemma 2.x).
Lattices too large for the CPU are given the value of the largest tuned lattice
of the same eps plus a stated safety margin.

usage: python -m oracle.tune_m0 --dims 8,8,8,8 --eps 0.4 --seed 1 --gap 1e-3 --name lattice_8x8x8x8
       python -m oracle.tune_m0 --dims 64,32,32,32 --eps 0.5 --seed 3 --gap 0.06 \
              --derive-from lattice_8x8x8x8_eps0.5 --name lattice_32x32x32x64
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import scipy.sparse.linalg as sla

from oracle.dirac import DiracOperator
from paper_1303_1377_gb300 import synth

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1303_1377_gb300", "workloads.json")


def leftmost(dims, eps, seed, c_sw=1.0, k=4, tol=1e-8, ncv=40):
    U = synth.gauge_field(dims, eps, seed)
    D = DiracOperator(U, dims, 0.0, c_sw)
    n = 12 * D.V
    A = sla.LinearOperator((n, n), matvec=lambda x: D.apply(x.reshape(D.V, 4, 3)).ravel(), dtype=np.complex128)
    t = time.time()
    vals = sla.eigs(A, k=k, which="SR", ncv=max(2 * k + 1, ncv), tol=tol, maxiter=20000, return_eigenvectors=False)
    vals = vals[np.argsort(vals.real)]
    return vals, time.time() - t


def derive(name: str, source: str, gap: float, dims, eps: float, seed: int):
    """A lattice too large for CPU Arnoldi takes m0 = -Re(lambda_L of `source`) + gap, where
    `source` is a tuned lattice of the same eps (the spectral edge of a larger volume of the
    same ensemble lies at or left of the smaller one's, so the gap is an upper bound on the
    smallest |eigenvalue| of the derived workload)."""
    data = json.load(open(OUT))
    lam = data[source]["lambda_L_m0_0"]
    data[name] = {"dims": list(dims), "eps": eps, "seed": seed, "c_sw": 1.0, "m0": -lam[0] + gap, "gap": gap,
                  "derived_from": source, "lambda_L_source": lam}
    json.dump(data, open(OUT, "w"), indent=1)
    print(name, data[name])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", required=True)
    ap.add_argument("--eps", type=float, required=True)
    ap.add_argument("--seed", type=int, required=True)
    ap.add_argument("--derive-from", default=None)
    ap.add_argument("--gap", type=float, default=1e-3)
    ap.add_argument("--name", required=True)
    ap.add_argument("--k", type=int, default=4)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--ncv", type=int, default=40)
    a = ap.parse_args()
    dims = tuple(int(v) for v in a.dims.split(","))
    if a.derive_from:
        return derive(a.name, a.derive_from, a.gap, dims, a.eps, a.seed)
    vals, secs = leftmost(dims, a.eps, a.seed, k=a.k, tol=a.tol, ncv=a.ncv)
    lam = vals[0]
    m0 = -lam.real + a.gap
    rec = {"dims": list(dims), "eps": a.eps, "seed": a.seed, "c_sw": 1.0, "lambda_L_m0_0": [lam.real, lam.imag],
           "gap": a.gap, "m0": m0, "arpack": {"k": a.k, "tol": a.tol, "ncv": a.ncv}, "leftmost_eigenvalues": [[v.real, v.imag] for v in vals], "arpack_seconds": secs}
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data[a.name] = rec
    json.dump(data, open(OUT, "w"), indent=1)
    print(a.name, rec)


if __name__ == "__main__":
    main()
