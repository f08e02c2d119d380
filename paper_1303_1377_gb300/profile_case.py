"""Run each hot kernel of the solve once on a small lattice, for ncu captures.

usage: python -m paper_1303_1377_gb300.profile_case [--dims 24,24,24,24] [--precision half] [--nrhs 12]

It builds D for a synthetic gauge field, an interpolation from seeded random test
vectors, then applies one SAP iteration, three steps of the odd-even coarse GMRES,
one double-word Dslash, one FP32 Dslash, one restriction and one prolongation to
nrhs right-hand sides resident on the GPU.
"""
from __future__ import annotations

import argparse

import torch

from . import ddamg, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", default="24,24,24,24")
    ap.add_argument("--precision", default="half", choices=["single", "half", "double"])
    ap.add_argument("--nrhs", type=int, default=12)
    ap.add_argument("--m0", type=float, default=-0.93)
    a = ap.parse_args()
    dims = tuple(int(v) for v in a.dims.split(","))
    prec = {"single": ddamg.PREC_SINGLE, "half": ddamg.PREC_HALF, "double": ddamg.PREC_DOUBLE}[a.precision]
    U = synth.gauge_field(dims, 0.5, 1)
    s = ddamg.Solver(dims, U, a.m0, 1.0, ddamg.default_params(n_vec=20, precision=prec), setup=False)
    s.setup_from_vectors(synth.random_test_vectors(dims, 20, 2))
    x = torch.from_numpy(synth.gaussian_spinors(dims, a.nrhs, 3)).cuda()
    s.apply_sap(x, 1)
    e = torch.from_numpy(synth.gaussian_coarse(s.n_coarse, s.coarse_dof, a.nrhs, 4)).cuda()
    s.coarse_solve(e, fixed_iters=3)
    if prec != ddamg.PREC_DOUBLE:
        s.apply_D_mixed(x.to(torch.complex64))
        s.apply_D_f32(x.to(torch.complex64))
    s.prolong(s.restrict(x))
    torch.cuda.synchronize()
    s.close()
    print("ok")


if __name__ == "__main__":
    main()
