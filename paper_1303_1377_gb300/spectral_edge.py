"""The leftmost eigenvalues of D(0) for a lattice too large for a host eigensolver, with the library's
own solver on the GPU, and the near-critical mass that follows from them.

D(m) = D(0) + m I (the mass enters only the site term (m + 4) I, Sec. 2.2), so the eigenvalues of
D(m_s) closest to zero are those of D(0) at the left edge of the spectrum, shifted by m_s.  With a
shift m_s at which D(m_s) is still comfortably nonsingular, block inverse (shift-invert subspace)
iteration finds them: X <- D(m_s)^{-1} X (one batched solve of k right-hand sides), orthonormalise,
Rayleigh-Ritz with D(m_s) on span X, X <- the Ritz vectors.  It converges to the k eigenvalues of
D(m_s) of smallest modulus at the rate |theta_i / theta_{k+1}|.  With theta_left the converged Ritz
value of smallest real part, the leftmost eigenvalue of D(0) is lambda_L = theta_left - m_s, and the
workload's mass is m0 = -Re lambda_L + gap, which puts the smallest |eigenvalue| of D(m0) at about gap
(at sqrt(gap^2 + Im(lambda_L)^2) when lambda_L is not real).

The mass is an input of the benchmark, not a parity quantity: no oracle test uses a mass written by
this tool.

usage: python -m paper_1303_1377_gb300.spectral_edge --dims 64,32,32,32 --eps 0.5 --seed 3 --shift -0.93 \\
           --gap 1e-3 --name lattice_32x32x32x64_critical [--write]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
WORKLOADS = os.path.join(HERE, "workloads.json")


def _gram(A, B):
    """A^H B for fields [k, ...] (complex128 torch tensors) -> numpy [k, k]."""
    import torch

    k = A.shape[0]
    return torch.matmul(A.reshape(k, -1).conj(), B.reshape(k, -1).transpose(0, 1)).cpu().numpy()


def edge(dims, eps, seed, shift, k=12, iters=20, res_tol=1e-4, solve_tol=1e-8, n_vec=20, precision="half", c_sw=1.0, log=print,
         **params):
    import torch

    from . import ddamg, synth

    prec = {"single": ddamg.PREC_SINGLE, "half": ddamg.PREC_HALF, "double": ddamg.PREC_DOUBLE}[precision]
    t0 = time.perf_counter()
    U = synth.gauge_field(dims, eps, seed)
    s = ddamg.Solver(dims, U, shift, c_sw, ddamg.default_params(n_vec=n_vec, precision=prec, **params), setup=True)
    s.set_stream(torch.cuda.current_stream().cuda_stream)  # the library's work and torch's in one stream order
    del U
    t_setup = time.perf_counter() - t0
    X = torch.from_numpy(synth.gaussian_spinors(dims, k, seed=seed + 500)).cuda()
    hist = []
    theta = None
    for it in range(iters):
        t1 = time.perf_counter()
        Y, st, rc = s.solve_zero_guess(X, tol=solve_tol, allow_fail=True)
        # orthonormalise Y (Cholesky of the Gram matrix, twice for stability)
        for _ in range(2):
            G = _gram(Y, Y)
            L = np.linalg.cholesky(0.5 * (G + G.conj().T))
            Linv = torch.from_numpy(np.linalg.inv(L).conj().T.copy()).cuda()  # Y <- Y L^{-H}
            Y = torch.einsum("k...,kj->j...", Y, Linv)
        DY = s.apply_D(Y)
        H = _gram(Y, DY)  # Rayleigh quotient matrix Y^H D Y
        theta, S = np.linalg.eig(H)
        order = np.argsort(np.abs(theta))
        theta, S = theta[order], S[:, order]
        St = torch.from_numpy(S.copy()).cuda()
        X = torch.einsum("k...,kj->j...", Y, St)
        R = torch.einsum("k...,kj->j...", DY, St) - torch.from_numpy(theta.copy()).cuda().reshape(k, *([1] * (X.ndim - 1))) * X
        res = (torch.linalg.vector_norm(R.reshape(k, -1), dim=1) / torch.linalg.vector_norm(X.reshape(k, -1), dim=1)).cpu().numpy()
        hist.append({"iteration": it, "seconds": time.perf_counter() - t1, "solve_status": int(rc),
                     "fgmres_iterations": max(q["iterations"] for q in st), "ritz": [[float(v.real), float(v.imag)] for v in theta[:4]],
                     "residuals": [float(v) for v in res[:4]]})
        log(json.dumps(hist[-1]))
        # converged once the leftmost Ritz pair's residual (an error bound for the Ritz value up to
        # the eigenvector conditioning) is below res_tol
        if res[int(np.argmin(theta.real))] < res_tol and it >= 3:
            break
    s.close()
    i_left = int(np.argmin(theta.real))
    lam = theta[i_left] - shift
    return {"lambda_L_m0_0": [float(lam.real), float(lam.imag)], "ritz_D_shift": [[float(v.real), float(v.imag)] for v in theta],
            "ritz_residuals": [float(v) for v in res], "shift": shift, "k": k, "iterations": len(hist), "solve_tol": solve_tol,
            "setup_seconds": t_setup, "history": hist}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--record", default=None, help="merge a record written by --out into workloads.json and exit")
    ap.add_argument("--dims", help="L0,L1,L2,L3 (time first)")
    ap.add_argument("--eps", type=float)
    ap.add_argument("--seed", type=int)
    ap.add_argument("--shift", type=float, help="mass m_s of the inverse iteration (D(m_s) must be nonsingular)")
    ap.add_argument("--gap", type=float, default=1e-3)
    ap.add_argument("--k", type=int, default=12)
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--out", default=None, help="also write the record (with its history) to this JSON file")
    ap.add_argument("--n-vec", type=int, default=20)
    ap.add_argument("--n-kv", type=int, default=25, help="FGMRES restart length of the solves")
    ap.add_argument("--lean", type=int, default=0, help="free the FP64 test vectors after the setup (large lattices)")
    ap.add_argument("--setup-group", type=int, default=0, help="test vectors per setup batch (0: all)")
    ap.add_argument("--name")
    ap.add_argument("--write", action="store_true", help="record the result in workloads.json")
    a = ap.parse_args()
    if a.record:
        data = json.load(open(WORKLOADS))
        data.update(json.load(open(a.record)))
        with open(WORKLOADS, "w") as f:
            json.dump(data, f, indent=1)
            f.write("\n")
        return
    dims = tuple(int(v) for v in a.dims.split(","))
    r = edge(dims, a.eps, a.seed, a.shift, k=a.k, iters=a.iters, n_vec=a.n_vec, n_kv=a.n_kv, lean=a.lean, setup_group=a.setup_group)
    rec = {"dims": list(dims), "eps": a.eps, "seed": a.seed, "c_sw": 1.0, "m0": -r["lambda_L_m0_0"][0] + a.gap, "gap": a.gap,
           "source": "GPU shift-invert subspace iteration (paper_1303_1377_gb300/spectral_edge.py)", **r}
    print(json.dumps({k: v for k, v in rec.items() if k != "history"}))
    if a.out:
        with open(a.out, "w") as f:
            json.dump({a.name: rec}, f, indent=1)
    if a.write:
        data = json.load(open(WORKLOADS))
        data[a.name] = rec
        with open(WORKLOADS, "w") as f:
            json.dump(data, f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main()
