"""The benchmark workload at full size (32^3 x 64, 12 right-hand sides, half-precision V-cycle,
GPU adaptive setup, default outer scheme), in the launch configuration the benchmark times.

The oracle cannot run the whole lattice, so each check is either evaluated by the oracle at
sampled sites / aggregates, or is a property that holds at any size:
- the solve reaches an FP64 relative residual <= 1e-10 for every right-hand side, measured with
  the FP64 Dslash (itself pinned to the oracle at this size) and with the oracle at sampled sites;
- restriction and prolongation on sampled aggregates equal the oracle's P^H x and P e, with P
  built by the oracle's Gram-Schmidt from the GPU setup's own test vectors (FP16-stored P: 2e-3);
- D_c e equals P^H D P e (FP16-stored D_c and P: 1e-2).
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle.aggregation import modified_gram_schmidt  # noqa: E402
from oracle.dirac import apply_at_sites  # noqa: E402
from oracle.lattice import Blocking, Lattice  # noqa: E402
from paper_1303_1377_gb300 import synth  # noqa: E402

DIMS = (64, 32, 32, 32)
EPS, SEED, CSW, N = 0.5, 3, 1.0, 20
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def relerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def work():
    from paper_1303_1377_gb300 import ddamg

    m0 = json.load(open(os.path.join(ROOT, "paper_1303_1377_gb300", "workloads.json")))["lattice_32x32x32x64"]["m0"]
    U = synth.gauge_field(DIMS, EPS, SEED)
    p = ddamg.default_params(n_vec=N, nu=2, precision=ddamg.PREC_HALF)
    s = ddamg.Solver(DIMS, U, m0, CSW, p)
    yield dict(dd=ddamg, s=s, U=U, m0=m0, lat=Lattice(DIMS), rng=np.random.default_rng(7))
    s.close()


def test_full_size_solve_twelve_point_sources(work):
    s, U, m0 = work["s"], work["U"], work["m0"]
    b = synth.point_sources(DIMS)
    z, st, rc = s.solve(b)
    assert rc == 0
    y = s.apply_D(z)
    for r in range(12):
        res = np.linalg.norm(b[r] - y[r]) / np.linalg.norm(b[r])
        assert res <= 1e-10, (r, res)
        assert st[r]["rel_residual"] <= 1e-10
    # the oracle's D at sampled sites (the source site among them): |b - D z| <= 1e-10 |b| there
    sites = np.concatenate([[0], work["rng"].choice(np.prod(DIMS), 64, replace=False)])
    for r in (0, 5, 11):
        ref = apply_at_sites(U, DIMS, m0, CSW, z[r], sites)
        assert np.max(np.abs(b[r][sites] - ref)) <= 1e-10 * np.linalg.norm(b[r])


def _oracle_basis(work, vecs, blocks):
    """Q[c, h, 6*256, N]: the oracle's local Gram-Schmidt of the test vectors on sampled aggregates."""
    blk = Blocking(work["lat"], (4, 4, 4, 4))
    sites = blk.sites[blocks]  # [nb, 256]
    vb = np.moveaxis(vecs[:, sites], 0, -1)  # [nb, 256, 4, 3, N]
    nb = len(blocks)
    M = np.stack([vb[:, :, 0:2].reshape(nb, 256 * 6, N), vb[:, :, 2:4].reshape(nb, 256 * 6, N)], axis=1)
    return modified_gram_schmidt(M), sites


def test_full_size_transfers_on_sampled_aggregates(work):
    s = work["s"]
    vecs = s.vectors()
    blocks = work["rng"].choice(s.n_coarse, 6, replace=False)
    Q, sites = _oracle_basis(work, vecs, blocks)
    del vecs
    x = synth.gaussian_spinors(DIMS, 12, seed=11)
    e = s.restrict(x)
    for q, c in enumerate(blocks):
        xs = x[:, sites[q]]  # [12, 256, 4, 3]
        for h in range(2):
            xh = xs[:, :, 2 * h:2 * h + 2].reshape(12, 256 * 6)
            ref = xh @ np.conj(Q[q, h])  # [12, N]
            assert relerr(e[:, c, h * N:(h + 1) * N], ref) < 2e-3
    ec = synth.gaussian_coarse(s.n_coarse, s.coarse_dof, 12, seed=12)
    y = s.prolong(ec)
    for q, c in enumerate(blocks):
        for h in range(2):
            ref = (Q[q, h] @ ec[:, c, h * N:(h + 1) * N].T).T.reshape(12, 256, 2, 3)
            assert relerr(y[:, sites[q], 2 * h:2 * h + 2], ref) < 2e-3


def test_full_size_coarse_operator_is_galerkin(work):
    s = work["s"]
    e = synth.gaussian_coarse(s.n_coarse, s.coarse_dof, 12, seed=13)
    lhs = s.apply_Dc(e)
    rhs = s.restrict(s.apply_D(s.prolong(e)))
    assert relerr(lhs, rhs) < 1e-2

