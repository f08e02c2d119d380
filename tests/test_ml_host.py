"""The CUDA library's level-1 operations for the recursion to a third level (ml_geom.h, ml_ops.cuh),
run on the host through their loop executor, against the oracle's multilevel classes.

The same functors and orchestration run on the GPU through a grid-stride kernel; this checks their
index arithmetic and algebra without a GPU.  The harness is built with nvcc as host code."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.aggregation import Aggregation
from oracle.coarse import CoarseOperator
from oracle.dirac import DiracOperator
from oracle.lattice import Blocking, Lattice
from oracle.multilevel import StencilAggregation, StencilCoarse, StencilOperator, StencilSAP
from paper_1303_1377_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1303_1377_gb300", "csrc")

# (fine dims, level-0 aggregate, N0, level-1 block, N1)
CASES = {
    "8^4 -> 4^4 (2^4 blocks)": ((8, 8, 8, 8), (2, 2, 2, 2), 3, (2, 2, 2, 2), 3),
    "4^4 -> 2x2x2x4 (1x1x1x2 blocks)": ((4, 4, 4, 4), (2, 2, 2, 1), 2, (1, 1, 1, 2), 2),
}

P_D = ctypes.POINTER(ctypes.c_double)
P_I = ctypes.POINTER(ctypes.c_int)


def dp(a):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(P_D)


def ip(a):
    return np.ascontiguousarray(a, dtype=np.int32).ctypes.data_as(P_I)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("mlh") / "libmlh.so"
    subprocess.run([nvcc, "-x", "cu", "-shared", "-Xcompiler", "-fPIC", "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-I", CSRC,
                    "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "ml_host", "ml_harness.cu"), "-o", str(out)],
                   check=True)
    return ctypes.CDLL(str(out))


class Level1:
    """Level 1 of the oracle (D_1 = P_0^H D P_0) and the harness's internal orders."""

    def __init__(self, lib, name):
        dims, agg0, N0, b1, N1 = CASES[name]
        D = DiracOperator(synth.gauge_field(dims, 0.4, seed=91), dims, 0.1, 1.0)
        Dc = CoarseOperator(D, Aggregation(D.lat, agg0, synth.random_test_vectors(dims, N0, seed=92)))
        self.A = StencilOperator(Dc.clat, Dc.B)
        self.L1 = np.array(Dc.clat.dims, dtype=np.int32)
        self.b1 = np.array(b1, dtype=np.int32)
        self.nc, self.N1, self.lib = self.A.n, N1, lib
        sz = np.zeros(4, dtype=np.int32)
        assert lib.mlh_geom_sizes(ip(self.L1), ip(self.b1), ip(sz)) == 0
        self.NB, self.NB2, self.Vb1, self.Vb1e = (int(s) for s in sz)
        g = {k: np.zeros(n, dtype=np.int32) for k, n in (("lex1", self.NB), ("nbr1", 8 * self.NB), ("sites", self.NB2 * self.Vb1),
                                                         ("blk_of", self.NB), ("loc_of", self.NB), ("nbr2", 8 * self.NB2),
                                                         ("lex2", self.NB2))}
        same = np.zeros(8 * self.NB, dtype=np.uint8)
        assert lib.mlh_geom_fill(ip(self.L1), ip(self.b1), *(g[k].ctypes.data_as(P_I) for k in ("lex1", "nbr1", "sites", "blk_of", "loc_of")),
                                 same.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), g["nbr2"].ctypes.data_as(P_I),
                                 g["lex2"].ctypes.data_as(P_I)) == 0
        self.g, self.same = g, same.reshape(8, self.NB)
        lex1 = g["lex1"]
        # column-major blocks in internal order; inverses of the even self blocks
        self.B1 = np.ascontiguousarray(self.A.B[lex1].transpose(0, 1, 3, 2))
        self.Dinv1 = np.ascontiguousarray(np.linalg.inv(self.A.B[lex1[: self.NB // 2], 0]).transpose(0, 2, 1))

    def to_int(self, x):  # [nrhs, NB, nc] lexicographic -> internal
        return np.ascontiguousarray(x[:, self.g["lex1"]])

    def to_lex(self, x):
        out = np.empty_like(x)
        out[:, self.g["lex1"]] = x
        return out


@pytest.fixture(scope="module", params=list(CASES))
def lv(request, lib):
    return Level1(lib, request.param)


def test_blocking_matches_the_oracle(lv):
    """Internal order (even sites first), neighbours, blocks, in-block flags and the level-2 lattice
    agree with the oracle's lattice and blocking."""
    lat = Lattice(tuple(lv.L1))
    lex1, lex2 = lv.g["lex1"], lv.g["lex2"]
    assert sorted(lex1) == list(range(lv.NB))
    assert np.all(lat.parity[lex1[: lv.NB // 2]] == 0) and np.all(lat.parity[lex1[lv.NB // 2:]] == 1)
    int1 = np.empty(lv.NB, dtype=np.int64)
    int1[lex1] = np.arange(lv.NB)
    blk = Blocking(lat, tuple(lv.b1))
    nbr1 = lv.g["nbr1"].reshape(8, lv.NB)
    for d in range(8):
        mu, s = d >> 1, (-1 if d & 1 else 1)
        assert np.array_equal(nbr1[d], int1[lat.neighbour(mu, s)[lex1]])
        assert np.array_equal(lv.same[d].astype(bool), blk.same_block(mu, s)[lex1])
    sites = lv.g["sites"].reshape(lv.NB2, lv.Vb1)
    assert lv.Vb1e == lv.Vb1 // 2
    for c2 in range(lv.NB2):
        assert set(lex1[sites[c2]]) == set(blk.sites[lex2[c2]])
        assert np.all(sites[c2, : lv.Vb1e] < lv.NB // 2) and np.all(sites[c2, lv.Vb1e:] >= lv.NB // 2)
        assert np.all(lv.g["blk_of"][sites[c2]] == c2) and np.array_equal(lv.g["loc_of"][sites[c2]], np.arange(lv.Vb1))
    lat2 = Lattice(blk.nb_dims)
    assert np.all(lat2.parity[lex2[: lv.NB2 // 2]] == 0) and np.all(lat2.parity[lex2[lv.NB2 // 2:]] == 1)
    int2 = np.empty(lv.NB2, dtype=np.int64)
    int2[lex2] = np.arange(lv.NB2)
    nbr2 = lv.g["nbr2"].reshape(8, lv.NB2)
    for d in range(8):
        assert np.array_equal(nbr2[d], int2[lat2.neighbour(d >> 1, -1 if d & 1 else 1)[lex2]])


def test_operator_apply(lv):
    x = synth.gaussian_coarse(lv.NB, lv.nc, 2, seed=93)
    y = np.zeros_like(x)
    assert lv.lib.mlh_apply(ip(lv.L1), ip(lv.b1), lv.nc, dp(lv.B1), dp(lv.to_int(x)), dp(y), 2) == 0
    ref = np.stack([lv.A.apply(x[r]) for r in range(2)])
    assert np.max(np.abs(lv.to_lex(y) - ref)) < 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("nu", [1, 2])
def test_sap_matches_the_oracle(lv, nu):
    """nu red-black SAP iterations with MR(4) block solves, from zero and from a nonzero start."""
    b = synth.gaussian_coarse(lv.NB, lv.nc, 3, seed=94)
    sap = StencilSAP(lv.A, tuple(lv.b1), mr_steps=4)
    for z0 in (np.zeros_like(b), synth.gaussian_coarse(lv.NB, lv.nc, 3, seed=95)):
        ref = []
        for r in range(3):
            z = z0[r].copy()
            for _ in range(nu):
                z = sap.iterate(z, b[r])
            ref.append(z)
        ref = np.stack(ref)
        z = lv.to_int(z0)
        assert lv.lib.mlh_sap(ip(lv.L1), ip(lv.b1), lv.nc, dp(lv.B1), dp(lv.Dinv1), dp(lv.to_int(b)), dp(z), 3, nu, 4) == 0
        assert np.max(np.abs(lv.to_lex(z) - ref)) < 1e-12 * np.max(np.abs(ref))


def test_gram_schmidt_and_transfers_match_the_oracle(lv):
    """P_1 from the harness's ordered Gram-Schmidt restricts and prolongs like the oracle's
    aggregation of the same level-1 test vectors."""
    vec = synth.gaussian_coarse(lv.NB, lv.nc, lv.N1, seed=96)  # [N1, NB, nc]
    P = np.zeros((lv.NB2, 2, lv.Vb1 * lv.nc // 2, lv.N1), dtype=np.complex128)
    assert lv.lib.mlh_gram_schmidt(ip(lv.L1), ip(lv.b1), lv.nc, lv.N1, dp(lv.to_int(vec)), dp(P)) == 0
    agg = StencilAggregation(Lattice(tuple(lv.L1)), tuple(lv.b1), vec)
    x = synth.gaussian_coarse(lv.NB, lv.nc, 2, seed=97)
    e = np.zeros((2, lv.NB2, 2 * lv.N1), dtype=np.complex128)
    assert lv.lib.mlh_restrict(ip(lv.L1), ip(lv.b1), lv.nc, lv.N1, dp(P), dp(lv.to_int(x)), dp(e), 2) == 0
    lex2 = lv.g["lex2"]
    ref = np.stack([agg.restrict(x[r]) for r in range(2)])[:, lex2]
    assert np.max(np.abs(e - ref)) < 1e-12 * np.max(np.abs(ref))
    ec = synth.gaussian_coarse(lv.NB2, 2 * lv.N1, 2, seed=98)  # internal level-2 order
    y = np.zeros((2, lv.NB, lv.nc), dtype=np.complex128)
    assert lv.lib.mlh_prolong(ip(lv.L1), ip(lv.b1), lv.nc, lv.N1, dp(P), dp(ec), dp(y), 2) == 0
    ec_lex = np.empty_like(ec)
    ec_lex[:, lex2] = ec
    ref = np.stack([agg.prolong(ec_lex[r]) for r in range(2)])
    assert np.max(np.abs(lv.to_lex(y) - ref)) < 1e-12 * np.max(np.abs(ref))


def test_galerkin_stencil_matches_the_oracle(lv):
    """D_2 = P_1^H D_1 P_1 assembled by the harness equals the oracle's stencil, block by block."""
    vec = synth.gaussian_coarse(lv.NB, lv.nc, lv.N1, seed=99)
    P = np.zeros((lv.NB2, 2, lv.Vb1 * lv.nc // 2, lv.N1), dtype=np.complex128)
    assert lv.lib.mlh_gram_schmidt(ip(lv.L1), ip(lv.b1), lv.nc, lv.N1, dp(lv.to_int(vec)), dp(P)) == 0
    nc2 = 2 * lv.N1
    B2 = np.zeros((lv.NB2, 9, nc2, nc2), dtype=np.complex128)
    assert lv.lib.mlh_galerkin(ip(lv.L1), ip(lv.b1), lv.nc, lv.N1, dp(lv.B1), dp(P), dp(B2)) == 0
    ref = StencilCoarse(lv.A, StencilAggregation(Lattice(tuple(lv.L1)), tuple(lv.b1), vec)).B
    ref_int = ref[lv.g["lex2"]].transpose(0, 1, 3, 2)
    assert np.max(np.abs(B2 - ref_int)) < 1e-12 * np.max(np.abs(ref))


def test_rank_deficient_level1_vectors_are_reported(lv):
    vec = synth.gaussian_coarse(lv.NB, lv.nc, lv.N1, seed=100)
    vec[-1] = vec[0]
    P = np.zeros((lv.NB2, 2, lv.Vb1 * lv.nc // 2, lv.N1), dtype=np.complex128)
    assert lv.lib.mlh_gram_schmidt(ip(lv.L1), ip(lv.b1), lv.nc, lv.N1, dp(lv.to_int(vec)), dp(P)) == -8


def test_invalid_level1_blockings_are_refused(lib):
    sz = np.zeros(4, dtype=np.int32)
    for L1, b1 in (((4, 4, 4, 4), (4, 2, 2, 2)),   # one block in a direction (odd count)
                   ((4, 4, 4, 4), (3, 2, 2, 2)),   # does not divide
                   ((2, 2, 2, 2), (1, 1, 1, 1))):  # every block extent odd
        assert lib.mlh_geom_sizes(ip(np.array(L1)), ip(np.array(b1)), ip(sz)) == -1


def _level1_oracle(lv, vec=None, **kw):
    from oracle.mg import Params
    from oracle.multilevel import StencilTwoLevel

    p = Params(N=lv.N1, agg_block=tuple(lv.b1), sap_block=tuple(lv.b1), nu=2, coarse_tol=1e-14, coarse_maxiter=5000, **kw)
    return StencilTwoLevel(lv.A, p, vectors=vec)


def _dense_inverse_internal(lv, Dc):
    """Inverse of the oracle's D_2 as a dense matrix in the harness's internal level-2 order."""
    nc2 = 2 * lv.N1
    perm = (lv.g["lex2"][:, None] * nc2 + np.arange(nc2)[None, :]).ravel()
    return np.ascontiguousarray(np.linalg.inv(Dc.dense())[np.ix_(perm, perm)])


def test_level1_vcycle_matches_the_oracle(lv):
    """x = P_1 D_2^{-1} P_1^H r, then two SAP iterations on D_1 x = r (exact level-2 solve on both sides)."""
    vec = synth.gaussian_coarse(lv.NB, lv.nc, lv.N1, seed=101)
    P = np.zeros((lv.NB2, 2, lv.Vb1 * lv.nc // 2, lv.N1), dtype=np.complex128)
    assert lv.lib.mlh_gram_schmidt(ip(lv.L1), ip(lv.b1), lv.nc, lv.N1, dp(lv.to_int(vec)), dp(P)) == 0
    tl = _level1_oracle(lv, vec)
    inv = _dense_inverse_internal(lv, tl.Dc)
    r = synth.gaussian_coarse(lv.NB, lv.nc, 2, seed=102)
    x = np.zeros_like(r)
    assert lv.lib.mlh_vcycle1(ip(lv.L1), ip(lv.b1), lv.nc, lv.N1, dp(lv.B1), dp(lv.Dinv1), dp(P), dp(inv), dp(lv.to_int(r)), dp(x), 2, 2,
                              4) == 0
    ref = np.stack([tl.vcycle(r[q]) for q in range(2)])
    assert np.max(np.abs(lv.to_lex(x) - ref)) < 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("update", ["ddalpha", "idsetup"])
def test_level1_setup_matches_the_oracle(lv, update):
    """Algorithm 1 phase 1 and one round of Algorithm 2 (or of Algorithm 1's update) on D_1, all level-1
    vectors as one batch, then the final rebuild: the vectors and D_2 equal the oracle's."""
    vec0 = synth.gaussian_coarse(lv.NB, lv.nc, lv.N1, seed=103)
    tl = _level1_oracle(lv, n_inv=1, setup_update=update)
    ref = tl.setup(vec0)
    vec = lv.to_int(vec0)
    nc2 = 2 * lv.N1
    P = np.zeros((lv.NB2, 2, lv.Vb1 * lv.nc // 2, lv.N1), dtype=np.complex128)
    B2 = np.zeros((lv.NB2, 9, nc2, nc2), dtype=np.complex128)
    assert lv.lib.mlh_setup1(ip(lv.L1), ip(lv.b1), lv.nc, lv.N1, dp(lv.B1), dp(lv.Dinv1), dp(vec), 1, int(update == "idsetup"), 2, 4, dp(P),
                             dp(B2)) == 0
    assert np.max(np.abs(lv.to_lex(vec) - ref)) < 1e-9 * np.max(np.abs(ref))
    Bref = tl.Dc.B[lv.g["lex2"]].transpose(0, 1, 3, 2)
    assert np.max(np.abs(B2 - Bref)) < 1e-9 * np.max(np.abs(Bref))


def test_sap_in_fp32_stays_at_single_precision(lv):
    """The FP32 instantiation (SINGLE and HALF handles): two SAP iterations agree with the FP64
    oracle to the FP32 level of iterated MR steps (2e-5 relative to the field maximum)."""
    b = synth.gaussian_coarse(lv.NB, lv.nc, 2, seed=104)
    sap = StencilSAP(lv.A, tuple(lv.b1), mr_steps=4)
    ref = np.stack([sap.apply(b[r], 2) for r in range(2)])
    z = np.zeros((2, lv.NB, lv.nc), dtype=np.complex128)
    assert lv.lib.mlh_sap_f32(ip(lv.L1), ip(lv.b1), lv.nc, dp(lv.B1), dp(lv.Dinv1), dp(lv.to_int(b)), dp(z), 2, 2, 4) == 0
    err = np.max(np.abs(lv.to_lex(z) - ref)) / np.max(np.abs(ref))
    assert 1e-9 < err < 2e-5  # FP32 rounding is visible, and small


@pytest.mark.parametrize("L1,b1", [((4, 2, 6, 4), (2, 1, 3, 2)), ((2, 4, 4, 8), (1, 2, 1, 2)), ((6, 6, 2, 4), (3, 3, 1, 2)),
                                   ((4, 4, 4, 4), (2, 2, 2, 2)), ((8, 4, 2, 2), (4, 2, 1, 1))])
def test_blocking_of_asymmetric_lattices(lib, L1, b1):
    """Internal order, neighbours, in-block flags, block membership (even sites first) and the next
    level's order and neighbours against the oracle's lattice and blocking, for lattices and blocks of
    unequal and odd extents."""
    L1a, b1a = np.array(L1, dtype=np.int32), np.array(b1, dtype=np.int32)
    sz = np.zeros(4, dtype=np.int32)
    assert lib.mlh_geom_sizes(ip(L1a), ip(b1a), ip(sz)) == 0
    NB, NB2, Vb1, Vb1e = (int(v) for v in sz)
    g = {k: np.zeros(n, dtype=np.int32) for k, n in (("lex1", NB), ("nbr1", 8 * NB), ("sites", NB2 * Vb1), ("blk_of", NB),
                                                     ("loc_of", NB), ("nbr2", 8 * NB2), ("lex2", NB2))}
    same = np.zeros(8 * NB, dtype=np.uint8)
    assert lib.mlh_geom_fill(ip(L1a), ip(b1a), *(g[k].ctypes.data_as(P_I) for k in ("lex1", "nbr1", "sites", "blk_of", "loc_of")),
                             same.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), g["nbr2"].ctypes.data_as(P_I),
                             g["lex2"].ctypes.data_as(P_I)) == 0
    lat, blk = Lattice(L1), Blocking(Lattice(L1), b1)
    lex1, lex2 = g["lex1"], g["lex2"]
    assert NB == lat.V and NB2 == blk.nblocks and Vb1 == blk.bvol and Vb1e == Vb1 // 2
    assert np.all(lat.parity[lex1[: NB // 2]] == 0) and np.all(lat.parity[lex1[NB // 2:]] == 1)
    int1 = np.empty(NB, dtype=np.int64)
    int1[lex1] = np.arange(NB)
    for d in range(8):
        mu, s = d >> 1, (-1 if d & 1 else 1)
        assert np.array_equal(g["nbr1"].reshape(8, NB)[d], int1[lat.neighbour(mu, s)[lex1]])
        assert np.array_equal(same.reshape(8, NB)[d].astype(bool), blk.same_block(mu, s)[lex1])
    sites = g["sites"].reshape(NB2, Vb1)
    for c2 in range(NB2):
        assert set(lex1[sites[c2]]) == set(blk.sites[lex2[c2]])
        assert np.all(lat.parity[lex1[sites[c2, :Vb1e]]] == 0) and np.all(lat.parity[lex1[sites[c2, Vb1e:]]] == 1)
    lat2 = Lattice(blk.nb_dims)
    int2 = np.empty(NB2, dtype=np.int64)
    int2[lex2] = np.arange(NB2)
    assert np.all(lat2.parity[lex2[: NB2 // 2]] == 0)
    for d in range(8):
        assert np.array_equal(g["nbr2"].reshape(8, NB2)[d], int2[lat2.neighbour(d >> 1, -1 if d & 1 else 1)[lex2]])


def test_level1_vcycle_in_fp32(lv):
    """The FP32 level-1 V-cycle of SINGLE and HALF handles (restriction, level-2 solve, prolongation,
    two SAP iterations, all in FP32) against the FP64 oracle: within 1e-4 relative to the field
    maximum, and visibly rounded."""
    vec = synth.gaussian_coarse(lv.NB, lv.nc, lv.N1, seed=105)
    P = np.zeros((lv.NB2, 2, lv.Vb1 * lv.nc // 2, lv.N1), dtype=np.complex128)
    assert lv.lib.mlh_gram_schmidt(ip(lv.L1), ip(lv.b1), lv.nc, lv.N1, dp(lv.to_int(vec)), dp(P)) == 0
    tl = _level1_oracle(lv, vec)
    inv = _dense_inverse_internal(lv, tl.Dc)
    r = synth.gaussian_coarse(lv.NB, lv.nc, 2, seed=106)
    x = np.zeros_like(r)
    assert lv.lib.mlh_vcycle1_f32(ip(lv.L1), ip(lv.b1), lv.nc, lv.N1, dp(lv.B1), dp(lv.Dinv1), dp(P), dp(inv), dp(lv.to_int(r)), dp(x), 2,
                                  2, 4) == 0
    ref = np.stack([tl.vcycle(r[q]) for q in range(2)])
    err = np.max(np.abs(lv.to_lex(x) - ref)) / np.max(np.abs(ref))
    assert 1e-9 < err < 1e-4
