"""The three-level path of the CUDA library (ddamg_ml_*) against the oracle's multilevel recursion.

The level-1 functors it drives are also checked on the host in tests/test_ml_host.py.

Case: 8^4 fine lattice, 2^4 blocks, N = 4 -> level 1 = 4^4 coarse sites of 8 components; level-1
blocks 2^4, N_1 = 3 -> level 2 = 2^4 sites of 6 components.  DOUBLE precision throughout, so the
stated tolerances are rounding-level: 1e-13 for FP64 results (single applications, V-cycles whose
coarse solves run to 1e-14, the level-1 setup), 1e-6 for FP32 applications."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle.dirac import DiracOperator  # noqa: E402
from oracle.mg import Params as OParams  # noqa: E402
from oracle.multilevel import MultiLevel  # noqa: E402
from paper_1303_1377_gb300 import synth  # noqa: E402

DIMS, BLK, N0, BLK1, N1 = (8, 8, 8, 8), (2, 2, 2, 2), 4, (2, 2, 2, 2), 3
M0, CSW = 0.05, 1.0


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def case():
    from paper_1303_1377_gb300 import ddamg

    U = synth.gauge_field(DIMS, 0.5, seed=111)
    D = DiracOperator(U, DIMS, M0, CSW)
    v0 = synth.random_test_vectors(DIMS, N0, seed=112)
    v1 = synth.gaussian_coarse(4 ** 4, 2 * N0, N1, seed=113)  # level-1 vectors, lexicographic coarse sites

    def oracle(inner="fgmres", coarse_tol=1e-14, inner_tol=5e-2):
        ml = MultiLevel(D, [OParams(N=N0, agg_block=BLK, sap_block=BLK, nu=2, coarse_tol=coarse_tol, coarse_maxiter=5000),
                            OParams(N=N1, agg_block=BLK1, sap_block=BLK1, nu=2, coarse_tol=coarse_tol, coarse_maxiter=5000)],
                        inner=inner, inner_tol=inner_tol)
        ml.build([v0, v1])
        return ml

    def handle(coarse_tol=1e-14):
        p = ddamg.default_params(n_vec=N0, block=BLK, precision=ddamg.PREC_DOUBLE, nu=2, coarse_tol=coarse_tol)
        s = ddamg.Solver(DIMS, U, M0, CSW, p, setup=False)
        s.setup_from_vectors(v0)
        return s

    def gpu(inner=0, coarse_tol=1e-14, inner_tol=5e-2):
        s = handle(coarse_tol)
        s.ml_build(v1, ddamg.ml_default_params(block1=BLK1, n_vec1=N1, nu1=2, inner=inner, coarse_tol=coarse_tol, inner_tol=inner_tol,
                                               coarse_maxiter=5000))
        return s

    return dict(D=D, oracle=oracle, gpu=gpu, handle=handle, ddamg=ddamg)


def test_level1_pieces(case):
    """Level-1 restriction and prolongation, D_2, and level-1 SAP (nu = 2, MR(4))."""
    ml = case["oracle"]()
    l1 = ml.levels[1]
    with case["gpu"]() as s:
        x = synth.gaussian_coarse(4 ** 4, 2 * N0, 2, seed=114)
        assert rel(s.ml_restrict1(x), np.stack([l1.agg.restrict(x[r]) for r in range(2)])) < 1e-13
        e = synth.gaussian_coarse(2 ** 4, 2 * N1, 2, seed=115)
        assert rel(s.ml_prolong1(e), np.stack([l1.agg.prolong(e[r]) for r in range(2)])) < 1e-13
        assert rel(s.ml_apply_D2(e), np.stack([l1.Dc.apply(e[r]) for r in range(2)])) < 1e-13
        assert rel(s.ml_apply_sap1(x, 2), np.stack([l1.sap.apply(x[r], 2) for r in range(2)])) < 1e-13


def test_level1_vcycle(case):
    ml = case["oracle"]()
    x = synth.gaussian_coarse(4 ** 4, 2 * N0, 2, seed=116)
    with case["gpu"]() as s:
        assert rel(s.ml_vcycle1(x), np.stack([ml.levels[1].vcycle(x[r]) for r in range(2)])) < 1e-13


@pytest.mark.parametrize("inner", ["fgmres", "vcycle"])
def test_fine_vcycle_with_recursive_coarse_solve(case, inner):
    """The fine V-cycle whose coarse solve is 3 FGMRES steps on D_1 with the level-1 V-cycle (or one
    level-1 V-cycle)."""
    ml = case["oracle"](inner=inner)
    r = synth.gaussian_spinors(DIMS, 2, seed=117)
    ref = np.stack([ml.levels[0].vcycle(r[q], coarse_fixed_iters=3) for q in range(2)])
    with case["gpu"](inner=0 if inner == "fgmres" else 1) as s:
        assert rel(s.ml_vcycle(r, 3), ref) < 1e-13


def test_three_level_solve(case):
    """Default inner solves (5e-2): true residual <= 1e-10 under the oracle's D, the oracle's solution
    to 1e-8, and the counters show the recursion ran."""
    D = case["D"]
    b = synth.gaussian_spinors(DIMS, 2, seed=118)
    ml = case["oracle"](coarse_tol=5e-2)
    with case["gpu"](coarse_tol=5e-2) as s:
        z, st, rc = s.ml_solve(b)
        counts = s.ml_counts()
    assert rc == 0
    for q in range(2):
        assert np.linalg.norm(b[q] - D.apply(z[q])) <= 1e-10 * np.linalg.norm(b[q])
        zo, _ = ml.solve(b[q])
        assert np.linalg.norm(z[q] - zo) <= 1e-8 * np.linalg.norm(zo)
    assert counts["fgmres_steps_D1"] > 0 and counts["gmres_steps_D2"] > 0 and counts["vcycles1"] > 0


def test_stale_third_level_and_argument_checks(case):
    """A mass change makes the third level stale (NOT_READY until it is built again); level-1 blocks
    that do not divide the level-1 lattice and too many level-1 vectors are refused."""
    ddamg = case["ddamg"]
    with case["gpu"]() as s:
        s.set_mass(M0 + 0.01)
        with pytest.raises(ddamg.DDAMGError) as e:
            s.ml_vcycle1(synth.gaussian_coarse(4 ** 4, 2 * N0, 1, seed=119))
        assert e.value.status == -7
    with case["handle"]() as s:
        v1 = synth.gaussian_coarse(4 ** 4, 2 * N0, N1, seed=113)
        for kw in ({"block1": (3, 2, 2, 2), "n_vec1": N1}, {"block1": BLK1, "n_vec1": 2 ** 4 * N0 + 1}):
            with pytest.raises(ddamg.DDAMGError) as e:
                s.ml_build(v1, ddamg.ml_default_params(**kw))
            assert e.value.status == -1
        assert s.ml_levels() == 2


@pytest.mark.parametrize("update", ["ddalpha", "idsetup"])
def test_level1_setup(case, update):
    """ddamg_ml_setup: Algorithm 1 phase 1 and one round of Algorithm 2 (or Algorithm 1's update) on D_1
    with exact level-2 solves on both sides: the final level-1 vectors and D_2 equal the oracle's."""
    from oracle.multilevel import StencilTwoLevel

    ddamg = case["ddamg"]
    A1 = case["oracle"]().levels[1].D
    v10 = synth.gaussian_coarse(4 ** 4, 2 * N0, N1, seed=120)
    tl = StencilTwoLevel(A1, OParams(N=N1, agg_block=BLK1, sap_block=BLK1, nu=2, n_inv=1, coarse_tol=1e-14, coarse_maxiter=5000,
                                     setup_update=update))
    ref = tl.setup(v10)
    with case["handle"]() as s:
        out = s.ml_setup(v10, ddamg.ml_default_params(block1=BLK1, n_vec1=N1, nu1=2, coarse_tol=1e-14, coarse_maxiter=5000, n_inv1=1,
                                                      setup_update1=ddamg.SETUP_IDSETUP if update == "idsetup" else ddamg.SETUP_DDALPHA))
        assert rel(out, ref) < 1e-13
        e = synth.gaussian_coarse(2 ** 4, 2 * N1, 2, seed=121)
        assert rel(s.ml_apply_D2(e), np.stack([tl.Dc.apply(e[r]) for r in range(2)])) < 1e-13


@pytest.mark.parametrize("prec", ["SINGLE", "HALF"])
def test_three_level_solve_mixed_precision(case, prec):
    """SINGLE and HALF handles: level-1 and level-2 solves in FP32 inside the handle's outer scheme;
    the true FP64 residual still reaches 1e-10 and the recursion runs.  The level-1 SAP reads D_1 in
    FP32 on SINGLE handles (stated 1e-6) and in FP16 on HALF handles (stated 2e-3 relative to the
    field maximum, the bound of the fine smoother with its FP16 operator)."""
    ddamg, D = case["ddamg"], case["D"]
    U = synth.gauge_field(DIMS, 0.5, seed=111)
    p = ddamg.default_params(n_vec=N0, block=BLK, precision=getattr(ddamg, "PREC_" + prec), nu=2)
    b = synth.gaussian_spinors(DIMS, 2, seed=122)
    with ddamg.Solver(DIMS, U, M0, CSW, p, setup=False) as s:
        s.setup_from_vectors(synth.random_test_vectors(DIMS, N0, seed=112))
        s.ml_build(synth.gaussian_coarse(4 ** 4, 2 * N0, N1, seed=113), ddamg.ml_default_params(block1=BLK1, n_vec1=N1, nu1=2))
        x = synth.gaussian_coarse(4 ** 4, 2 * N0, 2, seed=123)
        ref = case["oracle"]().levels[1].sap
        assert rel(s.ml_apply_sap1(x, 2), np.stack([ref.apply(x[r], 2) for r in range(2)])) < {"SINGLE": 1e-6, "HALF": 2e-3}[prec]
        z, st, rc = s.ml_solve(b)
        counts = s.ml_counts()
    assert rc == 0
    for q in range(2):
        assert np.linalg.norm(b[q] - D.apply(z[q])) <= 1e-10 * np.linalg.norm(b[q])
    assert counts["fgmres_steps_D1"] > 0 and counts["gmres_steps_D2"] > 0


def test_four_levels():
    """16^4 fine lattice, 2^4 blocks on every level, N = N_1 = N_2 = 2: levels 8^4, 4^4 and 2^4.  The
    GPU hierarchy built from the oracle's vectors solves to a true residual of 1e-10 and agrees
    with the oracle's four-level solve."""
    from paper_1303_1377_gb300 import ddamg

    dims = (16, 16, 16, 16)
    U = synth.gauge_field(dims, 0.5, seed=131)
    D = DiracOperator(U, dims, M0, CSW)
    v0 = synth.random_test_vectors(dims, 2, seed=132)
    v1 = synth.gaussian_coarse(8 ** 4, 4, 2, seed=133)
    v2 = synth.gaussian_coarse(4 ** 4, 4, 2, seed=134)
    ps = [OParams(N=2, agg_block=BLK, sap_block=BLK, nu=2) for _ in range(3)]
    ml = MultiLevel(D, ps)
    ml.build([v0, v1, v2])
    b = synth.gaussian_spinors(dims, 1, seed=135)
    zo, _ = ml.solve(b[0])
    p = ddamg.default_params(n_vec=2, block=BLK, precision=ddamg.PREC_DOUBLE, nu=2)
    with ddamg.Solver(dims, U, M0, CSW, p, setup=False) as s:
        s.setup_from_vectors(v0)
        mp = ddamg.ml_default_params(block1=BLK, n_vec1=2, nu1=2)
        s.ml_build(v1, mp)
        s.ml_add_level(v2, mp, setup=False)
        assert s.ml_levels() == 4
        z, st, rc = s.ml_solve(b)
    assert rc == 0
    assert np.linalg.norm(b[0] - D.apply(z[0])) <= 1e-10 * np.linalg.norm(b[0])
    assert np.linalg.norm(z[0] - zo) <= 1e-8 * np.linalg.norm(zo)


@pytest.mark.parametrize("prec,tol", [("SINGLE", 1e-6), ("HALF", 4e-3)])
def test_coarsest_operator_at_benchmark_shape(prec, tol):
    """D_2 with 2 N_1 = 40 components per site and 12 right-hand sides, the shape of the benchmark's
    coarsest level: a SINGLE handle applies it in FP32, a HALF handle through the FP16 tensor-core
    stencil that its odd-even GMRES uses (one FP16 rounding per stored entry; stated tolerance 4e-3
    relative to the field maximum, as for the level-1 stencil).  A three-level solve on the HALF
    handle still reaches a true residual of 1e-10 under the oracle's D.  The HALF product is also
    compared with the oracle's D_2 whose entries are rounded as the kernel stores them (FP64 -> FP32 ->
    FP16, real and imaginary parts): the right-hand sides enter as FP16 hi + lo pairs, so that product
    must hold to FP32 accumulation (stated 5e-6 relative to the field maximum for 360 terms per row)."""
    from oracle.multilevel import StencilOperator
    from paper_1303_1377_gb300 import ddamg

    blk, n0, n1, nr = (2, 2, 2, 2), 20, 20, 12
    U = synth.gauge_field(DIMS, 0.5, seed=141)
    D = DiracOperator(U, DIMS, M0, CSW)
    v0 = synth.random_test_vectors(DIMS, n0, seed=142)
    v1 = synth.gaussian_coarse(4 ** 4, 2 * n0, n1, seed=143)
    ml = MultiLevel(D, [OParams(N=n0, agg_block=blk, sap_block=blk, nu=2), OParams(N=n1, agg_block=blk, sap_block=blk, nu=2)])
    ml.build([v0, v1])
    e = synth.gaussian_coarse(2 ** 4, 2 * n1, nr, seed=144)
    ref = np.stack([ml.levels[1].Dc.apply(e[r]) for r in range(nr)])
    p = ddamg.default_params(n_vec=n0, block=blk, precision=getattr(ddamg, "PREC_" + prec), nu=2)
    b = synth.gaussian_spinors(DIMS, 4, seed=145)
    with ddamg.Solver(DIMS, U, M0, CSW, p, setup=False) as s:
        s.setup_from_vectors(v0)
        s.ml_build(v1, ddamg.ml_default_params(block1=blk, n_vec1=n1, nu1=2))
        assert rel(s.ml_apply_D2(e), ref) < tol
        assert rel(s.ml_apply_D2(e[:5]), ref[:5]) < tol
        # level-1 V-cycles whose level-2 GMRES steps run eagerly, are captured as CUDA graphs, then
        # replayed: the three agree bit for bit
        x1 = synth.gaussian_coarse(4 ** 4, 2 * n0, nr, seed=146)
        v1s = [s.ml_vcycle1(x1) for _ in range(3)]
        assert all(np.array_equal(o, v1s[0]) for o in v1s[1:])
        if prec == "HALF":
            D2 = ml.levels[1].Dc
            r16 = lambda a: a.astype(np.float32).astype(np.float16).astype(np.float64)  # noqa: E731
            D2h = StencilOperator(D2.lat, r16(D2.B.real) + 1j * r16(D2.B.imag))
            assert rel(s.ml_apply_D2(e), np.stack([D2h.apply(e[r]) for r in range(nr)])) < 5e-6
        z, st, rc = s.ml_solve(b)
        counts = s.ml_counts()
    assert rc == 0 and counts["gmres_steps_D2"] > 0
    for q in range(4):
        assert np.linalg.norm(b[q] - D.apply(z[q])) <= 1e-10 * np.linalg.norm(b[q])
