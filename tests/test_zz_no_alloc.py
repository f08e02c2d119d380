"""The allocation-free coarse-operator entry point (ddamg_apply_Dc_noalloc).

It serves callers that cannot let the library allocate device memory during the
call (a full memory pool, or a loop that cannot pay cudaMalloc's implicit device
synchronisation).  Its result must equal ddamg_apply_Dc's, on consecutive calls
(the fixed scratch array is reused), in double and single precision.  This file
is named to be collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_apply_Dc_noalloc_matches_apply_Dc():
    torch = pytest.importorskip("torch")
    from paper_1303_1377_gb300 import ddamg, synth

    dims, block, N = (8, 8, 8, 8), (4, 4, 4, 4), 4
    U = synth.gauge_field(dims, 0.5, seed=201)
    V = synth.random_test_vectors(dims, N, seed=202)
    for prec, tol in ((ddamg.PREC_DOUBLE, 1e-13), (ddamg.PREC_SINGLE, 1e-6)):
        p = ddamg.default_params(n_vec=N, block=block, precision=prec)
        with ddamg.Solver(dims, U, 0.1, 1.0, p, setup=False) as s:
            s.setup_from_vectors(V)
            for call in range(2):
                e = synth.gaussian_coarse(s.n_coarse, s.coarse_dof, 3, seed=203 + call)
                ref = s.apply_Dc(e)
                ed = torch.from_numpy(e).to("cuda")
                out = torch.empty_like(ed)
                s.apply_Dc_noalloc(ed, out)
                torch.cuda.synchronize()
                got = out.cpu().numpy()
                assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


def test_apply_Dc_noalloc_rejects_oversize_and_host_pointers():
    torch = pytest.importorskip("torch")
    from paper_1303_1377_gb300 import ddamg, synth

    dims, block, N = (8, 8, 8, 8), (4, 4, 4, 4), 4
    p = ddamg.default_params(n_vec=N, block=block, precision=ddamg.PREC_SINGLE)
    with ddamg.Solver(dims, synth.gauge_field(dims, 0.5, seed=201), 0.1, 1.0, p, setup=False) as s:
        s.setup_from_vectors(synth.random_test_vectors(dims, N, seed=202))
        # 16 MiB / (2 * 16 coarse sites * 8 components * 8 bytes) = 8192 right-hand sides at most
        big = torch.zeros((9000, s.n_coarse, s.coarse_dof), dtype=torch.complex128, device="cuda")
        with pytest.raises(ddamg.DDAMGError) as e:
            s.apply_Dc_noalloc(big, torch.empty_like(big))
        assert e.value.status == -1 and "at most 8192" in str(e.value)
        host = np.zeros((1, s.n_coarse, s.coarse_dof), dtype=np.complex128)
        with pytest.raises(ddamg.DDAMGError) as e:
            s.apply_Dc_noalloc(host, np.zeros_like(host))
        assert e.value.status == -1
