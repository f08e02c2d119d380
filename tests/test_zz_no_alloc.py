"""The allocation-free coarse-operator entry point (ddamg_apply_Dc_noalloc).

It serves callers that cannot let the library allocate device memory during the
call (a full memory pool, or a loop that cannot pay cudaMalloc's implicit device
synchronisation).  Its result must equal ddamg_apply_Dc's, on consecutive calls
(the fixed scratch array is reused), in double, single and half precision (the
half-precision handle takes the FP16 tensor-core stencil).  This file is named to
be collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_apply_Dc_noalloc_matches_apply_Dc():
    torch = pytest.importorskip("torch")
    from paper_1303_1377_gb300 import ddamg, synth

    dims, block, N = (8, 8, 8, 8), (4, 4, 4, 4), 4
    U = synth.gauge_field(dims, 0.5, seed=201)
    V = synth.random_test_vectors(dims, N, seed=202)
    # both entry points run the same kernels on the same operator: FP64 to rounding, FP32/FP16
    # storage to the FP32 accumulation's rounding
    for prec, tol in ((ddamg.PREC_DOUBLE, 1e-13), (ddamg.PREC_SINGLE, 1e-6), (ddamg.PREC_HALF, 1e-6)):
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
                assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref)), (prec, call)


def test_apply_Dc_noalloc_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    from paper_1303_1377_gb300 import ddamg, synth

    dims, block, N = (8, 8, 8, 8), (4, 4, 4, 4), 4
    p = ddamg.default_params(n_vec=N, block=block, precision=ddamg.PREC_SINGLE)
    with ddamg.Solver(dims, synth.gauge_field(dims, 0.5, seed=201), 0.1, 1.0, p, setup=False) as s:
        s.setup_from_vectors(synth.random_test_vectors(dims, N, seed=202))
        shape = (1, s.n_coarse, s.coarse_dof)
        # 16 MiB / (2 * 16 coarse sites * 8 components * 8 bytes) = 8192 right-hand sides at most
        big = torch.zeros((9000, s.n_coarse, s.coarse_dof), dtype=torch.complex128, device="cuda")
        with pytest.raises(ddamg.DDAMGError) as e:
            s.apply_Dc_noalloc(big, torch.empty_like(big))
        assert e.value.status == ddamg.ERR_INVALID_ARG and "at most 8192" in str(e.value)
        # the library itself rejects host pointers
        host = np.zeros(shape, dtype=np.complex128)
        rc = ddamg.lib.ddamg_apply_Dc_noalloc(s.h, ctypes.c_void_p(host.ctypes.data), ctypes.c_void_p(host.ctypes.data), 1)
        assert rc == ddamg.ERR_INVALID_ARG
        # the binding rejects what would make the library read or write past the caller's buffers
        good = torch.zeros(shape, dtype=torch.complex128, device="cuda")
        bad = [
            (host, np.zeros_like(host)),                                                    # host arrays
            (good.to(torch.complex64), torch.empty(shape, dtype=torch.complex64, device="cuda")),  # wrong dtype
            (torch.zeros((1, s.n_coarse, s.coarse_dof + 2), dtype=torch.complex128, device="cuda"), good),  # wrong trailing shape
            (torch.zeros((2, s.n_coarse, s.coarse_dof), dtype=torch.complex128, device="cuda"), good),  # output smaller than input
            (good, good.cpu()),                                                             # output not on the GPU
        ]
        for a, b in bad:
            with pytest.raises(ValueError):
                s.apply_Dc_noalloc(a, b)
