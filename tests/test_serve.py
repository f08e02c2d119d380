"""Continuous batching on the GPU: two resident operators of different lattice sizes, requests
arriving while others are in flight. Every result reaches a relative residual <= 1e-10 under the
oracle's D and equals the same right-hand side solved alone (a separate handle with the same
setup) to 1e-8, and a request submitted mid-flight is admitted before the running one finishes."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle.dirac import DiracOperator  # noqa: E402
from paper_1303_1377_gb300 import synth  # noqa: E402

OPS = {
    "8^4": ((8, 8, 8, 8), 0.4, 1, -0.55),
    "8^3x16": ((16, 8, 8, 8), 0.4, 2, -0.5),
}


def test_continuous_batching_results_equal_solves_alone():
    from paper_1303_1377_gb300 import ddamg, serve

    p = ddamg.default_params(n_vec=8, precision=ddamg.PREC_HALF)
    srv = serve.Server(reserve_bytes=1 << 30)
    U = {}
    for name, (dims, eps, seed, m0) in OPS.items():
        U[name] = synth.gauge_field(dims, eps, seed)
        assert srv.add_operator(name, dims, U[name], m0, 1.0, p, n_slots=4) == 4
    reqs = []
    rng = np.random.default_rng(3)
    for q in range(8):
        name = list(OPS)[q % 2]
        dims = OPS[name][0]
        reqs.append(srv.submit(name, synth.gaussian_spinors(dims, int(rng.integers(1, 4)), seed=100 + q)))
        time.sleep(0.02)
    for r in reqs:
        srv.wait(r, timeout=300)
    # B arrives while A runs: it enters at a later cycle boundary, before A has finished
    a = srv.submit("8^4", synth.gaussian_spinors(OPS["8^4"][0], 3, seed=200))
    while a.admitted[0] is None:
        time.sleep(0.0005)
    b_req = srv.submit("8^4", synth.gaussian_spinors(OPS["8^4"][0], 1, seed=201))
    srv.wait(a, timeout=300)
    srv.wait(b_req, timeout=300)
    cycles = {k: op.cycles for k, op in srv.ops.items()}
    srv.close()
    assert max(a.admitted) < b_req.admitted[0] < a.t_done
    assert all(c > 1 for c in cycles.values())
    reqs += [a, b_req]
    for name, (dims, eps, seed, m0) in OPS.items():
        D = DiracOperator(U[name], dims, m0, 1.0)
        mine = [r for r in reqs if r.op == name]
        b = np.concatenate([r.b for r in mine])
        z = np.concatenate([r.z for r in mine])
        with ddamg.Solver(dims, U[name], m0, 1.0, p) as alone:
            za, sta, rc = alone.solve(b)
        assert rc == 0
        for q in range(b.shape[0]):
            nb = np.linalg.norm(b[q])
            assert np.linalg.norm(b[q] - D.apply(z[q])) <= 1e-10 * nb
            assert np.linalg.norm(z[q] - za[q]) <= 1e-8 * np.linalg.norm(za[q])
