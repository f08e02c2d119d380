"""Host logic of the serving loop (paper_1303_1377_gb300/serve.py) with a fake solver on the CPU:
routing, slot ownership, admission between cycles (continuous batching) and the device-memory
admission of operators. The fake has the slot semantics of ddamg.Solver: a right-hand side b
finishes after round(b[0,0,0].real) cycles, and its result is 2 b."""
import threading
import time

import numpy as np
import pytest

serve = pytest.importorskip("paper_1303_1377_gb300.serve", reason="the serving layer imports the CUDA binding")
ddamg = serve.ddamg

DIMS = (2, 2, 2, 2)
V = 16


class FakeSolver:
    def __init__(self):
        self.lock = threading.Lock()
        self.max_running = 0

    def slots_open(self, n):
        self.n = n
        self.state = [ddamg.SLOT_FREE] * n
        self.left = [0] * n
        self.b = [None] * n

    def slot_put(self, slot, b):
        assert self.state[slot] == ddamg.SLOT_FREE
        self.state[slot] = ddamg.SLOT_RUNNING
        self.b[slot] = np.array(b)
        self.left[slot] = int(round(b[0, 0, 0].real))

    def slots_cycle(self):
        time.sleep(0.005)
        run = [s for s in range(self.n) if self.state[s] == ddamg.SLOT_RUNNING]
        self.max_running = max(self.max_running, len(run))
        for s in run:
            self.left[s] -= 1
            if self.left[s] <= 0:
                self.state[s] = ddamg.SLOT_DONE
        st = [{"rel_residual": 0.0, "iterations": 1, "status": 0} for _ in range(self.n)]
        return list(self.state), st

    def slot_take(self, slot, out):
        assert self.state[slot] in (ddamg.SLOT_DONE, ddamg.SLOT_FAILED)
        out[...] = 2 * self.b[slot]
        self.state[slot] = ddamg.SLOT_FREE

    def close(self):
        pass


def rhs(n, cycles, seed):
    b = np.random.default_rng(seed).standard_normal((n, V, 4, 3)) + 0j
    b[:, 0, 0, 0] = cycles
    return b


def make_server(budget=1 << 40, fakes=None):
    made = fakes if fakes is not None else []

    def factory(dims, U, m0, c_sw, p):
        f = FakeSolver()
        made.append(f)
        return f

    return serve.Server(reserve_bytes=0, mem_info=lambda: budget, solver_factory=factory), made


def test_requests_are_routed_and_complete():
    srv, _ = make_server()
    srv.add_operator("a", DIMS, None, 0.0, n_slots=3)
    srv.add_operator("b", DIMS, None, 0.0, n_slots=2)
    reqs = [srv.submit("a" if q % 2 else "b", rhs(1 + q % 3, 1 + q % 4, q)) for q in range(10)]
    for r in reqs:
        srv.wait(r, timeout=20)
        assert np.array_equal(r.z, 2 * r.b)
        assert r.latency is not None and r.latency >= 0
    srv.close()


def test_new_requests_join_between_cycles():
    """A short request submitted while a long one runs is admitted into a free slot at the next
    cycle boundary and finishes first; its second right-hand side waits for a slot to free up."""
    srv, fakes = make_server()
    srv.add_operator("a", DIMS, None, 0.0, n_slots=2)
    long_req = srv.submit("a", rhs(1, 40, 1))
    while long_req.admitted[0] is None:
        time.sleep(0.001)
    short = srv.submit("a", rhs(2, 3, 2))
    srv.wait(short, timeout=20)
    srv.wait(long_req, timeout=20)
    assert short.t_done < long_req.t_done
    assert short.admitted[0] < long_req.t_done and short.admitted[1] < long_req.t_done
    assert short.admitted[1] > short.admitted[0]  # queued until the first one's slot was free
    assert fakes[0].max_running == 2
    srv.close()


def test_operator_admission_by_device_memory():
    per_op = serve.estimate_bytes(64 ** 4, 20, 1, 25)
    srv, _ = make_server(budget=per_op + serve.estimate_bytes(64 ** 4, 20, 2, 25) // 4)
    slots = srv.add_operator("big", (64, 64, 64, 64), None, 0.0, n_slots=12)
    assert 1 <= slots < 12  # only as many slots as the budget holds
    with pytest.raises(MemoryError):
        srv.add_operator("huge", (128, 128, 128, 128), None, 0.0, n_slots=12)
    srv.close()
