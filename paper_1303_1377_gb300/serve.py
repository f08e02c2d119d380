"""Serving loop: continuous batching of solve requests over operators resident on one GPU.

Each operator (gauge field, mass, lattice) keeps its setup (P, D_c, clover inverses) on the
device in one ddamg handle with a fixed set of right-hand-side slots and its own CUDA stream.
A worker thread per operator runs outer cycles (`ddamg_slots_cycle`). Between two cycles it
takes finished right-hand sides out and admits queued ones into the freed slots, so a request
joins work that is already on the GPU instead of waiting for a batch to drain. Different
operators run on different streams, and their cycles overlap on the device. A new operator is
admitted only if its estimated device memory fits the free memory minus a reserve.

usage: python -m paper_1303_1377_gb300.serve --bench [--duration 60] [--rate 1.0] [--max-rhs 12]
prints one JSON line: p50/p99 latency and solves/s over a Poisson stream of requests on four
resident operators (16^4, 24^4, 32^4, 32^3 x 64; distinct seeds and masses).
"""
from __future__ import annotations

import argparse
import collections
import json
import threading
import time

import numpy as np

from . import ddamg


def estimate_bytes(V: int, n_vec: int, n_slots: int, n_kv: int) -> int:
    """Device memory of one operator: FP64/FP32/double-word links and site terms, the smoother's
    per-site copies of them (FP32: 5 + 2 x 18 float4; FP16 in half mode: 12 + 2 x 9 uint4), the test
    vectors and interpolation (FP64, FP32, FP16), the setup's work fields (N FP32 fields,
    three of them), and per slot the FP32 bases (n_kv + 1 + n_kv fields) plus the FP64 slot
    right-hand side, iterate and residual work fields."""
    per_site = 4 * 9 * (16 + 8 + 16) + 2 * 72 * (8 + 4 + 8)
    per_site += (4 * 5 + 2 * 18) * 16 + (4 * 3 + 2 * 9) * 16
    per_site += n_vec * 12 * (16 + 16 + 8 + 4)
    per_site += 3 * n_vec * 12 * 8
    per_slot = (2 * n_kv + 1) * 12 * 8 + 6 * 12 * 16
    return int(V * (per_site + n_slots * per_slot) * 1.1) + (256 << 20)


class Request:
    """Right-hand sides b[n, V, 4, 3] for one operator; z, stats and timing filled on completion."""

    def __init__(self, op: str, b: np.ndarray):
        self.op = op
        self.b = np.ascontiguousarray(b, dtype=np.complex128)
        n = self.b.shape[0]
        self.z = np.zeros_like(self.b)
        self.stats = [None] * n
        self.admitted = [None] * n  # time each right-hand side entered a slot
        self.remaining = n
        self.t_submit = None
        self.t_done = None
        self.event = threading.Event()

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.t_submit


def make_solver(dims, U, m0, c_sw, params):
    """A ddamg operator with its setup done, on a CUDA stream of its own."""
    import torch

    stream = torch.cuda.Stream()
    s = ddamg.Solver(dims, U, m0, c_sw, params, setup=False)
    s.set_stream(stream.cuda_stream)
    s.run_setup()
    s._stream = stream  # keep the stream alive with the handle
    return s


class Operator:
    """One resident operator: a set-up solver (anything with the slot calls of ddamg.Solver),
    its slots and the worker thread that cycles them."""

    def __init__(self, name, solver, n_slots):
        self.name = name
        self.solver = solver
        self.solver.slots_open(n_slots)
        self.n_slots = n_slots
        self.owner = [None] * n_slots  # (request, index) per slot
        self.pending = collections.deque()
        self.cv = threading.Condition()
        self.stopping = False
        self.cycles = 0
        self.busy_seconds = 0.0
        self.error = None
        self.thread = threading.Thread(target=self._run, name=f"op-{name}", daemon=True)
        self.thread.start()

    def submit(self, req: Request):
        with self.cv:
            for i in range(req.b.shape[0]):
                self.pending.append((req, i))
            self.cv.notify()

    def stop(self):
        with self.cv:
            self.stopping = True
            self.cv.notify()
        self.thread.join()
        self.solver.close()

    def _running(self):
        return any(o is not None for o in self.owner)

    def _run(self):
        try:
            while True:
                with self.cv:
                    while not self.stopping and not self.pending and not self._running():
                        self.cv.wait()
                    if self.stopping and not self._running():
                        return
                    admit = []
                    for slot in range(self.n_slots):
                        if self.owner[slot] is None and self.pending:
                            admit.append((slot, self.pending.popleft()))
                now = time.perf_counter()
                for slot, (req, i) in admit:
                    self.solver.slot_put(slot, req.b[i])
                    self.owner[slot] = (req, i)
                    req.admitted[i] = now
                t0 = time.perf_counter()
                states, st = self.solver.slots_cycle()
                self.busy_seconds += time.perf_counter() - t0
                self.cycles += 1
                for slot, state in enumerate(states):
                    if state in (ddamg.SLOT_DONE, ddamg.SLOT_FAILED) and self.owner[slot] is not None:
                        req, i = self.owner[slot]
                        self.solver.slot_take(slot, out=req.z[i])
                        req.stats[i] = st[slot]
                        self.owner[slot] = None
                        req.remaining -= 1
                        if req.remaining == 0:
                            req.t_done = time.perf_counter()
                            req.event.set()
        except Exception as e:  # surface the failure to every waiting request
            self.error = e
            with self.cv:
                for o in self.owner:
                    if o is not None:
                        o[0].event.set()
                for req, _ in self.pending:
                    req.event.set()


class Server:
    """Resident operators admitted by device memory; requests routed to their operator."""

    def __init__(self, reserve_bytes: int = 8 << 30, mem_info=None, solver_factory=None):
        self.ops: dict[str, Operator] = {}
        self.reserve = reserve_bytes
        self.admission_log = []
        self._mem_info = mem_info
        self._factory = solver_factory if solver_factory is not None else make_solver

    def _free_bytes(self):
        if self._mem_info is not None:
            return self._mem_info()
        import torch

        return torch.cuda.mem_get_info()[0]

    def add_operator(self, name, dims, U, m0, c_sw=1.0, params=None, n_slots=12):
        """Admit an operator if its estimated device memory fits the free memory minus the
        reserve, with as many of the n_slots slots as fit; returns the slot count."""
        p = params if params is not None else ddamg.default_params()
        V = int(np.prod(dims))
        free = self._free_bytes()
        slots = n_slots
        while slots > 0 and estimate_bytes(V, p.n_vec, slots, p.n_kv) > free - self.reserve:
            slots -= 1
        self.admission_log.append({"op": name, "free_bytes": free, "slots": slots,
                                   "estimate_bytes": estimate_bytes(V, p.n_vec, max(slots, 1), p.n_kv)})
        if slots == 0:
            raise MemoryError(f"operator {name} does not fit: {free} bytes free, reserve {self.reserve}")
        self.ops[name] = Operator(name, self._factory(dims, U, m0, c_sw, p), slots)
        return slots

    def submit(self, op: str, b: np.ndarray) -> Request:
        req = Request(op, b)
        req.t_submit = time.perf_counter()
        self.ops[op].submit(req)
        return req

    def wait(self, req: Request, timeout=None):
        if not req.event.wait(timeout):
            raise TimeoutError(f"request on {req.op} did not finish")
        err = self.ops[req.op].error
        if err is not None:
            raise RuntimeError(f"operator {req.op} failed") from err
        return req

    def close(self):
        for op in self.ops.values():
            op.stop()
        self.ops.clear()


# operators of the serving stream: lattice, eps, seed, m0 (near-critical, distinct per operator)
STREAM_OPERATORS = [
    ("16x16x16x16", (16, 16, 16, 16), 0.5, 11, -0.90),
    ("24x24x24x24", (24, 24, 24, 24), 0.5, 12, -0.91),
    ("32x32x32x32", (32, 32, 32, 32), 0.5, 13, -0.92),
    ("32x32x32x64", (64, 32, 32, 32), 0.5, 3, -0.931885),
]


def run_stream(duration: float, rate: float, seed: int, precision: int, max_rhs: int = 12):
    """Poisson arrivals at `rate` requests/s for `duration` s, each on a random operator with
    1..max_rhs Gaussian right-hand sides; returns the summary dict. Every operator serves one
    warm-up request right after its admission (its workspaces are allocated then), which is
    not counted."""
    from . import synth

    rng = np.random.default_rng(seed)
    srv = Server()
    t_setup = time.perf_counter()
    slots = {}
    for name, dims, eps, gseed, m0 in STREAM_OPERATORS:
        U = synth.gauge_field(dims, eps, gseed)
        slots[name] = srv.add_operator(name, dims, U, m0, 1.0, ddamg.default_params(precision=precision), n_slots=12)
        del U
        # the warm-up request allocates the operator's slot workspaces, so the free memory the
        # next admission sees is what is really left
        srv.wait(srv.submit(name, synth.gaussian_spinors(dims, 1, seed=1)))
    t_setup = time.perf_counter() - t_setup
    live, done = [], []

    def reap():
        for r in [r for r in live if r.event.is_set()]:
            srv.wait(r)
            done.append((r.latency, r.b.shape[0], max(s["rel_residual"] for s in r.stats)))
            live.remove(r)  # drop the request's host arrays

    t0 = time.perf_counter()
    t_next = t0
    while True:
        t_next += rng.exponential(1.0 / rate)
        if t_next - t0 > duration:
            break
        name, dims = STREAM_OPERATORS[rng.integers(len(STREAM_OPERATORS))][:2]
        b = synth.gaussian_spinors(dims, int(rng.integers(1, max_rhs + 1)), seed=int(rng.integers(1 << 30)))
        reap()
        delay = t_next - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        live.append(srv.submit(name, b))
        del b
    while live:
        time.sleep(0.01)
        reap()
    wall = time.perf_counter() - t0
    lat = np.array([d[0] for d in done])
    nsol = sum(d[1] for d in done)
    out = {
        "metric": "serving stream: p50/p99 request latency and solves/s (continuous batching, 4 resident operators)",
        "requests": len(done), "solves": nsol, "wall_s": wall, "solves_per_s": nsol / wall,
        "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
        "max_rel_residual": max(d[2] for d in done), "arrival_rate_per_s": rate, "rhs_per_request": [1, max_rhs],
        "setup_and_warmup_s": t_setup, "slots": slots, "cycles": {k: op.cycles for k, op in srv.ops.items()},
        "busy_s": {k: op.busy_seconds for k, op in srv.ops.items()}, "admission": srv.admission_log,
        "operators": [{"op": n, "eps": e, "seed": g, "m0": m} for n, _, e, g, m in STREAM_OPERATORS],
        "data": "synthetic",
    }
    srv.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--bench", action="store_true")
    ap.add_argument("--duration", type=float, default=60.0)
    ap.add_argument("--rate", type=float, default=1.0)
    ap.add_argument("--max-rhs", type=int, default=12)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--precision", default="half", choices=["single", "half"])
    a = ap.parse_args()
    if not a.bench:
        ap.print_help()
        return
    prec = ddamg.PREC_HALF if a.precision == "half" else ddamg.PREC_SINGLE
    print(json.dumps(run_stream(a.duration, a.rate, a.seed, prec, a.max_rhs)))


if __name__ == "__main__":
    main()
