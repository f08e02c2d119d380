#!/usr/bin/env python
"""Benchmark: batched DD-alpha-AMG solves to relative residual 1e-10 on one GB300.

One step = one call of ddamg_solve_batch on the 12 point sources (one per spin
and colour) of the 32^3 x 64 workload: FGMRES(25) in FP64, one V-cycle per
iteration (SAP 4^4 blocks, nu = 2, MR(4); 4^4 aggregates, N_v = 20; odd-even
GMRES(30) coarse solve to 5e-2), V-cycle in FP32 (single) or FP32 with FP16
coarse/interpolation storage (half).  The adaptive setup (Algorithm 2) runs
before the timed region and is reported separately.

Prints one JSON line (rank 0).  Multi-GPU runs (torchrun) are independent
replicas, one per GPU (weak scaling; the method needs no exchange between
independent solves).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

if __name__ == "__main__":  # each oracle worker runs on one core (set before numpy loads its BLAS)
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("OMP_NUM_THREADS", "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # lattice (L0 = time first), gauge eps/seed, right-hand sides, method parameters, default V-cycle
    # precision; m0_key: the mass record in workloads.json; oracle_m0_key: the mass of the 8^4
    # counterpart that the CPU baseline times (the 8^4 lattice's own near-critical mass for the
    # near-critical workloads)
    # headline: near-critical mass from the lattice's own spectral edge (smallest |eig| ~ 1e-3)
    # (three levels, the recursion of Sec. 3, with one level-1 V-cycle as the coarse solve; the
    # two-level solve of the same handle is reported beside it)
    "32x32x32x64": dict(dims=(64, 32, 32, 32), eps=0.5, seed=3, nrhs=12, rhs="point", N=20, nu=2, precision="half", levels=3,
                        ml_inner="vcycle", m0_key="lattice_32x32x32x64_critical", oracle_m0_key="lattice_8x8x8x8_eps0.5"),
    # the same lattice at m0 = -0.9319 (smallest |eig| ~ 0.063: an easier system)
    "32x32x32x64-m0.932": dict(dims=(64, 32, 32, 32), eps=0.5, seed=3, nrhs=12, rhs="point", N=20, nu=2, precision="half",
                               m0_key="lattice_32x32x32x64", oracle_m0_key="lattice_32x32x32x64"),
    # FP32 V-cycle, one Gaussian right-hand side, near-critical (the Dslash / SAP profile case)
    "16x16x16x16": dict(dims=(16, 16, 16, 16), eps=0.5, seed=1, nrhs=1, rhs="gaussian", N=20, nu=2, precision="single",
                        m0_key="lattice_16x16x16x16_critical", oracle_m0_key="lattice_8x8x8x8_eps0.5", oracle_seed=3,
                        count_key="32x32x32x64"),
    # memory-bound run: N_v = 24, FP16 interpolation and coarse blocks, FP32 smoother, FP64 outer
    # residual; the setup updates the test vectors in groups of 8 and frees the FP64 vectors after
    # (lean), FGMRES(10) (the paper's restart length at large volume), the 12 right-hand sides solved
    # in three groups of four (what fits the device next to the operator)
    "48x48x48x96": dict(dims=(96, 48, 48, 48), eps=0.55, seed=5, nrhs=12, rhs="point", N=24, nu=2, precision="half", n_kv=10,
                        lean=1, setup_group=8, rhs_group=4, levels=3, ml_inner="vcycle", m0_key="lattice_48x48x48x96_critical", gap=1e-3,
                        oracle_m0_key="lattice_8x8x8x8_eps0.55", count_key="48x48x48x96"),
    # the oracle's size, all FP64, nu = 3, smallest |eig| ~ 1e-3
    "8x8x8x8": dict(dims=(8, 8, 8, 8), eps=0.4, seed=1, nrhs=1, rhs="gaussian", N=20, nu=3, precision="double",
                    m0_key="lattice_8x8x8x8", oracle_m0_key="lattice_8x8x8x8"),
}
C_SW = 1.0
WORKLOADS_JSON = os.path.join(ROOT, "paper_1303_1377_gb300", "workloads.json")
TRAFFIC_JSON = os.path.join(ROOT, "profiles", "ncu_traffic.json")


def workload_m0(w, key="m0_key"):
    """The workload's mass: the record's m0, or -Re(lambda_L) + the workload's own gap when it sets one."""
    data = json.load(open(WORKLOADS_JSON))
    rec = data[w[key]]
    if key == "m0_key" and "gap" in w:
        return -float(rec["lambda_L_m0_0"][0]) + w["gap"], rec
    return float(rec["m0"]), rec


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index: int, path=None):
        self.gpu = gpu_index
        self.proc = None
        self.path = path
        self.tmp = False

    def start(self):
        try:
            self.tmp = self.path is None
            if self.tmp:
                fd, self.path = tempfile.mkstemp(prefix=f"clocks_gpu{self.gpu}_", suffix=".csv")
                os.close(fd)
            else:
                os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    @staticmethod
    def parse(lines):
        """Median SM clock, the maximum clock and every throttle reason seen Active, from the
        query lines (index, sm, max sm, power, active mask, then the four reasons)."""
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}

    def stop(self):
        if not self.proc:
            if self.tmp and self.path and os.path.exists(self.path):
                os.remove(self.path)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            out = self.parse(f)
        if self.tmp:
            os.remove(self.path)
        return out


def metric_name(workload):
    if workload.startswith("32x32x32x64"):
        return "solves/s to rel. residual 1e-10 (32^3x64, 12 point sources)"
    return f"solves/s to rel. residual 1e-10 ({workload})"


def workload_description(workload, w, m0):
    """The workload as both arms state it in config.workload."""
    rec = json.load(open(WORKLOADS_JSON)).get(w["m0_key"], {})
    lam = rec.get("lambda_L_m0_0") or rec.get("lambda_L_source")
    edge = ""
    if lam:
        src = "measured on this lattice" if rec.get("source") else f"of {rec.get('derived_from', 'a smaller lattice')}"
        edge = f" (leftmost eigenvalue of D(0) {lam[0]:.5f}{lam[1]:+.4f}i {src}: smallest |eig| of D ~ {abs(complex(lam[0] + m0, lam[1])):.1e})"
    return (f"{workload} lattice (L0={w['dims'][0]}), SU(3) links exp(i eps H) eps={w['eps']} seed={w['seed']}, c_sw={C_SW}, "
            f"m0={m0:.6f}{edge}, {w['nrhs']} {w['rhs']} sources per step, N_v={w['N']}, 4^4 SAP blocks and aggregates, nu={w['nu']}, "
            f"MR(4), FGMRES(25) tol 1e-10, coarse GMRES(30) tol 5e-2")


def make_rhs(w, V):
    from paper_1303_1377_gb300 import synth

    if w["rhs"] == "point":
        b = np.zeros((12, V, 4, 3), dtype=np.complex128)
        for k in range(12):
            b[k, 0, k // 3, k % 3] = 1.0
        return b[: w["nrhs"]]
    return synth.gaussian_spinors(w["dims"], w["nrhs"], seed=w["seed"] + 1000)


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample (the same workload on 8^4), on every host core
# ---------------------------------------------------------------------------
_ORACLE = {}


def _oracle_build(w, m0):
    """Worker initialiser: the oracle's two-level method on the workload's 8^4 counterpart (same eps,
    c_sw, m0, N_v, 4^4 blocks, nu; P from seeded random test vectors) and one point source."""
    from oracle.dirac import DiracOperator
    from oracle.mg import Params as OParams
    from oracle.mg import TwoLevel
    from paper_1303_1377_gb300 import synth

    sdims = (8, 8, 8, 8)
    U = synth.gauge_field(sdims, w["eps"], w.get("oracle_seed", w["seed"]))
    D = DiracOperator(U, sdims, m0, C_SW)
    mg = TwoLevel(D, OParams(N=w["N"], nu=w["nu"]), vectors=synth.random_test_vectors(sdims, w["N"], seed=w["seed"] + 7))
    b = np.zeros((D.V, 4, 3), dtype=np.complex128)
    b[0, 0, 0] = 1.0
    _ORACLE.update(D=D, mg=mg, b=b)


def _oracle_time(seconds_budget):
    """Time whole oracle FGMRES iterations (one V-cycle each) for about seconds_budget seconds."""
    from oracle.krylov import fgmres

    D, mg, b = _ORACLE["D"], _ORACLE["mg"], _ORACLE["b"]
    t0 = time.perf_counter()
    iters = 0
    while True:
        fgmres(D.apply, mg.vcycle, b, n_kv=25, tol=0.0, maxiter=1)
        iters += 1
        if time.perf_counter() - t0 > seconds_budget:
            break
    return iters, time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OracleBaseline:
    """The oracle timed on all host cores: one single-threaded worker process per core (spawned, so the
    pool is safe after CUDA has been initialised), each running independent FGMRES iterations.  The
    aggregate rate is the sum of the workers' rates, scaled by volume and by the oracle's own
    iteration count per solve: (sum_i iterations_i / seconds_i) / (V / 8^4) / iterations per solve."""

    def __init__(self, w, m0, fgmres_iters_per_solve, cores=None):
        import multiprocessing as mp

        self.w, self.iters_per_solve, self.m0 = w, fgmres_iters_per_solve, m0
        self.cores = cores or host_cores()
        os.environ["OPENBLAS_NUM_THREADS"] = os.environ["OMP_NUM_THREADS"] = "1"  # one thread per worker
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_build, initargs=(w, m0))

    def sample(self, seconds_budget):
        res = self.pool.map(_oracle_time, [seconds_budget] * self.cores)
        rate = sum(i / t for i, t in res)  # oracle FGMRES iterations per second, all workers
        scale = float(np.prod(self.w["dims"]) / 8 ** 4)
        value = rate / scale / self.iters_per_solve
        n_it = sum(i for i, _ in res)
        info = (f"{n_it} oracle FGMRES iterations (one point source each, {self.cores} single-threaded worker processes, "
                f"{seconds_budget:.0f} s each) on the 8^4 version of the workload (same eps, c_sw, N_v={self.w['N']}, 4^4 blocks, "
                f"seed={self.w.get('oracle_seed', self.w['seed'])}, "
                f"nu={self.w['nu']}, m0={self.m0:.6f}; P from seeded random vectors): {rate:.2f} iterations/s in aggregate, "
                f"divided by {self.iters_per_solve} FGMRES iterations per solve (the oracle's own count on that 8^4 lattice with "
                f"the adaptive setup)" + (f" and by the volume ratio {scale:.0f}: an extrapolation to the workload's size, not a run "
                                          f"at it" if scale != 1 else ": a run at the workload's size"))
        return value, info

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_iterations(workload):
    """FGMRES iterations per solve of the oracle's full method (adaptive setup) on the workload's
    8^4 counterpart, as recorded by oracle/count_iterations.py."""
    rec = json.load(open(WORKLOADS_JSON)).get("fgmres_iterations_8x8x8x8", {}).get(WORKLOADS[workload].get("count_key", workload))
    if not rec:
        return None, None
    return int(rec["iterations"]), f"oracle, 8^4 counterpart with the adaptive setup: {rec['iterations']} iterations"


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    m0, _ = workload_m0(w)
    m0_oracle, _ = workload_m0(w, "oracle_m0_key")
    iters_per_solve, src = oracle_iterations(args.workload)
    if iters_per_solve is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle iteration count for {args.workload}: "
                          f"run python -m oracle.count_iterations for it"}), flush=True)
        return 0
    base = OracleBaseline(w, m0_oracle, iters_per_solve)
    vals = []
    for k in range(args.warmup + args.steps):
        v, info = base.sample(4.0)
        if k >= args.warmup:
            vals.append(v)
    base.close()
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": metric_name(args.workload), "value": value,
        "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * w["nrhs"] / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_description(args.workload, w, m0), "precision": "FP64 throughout (the oracle)",
                   "l2": "oracle on host cores"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": base.cores, "kind": "oracle", "sample": info},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# --profile-case: each hot kernel of the solve once on a small lattice (for ncu captures)
# ---------------------------------------------------------------------------
def run_profile_case(args):
    """Build D for a synthetic gauge field and an interpolation from seeded random test vectors, then
    apply one SAP iteration, three steps of the odd-even coarse GMRES, one double-word Dslash, one FP32
    Dslash, one restriction and one prolongation to nrhs right-hand sides resident on the GPU; with
    --levels 3 also a level 2 from seeded random level-1 vectors, one level-1 SAP iteration, two
    level-1 restrictions, one level-2 operator product and one level-1 prolongation."""
    import torch

    from paper_1303_1377_gb300 import ddamg, synth

    dims = tuple(int(v) for v in args.dims.split(","))
    prec = {"single": ddamg.PREC_SINGLE, "half": ddamg.PREC_HALF, "half32": ddamg.PREC_HALF, "double": ddamg.PREC_DOUBLE}[args.precision]
    U = synth.gauge_field(dims, 0.5, 1)
    p = ddamg.default_params(n_vec=20, precision=prec, smoother_fp16=0 if args.precision == "half32" else 1)
    s = ddamg.Solver(dims, U, args.m0 if args.m0 is not None else -0.93, 1.0, p, setup=False)
    s.setup_from_vectors(synth.random_test_vectors(dims, 20, 2))
    x = torch.from_numpy(synth.gaussian_spinors(dims, args.nrhs, 3)).cuda()
    s.apply_sap(x, 1)
    e = torch.from_numpy(synth.gaussian_coarse(s.n_coarse, s.coarse_dof, args.nrhs, 4)).cuda()
    s.coarse_solve(e, fixed_iters=3)
    if prec != ddamg.PREC_DOUBLE:
        s.apply_D_mixed(x.to(torch.complex64))
        s.apply_D_f32(x.to(torch.complex64))
    s.prolong(s.restrict(x))
    if args.levels == 3:  # level-1 SAP colour steps, restriction, prolongation and level-2 operator
        mlp = ddamg.ml_default_params()
        s.ml_build(synth.gaussian_coarse(s.n_coarse, s.coarse_dof, mlp.n_vec1, 6), mlp)
        e = torch.from_numpy(synth.gaussian_coarse(s.n_coarse, s.coarse_dof, args.nrhs, 7)).cuda()
        s.ml_apply_sap1(e, 1)
        s.ml_apply_D2(s.ml_restrict1(e))
        s.ml_prolong1(s.ml_restrict1(e))
    torch.cuda.synchronize()
    s.close()
    print("ok")
    return 0


def run_small(name, reps=3):
    """Set up and solve one of the small workloads: setup seconds, median solve time of reps solves,
    iteration counts, the FP64 relative residual, and (16^4) the Dslash and SAP kernel times."""
    import torch

    from paper_1303_1377_gb300 import ddamg, synth

    w = WORKLOADS[name]
    m0, _ = workload_m0(w)
    prec = {"single": ddamg.PREC_SINGLE, "half": ddamg.PREC_HALF, "double": ddamg.PREC_DOUBLE}[w["precision"]]
    U = synth.gauge_field(w["dims"], w["eps"], w["seed"])
    t = time.perf_counter()
    s = ddamg.Solver(w["dims"], U, m0, C_SW, ddamg.default_params(n_vec=w["N"], nu=w["nu"], precision=prec), setup=True)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t
    b = torch.from_numpy(make_rhs(w, int(np.prod(w["dims"])))).to("cuda")
    z, st, rc = s.solve_zero_guess(b)
    times = []
    s.profile(["dslash_fp32", "dslash_fp64", "sap_block_mr"])
    for _ in range(reps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        z, st, rc = s.solve_zero_guess(b)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
    prof = s.profile_read()
    s.profile([])
    r = b - s.apply_D(z)
    rel = float((torch.linalg.vector_norm(r.reshape(b.shape[0], -1), dim=1) / torch.linalg.vector_norm(b.reshape(b.shape[0], -1), dim=1)).max())
    s.close()
    out = {"workload": workload_description(name, w, m0), "precision": w["precision"], "setup_seconds": t_setup,
           "solves_per_s": b.shape[0] / float(np.median(times)), "solve_seconds_median": float(np.median(times)), "status": rc,
           "fgmres_iterations": max(q["iterations"] for q in st), "coarse_iterations_per_solve": st[0]["coarse_iterations"],
           "max_rel_residual": rel}
    # per-launch times of the fine kernels (at these volumes the operator and vectors are L2-resident,
    # so the algorithmic GB/s says how fast the kernel streams from L2, not from HBM)
    out["kernels"] = {k: {"launches_per_solve": v["launches"] / reps, "avg_launch_us": 1e3 * v["total_ms"] / max(1, v["launches"]),
                          "algorithmic_gbs": v["bytes"] / max(1e-9, v["total_ms"]) / 1e6, "ms_per_solve": v["total_ms"] / reps}
                      for k, v in prof.items()}
    out["kernels_note"] = "operator and vectors fit in the 129 MB L2 at this volume: times, not HBM bandwidth"
    return out


def gpu_local_cpus(dev):
    """The host CPUs that nvidia-smi lists as local to CUDA device `dev` (matched by UUID), or None.
    Pinned buffers first touched by a thread running there sit in the GPU's own host memory."""
    import torch

    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid).lower()
        q = subprocess.run(["nvidia-smi", "--query-gpu=index,uuid", "--format=csv,noheader"], capture_output=True, text=True,
                           timeout=30).stdout
        idx = next((int(line.split(",")[0]) for line in q.splitlines()
                    if len(line.split(",")) >= 2 and line.split(",")[1].strip().lower().endswith(uuid)), None)
        if idx is None:
            return None
        topo = [line.split("\t") for line in subprocess.run(["nvidia-smi", "topo", "-m"], capture_output=True, text=True,
                                                             timeout=30).stdout.splitlines() if line.strip()]
        head = [c.strip() for c in topo[0]]
        col = head.index("CPU Affinity")
        row = next(r for r in topo[1:] if r[0].strip() == f"GPU{idx}")
        cpus = set()
        for part in row[col].strip().split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        return cpus & os.sched_getaffinity(0) or None
    except Exception:  # no nvidia-smi, another table layout: leave the placement to the OS
        return None


def measure_dslash(solver, b, hbm_peak, reps=10):
    """FP32 and FP64 Dslash (the fine D of Sec. 2.2) on the batch b (device, complex128): average launch
    time from the library's per-launch CUDA events and the algorithmic bytes per launch (links and site
    term once, each right-hand side's input and output once), as GB/s and as a fraction of HBM."""
    import torch

    out = {"nrhs": int(b.shape[0]), "reps": reps,
           "bytes_model": "V x (36 link + 72 site-term reals) x sizeof(real) once per launch + n_rhs x V x 24 reals x 2 (in, out)"}
    x32 = b.to(torch.complex64)
    torch.cuda.synchronize()  # x32 is written on torch's stream, read on the library's
    solver.profile(["dslash_fp32", "dslash_fp64"])
    for name, fn, arg in (("fp32", solver.apply_D_f32, x32), ("fp64", solver.apply_D, b)):
        fn(arg)  # warm-up (and staging buffers)
        torch.cuda.synchronize()
        solver.profile_reset()
        for _ in range(reps):
            fn(arg)
        torch.cuda.synchronize()
        d = solver.profile_read()["dslash_" + name]
        sec = d["total_ms"] / max(1, d["launches"]) / 1e3
        bpl = d["bytes"] / max(1, d["launches"])
        out[name] = {"gbs": bpl / sec / 1e9, "frac_of_hbm": bpl / sec / 1e9 / hbm_peak, "avg_launch_us": 1e6 * sec,
                     "algorithmic_bytes_per_launch": bpl, "launches": d["launches"]}
    solver.profile([])
    del x32
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="32x32x32x64", choices=list(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["single", "half", "half32", "double"],
                    help="V-cycle precision (default: the workload's); half32 = half with the smoother's links and site terms "
                         "kept in FP32")
    ap.add_argument("--outer", default="refine", choices=["refine", "dw"],
                    help="outer scheme of the mixed-precision modes: FP32 cycles + FP64 residual correction, or double-word FGMRES")
    ap.add_argument("--cycle-tol", type=float, default=1e-5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain single-RHS FP64 comparison solve")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving stream (continuous batching over four operators)")
    ap.add_argument("--serving-seconds", type=float, default=20.0)
    ap.add_argument("--no-small", action="store_true", help="skip the 8^4 and 16^4 configurations")
    ap.add_argument("--no-two-level", action="store_true", help="skip the two-level solve on the three-level handle")
    ap.add_argument("--no-conforming", action="store_true",
                    help="skip the half-precision variant whose smoother reads FP32 links and site terms")
    ap.add_argument("--clocks-csv", default=None, help="keep the nvidia-smi samples of the timed region in this file")
    ap.add_argument("--levels", type=int, default=None, choices=[2, 3],  # with --profile-case: 3 adds the level-1 kernels
                    help="2 or 3 (the recursion to a third level: level-1 blocks 2^4, N_1 = 20, adaptive level-1 setup); "
                         "default: the workload's")
    ap.add_argument("--ml-inner", default=None, choices=["fgmres", "vcycle"],
                    help="with --levels 3: the level-1 solve inside the fine V-cycle (FGMRES to 5e-2, or one level-1 V-cycle)")
    ap.add_argument("--profile-case", action="store_true", help="run each hot kernel once on --dims (for ncu) and exit")
    ap.add_argument("--dims", default="24,24,24,24", help="with --profile-case: the lattice")
    ap.add_argument("--nrhs", type=int, default=12, help="with --profile-case: right-hand sides")
    ap.add_argument("--m0", type=float, default=None,
                    help="override the workload's mass (with --profile-case: the mass, default -0.93)")
    args = ap.parse_args()
    if args.profile_case:
        args.precision = args.precision or "half"
        return run_profile_case(args)
    w = WORKLOADS[args.workload]
    args.precision = args.precision or w["precision"]
    args.levels = args.levels or w.get("levels", 2)
    args.ml_inner = args.ml_inner or w.get("ml_inner", "fgmres")
    if args.impl == "reference":
        return run_reference(args, w)

    import torch

    from paper_1303_1377_gb300 import ddamg, synth
    from paper_1303_1377_gb300.replicas import aggregate

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    m0, _ = workload_m0(w)
    if args.m0 is not None:
        m0 = args.m0
    dims = w["dims"]
    V = int(np.prod(dims))
    t = time.perf_counter()
    U = synth.gauge_field(dims, w["eps"], w["seed"])
    t_gauge = time.perf_counter() - t
    prec = {"single": ddamg.PREC_SINGLE, "half": ddamg.PREC_HALF, "half32": ddamg.PREC_HALF, "double": ddamg.PREC_DOUBLE}[args.precision]
    params = ddamg.default_params(n_vec=w["N"], nu=w["nu"], precision=prec,
                                  outer=ddamg.OUTER_REFINE if args.outer == "refine" else ddamg.OUTER_DW, cycle_tol=args.cycle_tol,
                                  smoother_fp16=0 if args.precision == "half32" else 1, n_kv=w.get("n_kv", 25),
                                  lean=w.get("lean", 0), setup_group=w.get("setup_group", 0))
    t = time.perf_counter()
    solver = ddamg.Solver(dims, U, m0, C_SW, params, setup=True)
    if args.levels == 3:
        mlp = ddamg.ml_default_params(inner=1 if args.ml_inner == "vcycle" else 0)
        solver.ml_setup(synth.gaussian_coarse(solver.n_coarse, solver.coarse_dof, mlp.n_vec1, seed=w["seed"] + 11), mlp)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t
    print(f"[bench] setup done in {t_setup:.1f} s (m0 = {m0:.6f})", file=sys.stderr, flush=True)
    del U
    stream = torch.cuda.Stream()
    solver.set_stream(stream.cuda_stream)
    bh = make_rhs(w, V)
    nr = bh.shape[0]
    b = torch.from_numpy(bh).to("cuda")
    z = torch.zeros_like(b)

    # the paper's zero initial guess: z is output only
    solve_fn = solver.ml_solve_zero_guess if args.levels == 3 else solver.solve_zero_guess

    group = w.get("rhs_group", nr)  # right-hand sides per solve call (all of them unless memory says otherwise)

    def step(fn=None):
        st = []
        for g0 in range(0, nr, group):
            zz, sg, rc = (fn or solve_fn)(b[g0:g0 + group], z[g0:g0 + group])
            if rc != 0:
                raise RuntimeError(f"solve status {rc}")
            st += sg
        return st

    for k in range(args.warmup):
        t_w = time.perf_counter()
        st = step()
        print(f"[bench] warm-up step {k}: {time.perf_counter() - t_w:.2f} s, FGMRES iterations {max(q['iterations'] for q in st)}",
              file=sys.stderr, flush=True)
    # identify the dominant kernel family on one profiled step
    solver.profile()
    solver.profile_reset()
    step()
    prof_all = solver.profile_read()
    # the dominant kernel family (families recorded without bytes time whole recursion stages)
    dominant = max((k for k in prof_all if prof_all[k]["bytes"] > 0), key=lambda k: prof_all[k]["total_ms"])
    solver.profile([dominant])
    solver.profile_reset()
    # timed region
    clocks = ClockSampler(local, args.clocks_csv)
    clocks.start()
    n_launch0 = ddamg.launch_count()
    launches_before_timed = n_launch0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = ddamg.launch_count() - n_launch0
    clk = clocks.stop()
    prof = solver.profile_read()
    solver.profile([])
    # whole-job throughput: solves summed over the replicas / slowest replica's time
    value, ms, _ = aggregate(ms, nr * args.steps, dist=dist, device="cuda")
    # residual check of the last solve, in FP64 through the library's D
    # (one right-hand side at a time on memory-lean workloads, beside the solver's resident work space)
    rel = 0.0
    chk = 1 if w.get("lean") else group
    for g0 in range(0, nr, chk):
        r = b[g0:g0 + chk] - solver.apply_D(z[g0:g0 + chk])
        ng = r.shape[0]
        rel = max(rel, (torch.linalg.vector_norm(r.reshape(ng, -1), dim=1) /
                        torch.linalg.vector_norm(b[g0:g0 + chk].reshape(ng, -1), dim=1)).max().item())
        del r
    # the two-level solve on the same handle (the fine V-cycle with the odd-even GMRES on D_c), for
    # comparison with the recursion
    two_level = None
    if args.levels == 3 and args.workload.startswith("32x32x32x64") and not args.no_two_level:
        step(solver.solve_zero_guess)
        t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0e.record(stream)
        st2 = [step(solver.solve_zero_guess) for _ in range(2)]
        t1e.record(stream)
        torch.cuda.synchronize()
        ms2 = t0e.elapsed_time(t1e) / 2
        two_level = {"value": nr / (ms2 / 1e3), "unit": "solves/s", "ms_per_step": ms2, "steps": 2,
                     "fgmres_iterations": max(q["iterations"] for q in st2[-1]),
                     "coarse_iterations_per_solve": st2[-1][0]["coarse_iterations"],
                     "coarse_solve": "odd-even GMRES(30) on D_c to 5e-2 (tensor-core stencil)"}
    # Dslash bandwidth at the workload's size and right-hand sides (half of the headline metric):
    # kernel time from CUDA events around each Dslash launch, algorithmic bytes per launch
    dslash_rates = measure_dslash(solver, b[:chk], peaks()[0])
    # and for one right-hand side (links and site terms not shared across fields: the HBM-bound case)
    dslash_1rhs = measure_dslash(solver, b[:1], peaks()[0]) if chk > 1 else None
    # end to end through the C ABI with host buffers (pinned), copies inside the timed region: b goes
    # in, z comes out; the zero-guess entry point never reads z (the paper's zero initial guess)
    e2e = None
    if not args.no_e2e:
        # the host buffers go to the GPU's own host memory: this thread runs on the GPU's local CPUs
        # while it allocates and first touches them (the oracle's worker pool later gets every core)
        aff0 = os.sched_getaffinity(0)
        local_cpus = gpu_local_cpus(local)
        if local_cpus:
            os.sched_setaffinity(0, local_cpus)
        bhost = torch.from_numpy(bh).pin_memory()
        zhost = torch.empty_like(bhost).pin_memory()
        solver.set_stream(None)
        def e2e_step():
            bn, zn = bhost.numpy(), zhost.numpy()
            for g0 in range(0, nr, group):
                solve_fn(bn[g0:g0 + group], zn[g0:g0 + group])
        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        e2e_s = time.perf_counter() - t0
        nbytes = bh.nbytes
        # the host link alone: one pinned-memory copy of b in each direction, timed with CUDA events
        dev = torch.empty_like(bhost, device="cuda")
        c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        c0.record()
        dev.copy_(bhost, non_blocking=True)
        c1.record()
        zhost.copy_(dev, non_blocking=True)
        c2.record()
        torch.cuda.synchronize()
        link = {"h2d_gbs": nbytes / c0.elapsed_time(c1) / 1e6, "d2h_gbs": nbytes / c1.elapsed_time(c2) / 1e6}
        del dev
        e2e = {"value": world * nr * args.steps / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "entry": "ddamg_ml_solve_zero_guess" if args.levels == 3 else "ddamg_solve_batch_zero_guess",
               "host_link_copy": link,
               "host_cpus": f"{len(local_cpus)} CPUs local to the GPU (nvidia-smi topo)" if local_cpus else "placement left to the OS"}
        os.sched_setaffinity(0, aff0)
    # roofline of the dominant kernel: HBM-bound families against the measured copy bandwidth;
    # families whose algorithmic flops per byte exceed the FP32 ridge against the FP32 FMA peak
    # (SMs x 128 FP32 lanes x 2 flops x the maximum SM clock)
    peak, peak_kind = peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    d = prof.get(dominant, {"launches": 0, "total_ms": 0.0, "bytes": 0.0, "flops": 0.0})
    n_l = max(1, d["launches"])
    sec = d["total_ms"] / n_l / 1e3 if d["launches"] else float("inf")
    bytes_pl, flops_pl = d["bytes"] / n_l, d.get("flops", 0.0) / n_l
    sm_mhz = clk.get("sm_max_mhz") or clk.get("sm_mhz") or 2070.0
    fp32_peak_tf = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    ridge = fp32_peak_tf * 1e12 / (peak * 1e9)
    tr = json.load(open(TRAFFIC_JSON)).get(f"{args.workload}/{args.precision}/{dominant}")
    traffic = tr["bytes_per_launch"] if tr else None  # null: no DRAM capture of this kernel version
    if flops_pl > 0 and flops_pl / bytes_pl > ridge:
        ach = flops_pl / sec / 1e12
        roof = {"bound": "alu", "kernel": dominant, "achieved": ach, "peak": fp32_peak_tf,
                "peak_kind": f"FP32 FMA peak from unit counts: {sms} SMs (device property) x 128 lanes x 2 flops x {sm_mhz:.0f} MHz "
                             f"(maximum SM clock)", "unit": "TFLOP/s",
                "frac": ach / fp32_peak_tf, "traffic": traffic, "hbm_achieved_gbs": bytes_pl / sec / 1e9, "hbm_peak_gbs": peak,
                "arithmetic_intensity": flops_pl / bytes_pl, "ridge": ridge}
    else:
        ach = bytes_pl / sec / 1e9
        roof = {"bound": "hbm", "kernel": dominant, "achieved": ach, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": ach / peak, "traffic": traffic}
    if traffic is None:
        roof["traffic_note"] = "no ncu DRAM capture of the current version of this kernel"
    roof.update({"launches": d["launches"], "avg_launch_us": 1e6 * sec, "algorithmic_bytes_per_launch": bytes_pl,
                 "algorithmic_flops_per_launch": flops_pl, "time_share_of_step": d["total_ms"] / ms if ms else None})
    iters = [s["iterations"] for s in stats[-1]]
    line = {
        "metric": metric_name(args.workload),
        "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"single": "f32+f64", "half": "f16-storage/f32+f64", "half32": "f16-storage/f32+f64",
                  "double": "f64"}[args.precision], "data": "synthetic",
        "config": {"workload": workload_description(args.workload, w, m0),
                   "l2": "inputs larger than L2 (b: %.1f GB)" % (bh.nbytes / 1e9), "precision": args.precision, "levels": args.levels, **({"ml_inner": args.ml_inner} if args.levels == 3 else {}),
                   "outer": (f"FP32 FGMRES cycles to {args.cycle_tol:g} + FP64 residual correction" if args.outer == "refine"
                             and args.precision != "double" else "double-word FGMRES" if args.precision != "double" else "FP64 FGMRES")},
        "roofline": roof,
        "clocks": clk,
        "gpu_launches": launches,
        "gpu_launches_before_timed": launches_before_timed,
        "solve_seconds_host": [s["solve_seconds"] for s in stats[-1]][:1],
        "coarse_seconds_host": [s["coarse_seconds"] for s in stats[-1]][:1],
        "e2e": e2e,
        "fgmres_iterations": iters,
        "fgmres_restarts": [s["restarts"] for s in stats[-1]],
        "coarse_iterations_per_solve": stats[-1][0]["coarse_iterations"],
        "max_rel_residual": rel,
        "setup_seconds": t_setup,
        "setup_rounds": solver.setup_report()[0],
        # one setup serving one batch: the batch's solves over setup + one step's time
        "amortised_incl_setup": {"value": nr / (t_setup + ms / args.steps / 1e3), "unit": "solves/s",
                                 "per": f"one setup and one batch of {nr} right-hand sides"},
        "gauge_generation_seconds": t_gauge,
        "kernel_profile_first_step": prof_all,
        "dslash": dslash_rates,
        "dslash_1rhs": dslash_1rhs,
        **({"two_level_same_handle": two_level} if two_level else {}),
    }
    if args.levels == 3:
        line["ml_counts_last_step"] = solver.ml_counts()  # FGMRES steps on D_1, GMRES steps on D_2, level-1 V-cycles
    solver.close()
    del b, z
    torch.cuda.empty_cache()
    # the plain path: one right-hand side, every step of the solve in FP64 (same library)
    if not args.no_plain and world == 1:
        Up = synth.gauge_field(dims, w["eps"], w["seed"])
        pp = ddamg.default_params(n_vec=w["N"], nu=w["nu"], precision=ddamg.PREC_DOUBLE)
        tps = time.perf_counter()
        plain = ddamg.Solver(dims, Up, m0, C_SW, pp, setup=True)
        t_plain_setup = time.perf_counter() - tps
        del Up
        b1 = torch.from_numpy(bh[:1]).to("cuda")
        z1 = torch.zeros_like(b1)
        plain.solve_zero_guess(b1, z1)  # warm-up
        torch.cuda.synchronize()
        times = []
        for _ in range(5):
            tp0 = time.perf_counter()
            _, st1, rc1 = plain.solve_zero_guess(b1, z1)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - tp0)
        tp = float(np.median(times))
        line["plain_fp64_single_rhs"] = {"value": 1.0 / tp, "unit": "solves/s", "timing": "median of 5 solves (wall clock)",
                                         "seconds": times, "fgmres_iterations": st1[0]["iterations"],
                                         "rel_residual": st1[0]["rel_residual"], "status": rc1, "setup_seconds": t_plain_setup,
                                         "speedup_of_value": value / (1.0 / tp)}
        plain.close()
    # the half-precision variant whose smoother keeps FP32 links and site terms (FP16 only on P, D_c
    # and D_ee^-1): its own handle and setup, one warm-up and two timed steps of the same batch
    if (args.precision == "half" and args.workload.startswith("32x32x32x64") and not args.no_conforming and world == 1):
        Uc = synth.gauge_field(dims, w["eps"], w["seed"])
        pc = ddamg.default_params(n_vec=w["N"], nu=w["nu"], precision=ddamg.PREC_HALF,
                                  outer=ddamg.OUTER_REFINE if args.outer == "refine" else ddamg.OUTER_DW, cycle_tol=args.cycle_tol,
                                  smoother_fp16=0, n_kv=w.get("n_kv", 25), lean=w.get("lean", 0), setup_group=w.get("setup_group", 0))
        sc = ddamg.Solver(dims, Uc, m0, C_SW, pc, setup=True)
        del Uc
        if args.levels == 3:
            mlc = ddamg.ml_default_params(inner=1 if args.ml_inner == "vcycle" else 0)
            sc.ml_setup(synth.gaussian_coarse(sc.n_coarse, sc.coarse_dof, mlc.n_vec1, seed=w["seed"] + 11), mlc)
        sc.set_stream(stream.cuda_stream)
        fn_c = sc.ml_solve_zero_guess if args.levels == 3 else sc.solve_zero_guess
        bc = torch.from_numpy(bh).to("cuda")
        zc = torch.zeros_like(bc)

        def step_c():
            st = []
            for g0 in range(0, nr, group):
                _, sg, rc = fn_c(bc[g0:g0 + group], zc[g0:g0 + group])
                if rc != 0:
                    raise RuntimeError(f"solve status {rc}")
                st += sg
            return st

        step_c()
        torch.cuda.synchronize()
        c0e, c1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0e.record(stream)
        stc = [step_c() for _ in range(2)]
        c1e.record(stream)
        torch.cuda.synchronize()
        msc = c0e.elapsed_time(c1e) / 2
        line["fp32_smoother_variant"] = {"value": nr / (msc / 1e3), "unit": "solves/s", "ms_per_step": msc, "steps": 2, "warmup": 1,
                                         "fgmres_iterations": max(q["iterations"] for q in stc[-1]),
                                         "max_rel_residual": max(q["rel_residual"] for q in stc[-1]),
                                         "precision": "FP16 P, D_c and D_ee^-1; FP32 smoother links and site terms; FP32 V-cycle arithmetic"}
        sc.close()
        del bc, zc
        torch.cuda.empty_cache()
    # the smaller configurations, each set up and solved on its own: the oracle's 8^4 lattice (FP64
    # throughout, nu = 3) and the 16^4 lattice (FP32 V-cycle, one Gaussian right-hand side)
    if not args.no_small and world == 1 and args.workload.startswith("32x32x32x64"):
        line["small_configs"] = {name: run_small(name) for name in ("8x8x8x8", "16x16x16x16")}
    # the serving form: Poisson arrivals of 1-12 right-hand-side requests over four resident operators
    if not args.no_serving and world == 1:
        from paper_1303_1377_gb300.serve import run_stream

        sv = run_stream(args.serving_seconds, 1.0, 5, ddamg.PREC_HALF, max_rhs=12)
        line["serving"] = {k: sv[k] for k in ("requests", "solves", "wall_s", "solves_per_s", "latency_p50_s", "latency_p99_s",
                                              "max_rel_residual", "arrival_rate_per_s", "rhs_per_request", "slots", "operators")}
    if rank == 0 and world == 1 and not args.no_cpu:
        n_or, _ = oracle_iterations(args.workload)
        base = OracleBaseline(w, workload_m0(w, "oracle_m0_key")[0], n_or if n_or else max(iters))
        v, info = base.sample(12.0)
        base.close()
        line["cpu_baseline"] = {"value": v, "unit": "solves/s", "cores": base.cores, "kind": "oracle", "sample": info}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
