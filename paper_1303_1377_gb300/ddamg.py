"""Thin ctypes binding of libddamg.so (argument marshalling only).

Every computation runs in the CUDA library; this module converts arrays to
pointers and back.  Arrays may be numpy arrays (host memory: the library copies
through its stream) or torch CUDA tensors (device memory: used in place).
Layouts are those of include/ddamg.h: gauge [V,4,3,3] complex128, spinors
[n_rhs, V, 4, 3] complex128 (complex64 for apply_D_f32), coarse vectors
[n_rhs, n_coarse_sites, 2N] complex128; sites lexicographic, x0 slowest.

Importing this module loads the library and raises if it is missing: there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libddamg.so")

PREC_DOUBLE, PREC_SINGLE, PREC_HALF = 0, 1, 2
OUTER_DW, OUTER_REFINE = 0, 1
SETUP_DDALPHA, SETUP_IDSETUP = 0, 1
SLOT_FREE, SLOT_RUNNING, SLOT_DONE, SLOT_FAILED = 0, 1, 2, 3
OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_NONFINITE, ERR_TIMEOUT, ERR_NOT_READY, ERR_RANK = 0, -1, -2, -3, -4, -5, -6, -7, -8

STATUS = {
    0: "OK",
    -1: "INVALID_ARG",
    -2: "OOM",
    -3: "CUDA",
    -4: "NOT_CONVERGED",
    -5: "NONFINITE",
    -6: "TIMEOUT",
    -7: "NOT_READY",
    -8: "RANK",
}


class DDAMGError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} ({msg})")
        self.status = status


class Lattice(C.Structure):
    _fields_ = [("dims", C.c_int * 4)]


class Params(C.Structure):
    _fields_ = [
        ("n_inv", C.c_int),
        ("n_vec", C.c_int),
        ("block", C.c_int * 4),
        ("coarse_tol", C.c_double),
        ("coarse_restart", C.c_int),
        ("coarse_maxiter", C.c_int),
        ("n_kv", C.c_int),
        ("tol", C.c_double),
        ("max_outer", C.c_int),
        ("nu", C.c_int),
        ("mr_steps", C.c_int),
        ("precision", C.c_int),
        ("rebuild_after_last", C.c_int),
        ("seed", C.c_uint64),
        ("time_limit_s", C.c_double),
        ("outer", C.c_int),
        ("cycle_tol", C.c_double),
        ("setup_update", C.c_int),
        ("smoother_fp16", C.c_int),
        ("setup_group", C.c_int),
        ("n_inv_auto_rhs", C.c_int),
        ("lean", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("iterations", C.c_int),
        ("restarts", C.c_int),
        ("coarse_iterations", C.c_longlong),
        ("vcycles", C.c_int),
        ("rel_residual", C.c_double),
        ("solve_seconds", C.c_double),
        ("coarse_seconds", C.c_double),
        ("status", C.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MLParams(C.Structure):
    """ddamg_ml_params: the third level of the recursion (level-1 blocks, N_1, inner solves)."""

    _fields_ = [
        ("block1", C.c_int * 4),
        ("n_vec1", C.c_int),
        ("nu1", C.c_int),
        ("mr_steps1", C.c_int),
        ("inner", C.c_int),
        ("inner_kv", C.c_int),
        ("inner_tol", C.c_double),
        ("inner_maxiter", C.c_int),
        ("coarse_tol", C.c_double),
        ("coarse_restart", C.c_int),
        ("coarse_maxiter", C.c_int),
        ("n_inv1", C.c_int),
        ("setup_update1", C.c_int),
    ]


class KernelProfile(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_longlong), ("total_ms", C.c_double), ("bytes", C.c_double),
                ("flops", C.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1303_1377_gb300.build`")
    lib = C.CDLL(LIB_PATH)
    P, I, D, LL = C.c_void_p, C.c_int, C.c_double, C.c_longlong
    sig = {
        "ddamg_default_params": (None, [C.POINTER(Params)]),
        "ddamg_error_string": (C.c_char_p, [I]),
        "ddamg_last_error": (C.c_char_p, []),
        "ddamg_setup": (I, [C.POINTER(Lattice), P, D, D, C.POINTER(Params), C.POINTER(P)]),
        "ddamg_create": (I, [C.POINTER(Lattice), P, D, D, C.POINTER(Params), C.POINTER(P)]),
        "ddamg_run_setup": (I, [P, P]),
        "ddamg_setup_from_vectors": (I, [P, P, I]),
        "ddamg_get_vectors": (I, [P, P]),
        "ddamg_setup_report": (I, [P, C.POINTER(C.c_int), C.POINTER(C.c_double), I]),
        "ddamg_solve": (I, [P, P, P, D, C.POINTER(Stats)]),
        "ddamg_solve_batch": (I, [P, P, P, I, D, C.POINTER(Stats)]),
        "ddamg_solve_batch_zero_guess": (I, [P, P, P, I, D, C.POINTER(Stats)]),
        "ddamg_apply_D": (I, [P, P, P, I]),
        "ddamg_apply_D_f32": (I, [P, P, P, I]),
        "ddamg_apply_D_mixed": (I, [P, P, P, I]),
        "ddamg_apply_sap": (I, [P, P, P, I, I]),
        "ddamg_restrict": (I, [P, P, P, I]),
        "ddamg_prolong": (I, [P, P, P, I]),
        "ddamg_apply_Dc": (I, [P, P, P, I]),
        "ddamg_apply_Dc_noalloc": (I, [P, P, P, I]),
        "ddamg_get_coarse_stencil": (I, [P, P]),
        "ddamg_coarse_solve": (I, [P, P, P, I, I]),
        "ddamg_vcycle": (I, [P, P, P, I, I]),
        "ddamg_set_mass": (I, [P, D]),
        "ddamg_set_stream": (I, [P, P]),
        "ddamg_info": (I, [P, C.POINTER(LL), C.POINTER(LL), C.POINTER(I)]),
        "ddamg_profile_enable": (I, [P, I]),
        "ddamg_profile_read": (I, [P, C.POINTER(KernelProfile), I]),
        "ddamg_profile_reset": (I, [P]),
        "ddamg_profile_families": (I, [C.c_char_p, I]),
        "ddamg_launch_count": (LL, []),
        "ddamg_debug_fail_allocs": (None, [I]),
        "ddamg_slots_open": (I, [P, I]),
        "ddamg_slot_put": (I, [P, I, P]),
        "ddamg_slots_cycle": (I, [P, C.POINTER(I), C.POINTER(Stats)]),
        "ddamg_slot_take": (I, [P, I, P]),
        "ddamg_slots_close": (I, [P]),
        "ddamg_ml_default_params": (None, [C.POINTER(MLParams)]),
        "ddamg_ml_build": (I, [P, C.POINTER(MLParams), P]),
        "ddamg_ml_setup": (I, [P, C.POINTER(MLParams), P, P]),
        "ddamg_ml_add_level": (I, [P, C.POINTER(MLParams), P, I, P]),
        "ddamg_ml_levels": (I, [P]),
        "ddamg_ml_release": (I, [P]),
        "ddamg_ml_apply_sap1": (I, [P, P, P, I, I]),
        "ddamg_ml_restrict1": (I, [P, P, P, I]),
        "ddamg_ml_prolong1": (I, [P, P, P, I]),
        "ddamg_ml_apply_D2": (I, [P, P, P, I]),
        "ddamg_ml_vcycle1": (I, [P, P, P, I]),
        "ddamg_ml_vcycle": (I, [P, P, P, I, I]),
        "ddamg_ml_solve": (I, [P, P, P, I, D, C.POINTER(Stats)]),
        "ddamg_ml_solve_zero_guess": (I, [P, P, P, I, D, C.POINTER(Stats)]),
        "ddamg_ml_counts": (I, [P, C.POINTER(LL)]),
        "ddamg_destroy": (I, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def default_params(**kw) -> Params:
    p = Params()
    lib.ddamg_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "block":
            for m in range(4):
                p.block[m] = int(v[m])
        else:
            setattr(p, k, v)
    return p


def ml_default_params(**kw) -> MLParams:
    p = MLParams()
    lib.ddamg_ml_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "block1":
            for m in range(4):
                p.block1[m] = int(v[m])
        else:
            setattr(p, k, v)
    return p


def _check(rc: int, where: str, allow=()):
    if rc != 0 and rc not in allow:
        raise DDAMGError(rc, where, lib.ddamg_last_error().decode(errors="replace"))
    return rc


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if a.is_cuda:
            # the library works on its own stream: work that torch has queued on the tensor (on torch's
            # current stream) must be complete before the library reads or writes it
            import torch

            torch.cuda.current_stream(a.device).synchronize()
        return C.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return C.c_void_p(a.ctypes.data)


def _host(a, dtype):
    if _is_torch(a):
        return a
    return np.ascontiguousarray(a, dtype=dtype)


def _empty_like(a, shape, dtype):
    if _is_torch(a):
        import torch

        tdt = {np.complex128: torch.complex128, np.complex64: torch.complex64}[dtype]
        return torch.empty(shape, dtype=tdt, device=a.device)
    return np.empty(shape, dtype=dtype)


class Solver:
    """A DD-alpha-AMG operator D(U, m0, c_sw) with its two-level preconditioner."""

    def __init__(self, dims, U, m0: float, c_sw: float, params: Params | None = None, setup: bool = True, v0=None):
        self.dims = tuple(int(d) for d in dims)
        self.params = params if params is not None else default_params()
        lat = Lattice((C.c_int * 4)(*self.dims))
        U = _host(U, np.complex128)
        h = C.c_void_p()
        _check(lib.ddamg_create(C.byref(lat), _ptr(U), float(m0), float(c_sw), C.byref(self.params), C.byref(h)), "ddamg_create")
        self.h = h
        n, nc, dof = C.c_longlong(), C.c_longlong(), C.c_int()
        lib.ddamg_info(self.h, C.byref(n), C.byref(nc), C.byref(dof))
        self.V, self.n_coarse, self.coarse_dof = n.value, nc.value, dof.value
        if setup:
            self.run_setup(v0)

    # -- lifecycle --------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            lib.ddamg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- setup ------------------------------------------------------------------
    def run_setup(self, v0=None):
        p = C.c_void_p() if v0 is None else _ptr(_host(v0, np.complex128))
        _check(lib.ddamg_run_setup(self.h, p), "ddamg_run_setup")

    def setup_from_vectors(self, V):
        V = _host(V, np.complex128)
        _check(lib.ddamg_setup_from_vectors(self.h, _ptr(V), int(V.shape[0])), "ddamg_setup_from_vectors")

    def vectors(self):
        out = np.empty((self.params.n_vec, self.V, 4, 3), dtype=np.complex128)
        _check(lib.ddamg_get_vectors(self.h, _ptr(out)), "ddamg_get_vectors")
        return out

    def setup_report(self):
        """(update rounds of the last setup, estimated iterations per solve before each round when
        params.n_inv_auto_rhs balanced it)."""
        rounds = C.c_int(0)
        est = (C.c_double * 64)()
        n = lib.ddamg_setup_report(self.h, C.byref(rounds), est, 64)
        if n < 0:
            _check(n, "ddamg_setup_report")
        return rounds.value, [est[k] for k in range(min(n, 64))]

    def set_mass(self, m0: float):
        _check(lib.ddamg_set_mass(self.h, float(m0)), "ddamg_set_mass")

    def set_stream(self, stream_ptr: int | None):
        _check(lib.ddamg_set_stream(self.h, C.c_void_p(stream_ptr or 0)), "ddamg_set_stream")

    # -- solves -----------------------------------------------------------------
    def solve(self, b, z=None, tol: float = 0.0, allow_fail: bool = False):
        """Solve D z = b for a batch b[n_rhs, V, 4, 3] (or one field [V, 4, 3])."""
        b = _host(b, np.complex128)
        single = b.ndim == 3
        nr = 1 if single else int(b.shape[0])
        if z is None:
            z = _empty_like(b, b.shape, np.complex128)
            z[...] = 0
        st = (Stats * nr)()
        rc = lib.ddamg_solve_batch(self.h, _ptr(b), _ptr(z), nr, float(tol), st)
        _check(rc, "ddamg_solve_batch", allow=(-4, -5, -6) if allow_fail else ())
        return z, [s.as_dict() for s in st], rc

    def solve_zero_guess(self, b, z=None, tol: float = 0.0, allow_fail: bool = False):
        """Solve D z = b from the zero initial guess; z (optional) is output only and never read."""
        b = _host(b, np.complex128)
        nr = 1 if b.ndim == 3 else int(b.shape[0])
        if z is None:
            z = _empty_like(b, b.shape, np.complex128)
        st = (Stats * nr)()
        rc = lib.ddamg_solve_batch_zero_guess(self.h, _ptr(b), _ptr(z), nr, float(tol), st)
        _check(rc, "ddamg_solve_batch_zero_guess", allow=(-4, -5, -6) if allow_fail else ())
        return z, [s.as_dict() for s in st], rc

    # -- recursion to a third level ------------------------------------------------
    def ml_build(self, v1, params: MLParams | None = None):
        """Level 2 from the level-1 test vectors v1[N1, coarse sites, 2N] (coarse layout)."""
        self.ml_params = params if params is not None else ml_default_params()
        v1 = _host(v1, np.complex128)
        _check(lib.ddamg_ml_build(self.h, C.byref(self.ml_params), _ptr(v1)), "ddamg_ml_build")
        nb1 = [self.coarse_dims()[m] // self.ml_params.block1[m] for m in range(4)]
        self.n_level2 = int(np.prod(nb1))
        self.level2_dof = 2 * self.ml_params.n_vec1

    def ml_setup(self, v0, params: MLParams | None = None):
        """Level 2 by the adaptive setup on level 1 from the initial vectors v0[N1, coarse sites, 2N];
        returns the final level-1 test vectors."""
        self.ml_params = params if params is not None else ml_default_params()
        v0 = _host(v0, np.complex128)
        out = np.empty_like(v0) if not _is_torch(v0) else _empty_like(v0, tuple(v0.shape), np.complex128)
        _check(lib.ddamg_ml_setup(self.h, C.byref(self.ml_params), _ptr(v0), _ptr(out)), "ddamg_ml_setup")
        nb1 = [self.coarse_dims()[m] // self.ml_params.block1[m] for m in range(4)]
        self.n_level2 = int(np.prod(nb1))
        self.level2_dof = 2 * self.ml_params.n_vec1
        return out

    def ml_add_level(self, v, params: MLParams, setup: bool = True):
        """One more level below the current coarsest one; v[N, its sites, its components] are the
        initial vectors of its adaptive setup (setup=True) or the vectors themselves.  Returns the
        final vectors."""
        v = _host(v, np.complex128)
        out = np.empty_like(v) if not _is_torch(v) else _empty_like(v, tuple(v.shape), np.complex128)
        _check(lib.ddamg_ml_add_level(self.h, C.byref(params), _ptr(v), int(bool(setup)), _ptr(out)), "ddamg_ml_add_level")
        return out

    def ml_levels(self) -> int:
        return int(lib.ddamg_ml_levels(self.h))

    def coarse_dims(self):
        return tuple(self.dims[m] // self.params.block[m] for m in range(4))

    def ml_release(self):
        _check(lib.ddamg_ml_release(self.h), "ddamg_ml_release")

    def _ml_op(self, fn, x, out_shape, *extra):
        x = _host(x, np.complex128)
        nr = int(x.shape[0])
        out = _empty_like(x, (nr,) + tuple(out_shape), np.complex128)
        _check(fn(self.h, _ptr(x), _ptr(out), nr, *extra), fn.__name__)
        return out

    def ml_apply_sap1(self, x, nu: int):
        return self._ml_op(lib.ddamg_ml_apply_sap1, x, (self.n_coarse, self.coarse_dof), int(nu))

    def ml_restrict1(self, x):
        return self._ml_op(lib.ddamg_ml_restrict1, x, (self.n_level2, self.level2_dof))

    def ml_prolong1(self, e):
        return self._ml_op(lib.ddamg_ml_prolong1, e, (self.n_coarse, self.coarse_dof))

    def ml_apply_D2(self, e):
        return self._ml_op(lib.ddamg_ml_apply_D2, e, (self.n_level2, self.level2_dof))

    def ml_vcycle1(self, x):
        return self._ml_op(lib.ddamg_ml_vcycle1, x, (self.n_coarse, self.coarse_dof))

    def ml_vcycle(self, r, inner_fixed_iters: int = 0):
        return self._ml_op(lib.ddamg_ml_vcycle, r, (self.V, 4, 3), int(inner_fixed_iters))

    def ml_solve(self, b, z=None, tol: float = 0.0, allow_fail: bool = False):
        """Three-level solve of D z = b for b[n_rhs, V, 4, 3] (the outer scheme of the handle's
        precision, as solve; z is the initial guess, zero when not given)."""
        b = _host(b, np.complex128)
        nr = int(b.shape[0])
        if z is None:
            z = _empty_like(b, b.shape, np.complex128)
            z[...] = 0
        st = (Stats * nr)()
        rc = lib.ddamg_ml_solve(self.h, _ptr(b), _ptr(z), nr, float(tol), st)
        _check(rc, "ddamg_ml_solve", allow=(-4, -5, -6) if allow_fail else ())
        return z, [s.as_dict() for s in st], rc

    def ml_solve_zero_guess(self, b, z=None, tol: float = 0.0, allow_fail: bool = False):
        """Three-level solve from the zero initial guess; z (optional) is output only."""
        b = _host(b, np.complex128)
        nr = int(b.shape[0])
        if z is None:
            z = _empty_like(b, b.shape, np.complex128)
        st = (Stats * nr)()
        rc = lib.ddamg_ml_solve_zero_guess(self.h, _ptr(b), _ptr(z), nr, float(tol), st)
        _check(rc, "ddamg_ml_solve_zero_guess", allow=(-4, -5, -6) if allow_fail else ())
        return z, [s.as_dict() for s in st], rc

    def ml_counts(self):
        """Counters of the last ml_solve."""
        cnt = (C.c_longlong * 3)()
        _check(lib.ddamg_ml_counts(self.h, cnt), "ddamg_ml_counts")
        return {"fgmres_steps_D1": cnt[0], "gmres_steps_D2": cnt[1], "vcycles1": cnt[2]}

    # -- continuous batching ------------------------------------------------------
    def slots_open(self, n_slots: int):
        _check(lib.ddamg_slots_open(self.h, int(n_slots)), "ddamg_slots_open")
        self.n_slots = int(n_slots)

    def slot_put(self, slot: int, b):
        """Admit one right-hand side b[V, 4, 3] into a free slot (initial guess 0)."""
        b = _host(b, np.complex128)
        _check(lib.ddamg_slot_put(self.h, int(slot), _ptr(b)), "ddamg_slot_put")

    def slots_cycle(self):
        """One outer cycle over the running slots; returns (states[n_slots], stats)."""
        states = (C.c_int * self.n_slots)()
        st = (Stats * self.n_slots)()
        _check(lib.ddamg_slots_cycle(self.h, states, st), "ddamg_slots_cycle")
        return list(states), [x.as_dict() for x in st]

    def slot_take(self, slot: int, out=None):
        """The solution of a finished slot, which becomes free."""
        z = out if out is not None else np.empty((self.V, 4, 3), dtype=np.complex128)
        _check(lib.ddamg_slot_take(self.h, int(slot), _ptr(z)), "ddamg_slot_take")
        return z

    def slots_close(self):
        _check(lib.ddamg_slots_close(self.h), "ddamg_slots_close")
        self.n_slots = 0

    # -- operator pieces --------------------------------------------------------
    def _fine_op(self, fn, x, *extra, dtype=np.complex128):
        x = _host(x, dtype)
        nr = 1 if x.ndim == 3 else int(x.shape[0])
        out = _empty_like(x, x.shape, dtype)
        _check(fn(self.h, _ptr(x), _ptr(out), nr, *extra), fn.__name__)
        return out

    def apply_D(self, x):
        return self._fine_op(lib.ddamg_apply_D, x)

    def apply_D_f32(self, x):
        return self._fine_op(lib.ddamg_apply_D_f32, x, dtype=np.complex64)

    def apply_D_mixed(self, x):
        """D x for a complex64 field, complex128 result (double-word FP32 arithmetic)."""
        x = _host(x, np.complex64)
        nr = 1 if x.ndim == 3 else int(x.shape[0])
        out = _empty_like(x, x.shape, np.complex128)
        _check(lib.ddamg_apply_D_mixed(self.h, _ptr(x), _ptr(out), nr), "ddamg_apply_D_mixed")
        return out

    def apply_sap(self, x, nu: int):
        return self._fine_op(lib.ddamg_apply_sap, x, int(nu))

    def vcycle(self, r, coarse_fixed_iters: int = 0):
        return self._fine_op(lib.ddamg_vcycle, r, int(coarse_fixed_iters))

    def restrict(self, x):
        x = _host(x, np.complex128)
        nr = 1 if x.ndim == 3 else int(x.shape[0])
        out = _empty_like(x, (nr, self.n_coarse, self.coarse_dof), np.complex128)
        _check(lib.ddamg_restrict(self.h, _ptr(x), _ptr(out), nr), "ddamg_restrict")
        return out[0] if x.ndim == 3 else out

    def prolong(self, e):
        e = _host(e, np.complex128)
        nr = 1 if e.ndim == 2 else int(e.shape[0])
        out = _empty_like(e, (nr, self.V, 4, 3), np.complex128)
        _check(lib.ddamg_prolong(self.h, _ptr(e), _ptr(out), nr), "ddamg_prolong")
        return out[0] if e.ndim == 2 else out

    def _coarse_op(self, fn, e, *extra):
        e = _host(e, np.complex128)
        nr = 1 if e.ndim == 2 else int(e.shape[0])
        out = _empty_like(e, e.shape, np.complex128)
        _check(fn(self.h, _ptr(e), _ptr(out), nr, *extra), fn.__name__)
        return out

    def apply_Dc(self, e):
        return self._coarse_op(lib.ddamg_apply_Dc, e)

    def apply_Dc_noalloc(self, e_dev, out_dev):
        """D_c e without any allocation in the library: e_dev, out_dev are contiguous CUDA tensors of
        dtype complex128 and equal shape [n_rhs, n_coarse, 2N] (or [n_coarse, 2N]) on one device;
        the library's fixed scratch array is used.  The call is ordered on the handle's stream and
        does not wait for it."""
        import torch

        for name, t in (("e_dev", e_dev), ("out_dev", out_dev)):
            if not isinstance(t, torch.Tensor) or not t.is_cuda:
                raise ValueError(f"apply_Dc_noalloc: {name} must be a CUDA tensor")
            if t.dtype != torch.complex128:
                raise ValueError(f"apply_Dc_noalloc: {name} must be complex128, got {t.dtype}")
            if t.ndim not in (2, 3) or tuple(t.shape[-2:]) != (self.n_coarse, self.coarse_dof):
                raise ValueError(f"apply_Dc_noalloc: {name} must have shape [n_rhs, {self.n_coarse}, {self.coarse_dof}], "
                                 f"got {tuple(t.shape)}")
            if not t.is_contiguous():
                raise ValueError(f"apply_Dc_noalloc: {name} must be contiguous")
        if tuple(out_dev.shape) != tuple(e_dev.shape):
            raise ValueError(f"apply_Dc_noalloc: out_dev shape {tuple(out_dev.shape)} differs from e_dev {tuple(e_dev.shape)}")
        if out_dev.device != e_dev.device:
            raise ValueError("apply_Dc_noalloc: e_dev and out_dev are on different devices")
        nr = 1 if e_dev.ndim == 2 else int(e_dev.shape[0])
        return _check(lib.ddamg_apply_Dc_noalloc(self.h, _ptr(e_dev), _ptr(out_dev), nr), "ddamg_apply_Dc_noalloc")

    def coarse_solve(self, e, fixed_iters: int = 0):
        return self._coarse_op(lib.ddamg_coarse_solve, e, int(fixed_iters))

    def coarse_stencil(self):
        out = np.empty((self.n_coarse, 9, self.coarse_dof, self.coarse_dof), dtype=np.complex128)
        _check(lib.ddamg_get_coarse_stencil(self.h, _ptr(out)), "ddamg_get_coarse_stencil")
        return out

    # -- profiling ----------------------------------------------------------------
    def profile(self, families=None):
        """Record the named kernel families (None: all; [] : off)."""
        if families is None:
            mask = -1
        else:
            names = profile_families()
            mask = 0
            for f in families:
                mask |= 1 << names.index(f)
        lib.ddamg_profile_enable(self.h, mask)

    def profile_reset(self):
        lib.ddamg_profile_reset(self.h)

    def profile_read(self):
        arr = (KernelProfile * 16)()
        n = lib.ddamg_profile_read(self.h, arr, 16)
        return {arr[i].name.decode(): {"launches": arr[i].launches, "total_ms": arr[i].total_ms, "bytes": arr[i].bytes,
                                       "flops": arr[i].flops} for i in range(min(n, 16))}


def profile_families():
    buf = C.create_string_buffer(256)
    lib.ddamg_profile_families(buf, 256)
    return buf.value.decode().split(",")


def launch_count() -> int:
    return int(lib.ddamg_launch_count())


def debug_fail_allocs(n: int):
    lib.ddamg_debug_fail_allocs(int(n))
