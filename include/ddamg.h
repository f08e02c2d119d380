/*
 * ddamg.h - C ABI of libddamg.so, a GB300 (sm_103a) implementation of the
 * two-level DD-alpha-AMG solver for the clover-improved Wilson Dirac equation
 * D z = b (Frommer, Kahl, Krieg, Leder, Rottmann, arXiv:1303.1377).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice: periodic L0 x L1 x L2 x L3 (L0 = time), sites in lexicographic order
 *   with x0 slowest and x3 fastest (Sec. 2.2).
 * Complex numbers: interleaved (re, im) pairs of double (or float where stated).
 * Gauge field U: [site][mu 0..3][row 0..2][col 0..2] complex, U_mu(x) in SU(3)
 *   on the link from x to x + mu (Sec. 2.2).
 * Spinor field: [site][spin 0..3][colour 0..2] complex, 12 components per site,
 *   colour fastest (Sec. 2.1).  A batch of n_rhs spinors is n_rhs such fields
 *   back to back.
 * Coarse vector: [coarse site][2N] complex, coarse sites = lattice-blocks in
 *   lexicographic order of their block coordinates; component h*N + k is the
 *   k-th basis vector of the aggregate with spins {0,1} (h = 0) or {2,3} (h = 1)
 *   (standard aggregation, Sec. 3.2, Definition).
 * Pointers: every data pointer may be host or device memory (CUDA unified
 *   addressing decides).  Host data is copied through the handle's stream;
 *   device data must be readable/writable on the handle's device.  The caller
 *   keeps ownership of everything it passes; the handle owns all its device state.
 * Errors: every call returns a ddamg_status (0 = success, negative = error) and
 *   never throws.  ddamg_error_string() names a status; ddamg_last_error()
 *   gives a one-line description of the most recent failure on this thread.
 * Threads/streams: a handle is not thread safe; all its work is issued on its
 *   stream (ddamg_set_stream), and every call returns after that work has
 *   completed unless stated otherwise.
 */
#ifndef DDAMG_H
#define DDAMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DDAMG_OK = 0,
    DDAMG_ERR_INVALID_ARG = -1,   /* bad size, layout, null pointer or parameter */
    DDAMG_ERR_OOM = -2,           /* device allocation failed (or the test hook forced it) */
    DDAMG_ERR_CUDA = -3,          /* a CUDA runtime call or kernel launch failed */
    DDAMG_ERR_NOT_CONVERGED = -4, /* iteration cap reached; z holds the best iterate */
    DDAMG_ERR_NONFINITE = -5,     /* NaN/Inf met in a residual norm */
    DDAMG_ERR_TIMEOUT = -6,       /* wall-clock limit of the call exceeded */
    DDAMG_ERR_NOT_READY = -7,     /* the handle has no interpolation yet (setup missing) */
    DDAMG_ERR_RANK = -8           /* test vectors linearly dependent on an aggregate */
} ddamg_status;

/* Arithmetic of the V-cycle (smoother, P/P^H, coarse solve).  The final residual
 * and the iterate are FP64 in every mode; the outer FGMRES is FP64 in DOUBLE mode
 * and follows ddamg_outer in SINGLE and HALF mode (Sec. 6 runs the preconditioner
 * in single precision inside a double-precision FGMRES). */
typedef enum {
    DDAMG_PREC_DOUBLE = 0, /* V-cycle in FP64 */
    DDAMG_PREC_SINGLE = 1, /* V-cycle in FP32 (the paper's mixed precision, Sec. 6) */
    DDAMG_PREC_HALF = 2    /* V-cycle in FP32 with D_c and P stored in FP16 (FP32 accumulation); on
                              4^4 blocks the smoother also reads FP16 copies of the links and site terms */
} ddamg_precision;

/* Outer iteration of SINGLE and HALF mode (no counterpart in the paper, which
 * keeps the whole FGMRES in FP64; FP64 arithmetic runs at about 1/60 of FP32 on
 * this GPU).  Both certify the result with the true residual b - D z, accurate to
 * about 2^-48 relative to |D| |z|. */
typedef enum {
    DDAMG_OUTER_DW = 0,    /* one FGMRES(n_kv): double-word (~48-bit) Arnoldi basis and products D z,
                              FP64 iterate; true FP64 residual at every restart */
    DDAMG_OUTER_REFINE = 1 /* FGMRES cycles in FP32 (basis, D z, Gram-Schmidt), each ended once every
                              right-hand side has reduced its residual by cycle_tol (or after n_kv
                              steps); between cycles the FP64 iterate is updated and the true
                              residual b - D z starts the next cycle.  Here D z is formed without
                              FP64 arithmetic: z = z_h + z_l (an FP32 pair, ~2^-48 relative),
                              D z_h in double-word arithmetic, D z_l in FP32, b - D z in FP64 */
} ddamg_outer;

/* Test-vector update in the second phase of the adaptive setup (Sec. 5): after P and
 * D_c are rebuilt from v_1..v_N, every v_j is updated and normalised. */
typedef enum {
    DDAMG_SETUP_DDALPHA = 0, /* Algorithm 2 (DD-alphaAMG setup): v_j <- v_j + C (v_j - D v_j), one V-cycle
                                iteration on D v = v_j started from v_j */
    DDAMG_SETUP_IDSETUP = 1  /* Algorithm 1 (inexact-deflation setup): v_j <- C v_j, the same iteration
                                started from 0 */
} ddamg_setup_update;

typedef struct {
    int dims[4]; /* L0 (time), L1, L2, L3 */
} ddamg_lattice;

/* Method parameters; ddamg_default_params() fills the defaults of Table 1 (Sec. 6). */
typedef struct {
    int n_inv;            /* setup iterations of Algorithm 2 (6) */
    int n_vec;            /* test vectors N (20) */
    int block[4];         /* lattice-block of both the SAP domains and the aggregates (4,4,4,4) */
    double coarse_tol;    /* relative residual reduction of the coarse solve (5e-2) */
    int coarse_restart;   /* GMRES restart length on the coarse system (30, Sec. 6; at most 64) */
    int coarse_maxiter;   /* cap on coarse GMRES steps per coarse solve (1000) */
    int n_kv;             /* FGMRES restart length (25; at most 64) */
    double tol;           /* outer relative residual tolerance (1e-10) */
    int max_outer;        /* cap on FGMRES iterations per solve (10000) */
    int nu;               /* SAP post-smoothing iterations (2) */
    int mr_steps;         /* MR steps of the block solver (4) */
    int precision;        /* ddamg_precision (DDAMG_PREC_SINGLE) */
    int rebuild_after_last; /* 1: rebuild P, D_c after the last setup update (1) */
    uint64_t seed;        /* seed of the initial random test vectors (1) */
    double time_limit_s;  /* wall-clock limit per solve call (ddamg_solve, ddamg_solve_batch,
                             ddamg_solve_batch_zero_guess, ddamg_ml_solve), <= 0: none (0).
                             Checked on the host at every synchronisation of the outer
                             iteration (each FGMRES step); once passed, z takes the current
                             cycle's update and the call returns DDAMG_ERR_TIMEOUT with
                             st[r].rel_residual the last residual estimate. */
    int outer;            /* ddamg_outer of SINGLE and HALF mode (DDAMG_OUTER_REFINE) */
    double cycle_tol;     /* residual reduction of one FP32 cycle of DDAMG_OUTER_REFINE, in (0, 1) (1e-5) */
    int setup_update;     /* ddamg_setup_update: test-vector update of the setup's second phase
                             (DDAMG_SETUP_DDALPHA) */
    int smoother_fp16;    /* DDAMG_PREC_HALF only: 1 = the SAP smoother reads FP16 copies of the
                             links and site terms (FP32 arithmetic); 0 = FP32 copies, so that only
                             P, D_c and its inverses are stored in FP16 (1) */
    int setup_group;      /* the setup updates the test vectors in groups of this many (the
                             updates of one setup round are independent), bounding its work
                             fields to 2 * setup_group fine fields; <= 0: all n_vec at once (0) */
    int n_inv_auto_rhs;   /* > 0: balance the setup against this many right-hand sides (Sec. 6.2,
                             Table 4: more setup pays off over more solves).  n_inv becomes a cap;
                             before every setup round after the first, four FGMRES iterations on
                             a fixed random right-hand side estimate the iterations per solve,
                             and the setup stops once the last round saved less solve time over
                             n_inv_auto_rhs solves than it cost (0: n_inv rounds) */
    int lean;             /* DDAMG_PREC_SINGLE / HALF: 1 = after each setup free the FP64 test
                             vectors and FP64 interpolation (only the setup and ddamg_get_vectors
                             use them; the V-cycle reads its FP32 / FP16 copies): 2 * n_vec FP64
                             fields; ddamg_get_vectors then returns DDAMG_ERR_NOT_READY (0) */
} ddamg_params;

/* Statistics of one solve (the quantities reported in Tables 3-9). */
typedef struct {
    int iterations;        /* FGMRES iterations (max over the batch) */
    int restarts;          /* FGMRES restarts */
    long long coarse_iterations; /* total coarse GMRES steps */
    int vcycles;           /* preconditioner applications */
    double rel_residual;   /* final ||b - D z|| / ||b|| in FP64 (max over the batch) */
    double solve_seconds;  /* wall time of the call */
    double coarse_seconds; /* part of it spent in the coarse solves */
    int status;            /* ddamg_status of this solve */
} ddamg_stats;

typedef struct ddamg_handle ddamg_handle;

void ddamg_default_params(ddamg_params* p);
const char* ddamg_error_string(int status);
const char* ddamg_last_error(void);

/* Build the operator D(U, m0, c_sw) of Sec. 2.2 (clover term and even-site
 * inverses are formed here) and run the adaptive setup of Algorithm 2 (Sec. 5)
 * from N seeded random test vectors, leaving P and D_c = P^H D P ready.
 * lat: every extent divisible by params->block, with an even number (>= 2) of
 *   blocks per direction and even block extents; N <= 64.
 * U: gauge field (layout above), copied.  *out receives a new handle.
 * Errors: INVALID_ARG, OOM, CUDA, RANK. */
int ddamg_setup(const ddamg_lattice* lat, const double* U, double m0, double c_sw,
                const ddamg_params* params, ddamg_handle** out);

/* Like ddamg_setup but without the adaptive setup: only D is built.
 * Interpolation comes later from ddamg_setup_from_vectors or ddamg_run_setup. */
int ddamg_create(const ddamg_lattice* lat, const double* U, double m0, double c_sw,
                 const ddamg_params* params, ddamg_handle** out);

/* Run Algorithm 2 (Sec. 5) on the handle from the given initial vectors
 * v0 [N spinor fields] (NULL: seeded Gaussian vectors from params->seed). */
int ddamg_run_setup(ddamg_handle* h, const double* v0);

/* Build P (local orthonormalisation, Sec. 3.1) and D_c (Sec. 3.2) directly from
 * N given test vectors V [N spinor fields]; N must equal params->n_vec. */
int ddamg_setup_from_vectors(ddamg_handle* h, const double* V, int N);

/* Copy the current test vectors (N spinor fields, FP64) into V. */
int ddamg_get_vectors(const ddamg_handle* h, double* V);

/* The last adaptive setup of the handle: *rounds = update rounds run (n_inv, or fewer when
 * params.n_inv_auto_rhs stopped it, Sec. 6.2 / Table 4); est_iterations[k] (k < max) = the
 * estimated FGMRES iterations per solve of the probe before round k (n_inv_auto_rhs > 0 only).
 * Returns the number of probes (>= 0), or DDAMG_ERR_INVALID_ARG for a null handle or rounds. */
int ddamg_setup_report(const ddamg_handle* h, int* rounds, double* est_iterations, int max);

/* Solve D z = b to ||b - D z|| <= tol ||b|| by FGMRES(n_kv) right-preconditioned
 * with one V-cycle (Sec. 5); in SINGLE and HALF mode the FGMRES runs as the
 * params->outer scheme (ddamg_outer).  b, z: one spinor field each; z is the
 * initial guess on entry (pass zeros for the paper's zero guess; an all-zero z
 * skips the initial residual product) and the solution on exit.  The
 * convergence test is always on the true residual.  tol <= 0 uses params->tol.
 * st may be NULL.
 * Errors: INVALID_ARG, NOT_READY, OOM, CUDA, NOT_CONVERGED (z = last iterate),
 * NONFINITE, TIMEOUT. */
int ddamg_solve(ddamg_handle* h, const double* b, double* z, double tol, ddamg_stats* st);

/* n_rhs independent solves in one batched launch sequence (multi-RHS kernels):
 * b, z: n_rhs spinor fields each.  Each right-hand side keeps its own Krylov
 * space and stops at its own convergence; st (may be NULL) points to n_rhs stats. */
int ddamg_solve_batch(ddamg_handle* h, const double* b, double* z, int n_rhs, double tol,
                      ddamg_stats* st);

/* ddamg_solve_batch from the zero initial guess of Sec. 6 with z output only: z is
 * neither read nor copied to the device (for host buffers this saves one field
 * upload per right-hand side), and no initial residual product is formed.  Same
 * arguments, statistics and errors as ddamg_solve_batch. */
int ddamg_solve_batch_zero_guess(ddamg_handle* h, const double* b, double* z, int n_rhs, double tol,
                                 ddamg_stats* st);

/* Continuous batching (no counterpart in the paper).  A handle keeps up to n_slots
 * right-hand sides in flight.  ddamg_slots_cycle runs one outer cycle (one FGMRES cycle
 * of the handle's outer scheme, on all running slots in lock step); between calls the
 * host admits right-hand sides into free slots and takes finished ones out, so a new
 * request waits at most one cycle, not for a whole batch.  A slot is finished (DONE) when
 * the true residual at the start of a cycle meets tol * ||b|| (params.tol); FAILED means a
 * non-finite value or max_outer iterations.  Slot storage: 2 * n_slots FP64 fields on the
 * device, owned by the handle (freed by ddamg_slots_close or ddamg_destroy).  All calls
 * run on the handle's stream and return after it has synchronised; b and z may be host
 * or device pointers in the layout of ddamg_solve. */
typedef enum {
    DDAMG_SLOT_FREE = 0,
    DDAMG_SLOT_RUNNING = 1,
    DDAMG_SLOT_DONE = 2,
    DDAMG_SLOT_FAILED = 3
} ddamg_slot_state;
int ddamg_slots_open(ddamg_handle* h, int n_slots);            /* needs a setup; drops open slots */
int ddamg_slot_put(ddamg_handle* h, int slot, const double* b);  /* slot must be FREE; z starts at 0 */
int ddamg_slots_cycle(ddamg_handle* h, int* state, ddamg_stats* st); /* state[n_slots], st[n_slots] out, either may be NULL */
int ddamg_slot_take(ddamg_handle* h, int slot, double* z);       /* slot DONE or FAILED -> FREE */
int ddamg_slots_close(ddamg_handle* h);

/* out = D in (Sec. 2.2, FP64) for n_rhs spinor fields. */
int ddamg_apply_D(ddamg_handle* h, const double* in, double* out, int n_rhs);

/* out = D in in FP32 arithmetic on FP32 fields ([site][spin][colour] complex float). */
int ddamg_apply_D_f32(ddamg_handle* h, const float* in, float* out, int n_rhs);

/* out = D in for an FP32 field in ([site][spin][colour] complex float) with an
 * FP64 result accurate to ~1e-14 relative: the operator is applied in
 * double-word FP32 arithmetic (how FGMRES multiplies D with the FP32 V-cycle
 * output).  Needs a single- or half-precision handle. */
int ddamg_apply_D_mixed(ddamg_handle* h, const float* in, double* out, int n_rhs);

/* out = M_SAP^(nu) in (Sec. 2.3) in the V-cycle precision; FP64 fields in/out.  In
 * DDAMG_PREC_HALF on 4^4 blocks the links and site terms are read from FP16 copies (FP32
 * arithmetic): the result then differs from the FP64 operator's by the FP16 storage error,
 * a few 1e-4 relative to the field's maximum. */
int ddamg_apply_sap(ddamg_handle* h, const double* in, double* out, int n_rhs, int nu);

/* Coarse restriction out = P^H in (fine -> coarse) and prolongation out = P in
 * (coarse -> fine), Sec. 3.1; FP64 fields, V-cycle precision arithmetic.  In
 * DDAMG_PREC_HALF both are FP16 tensor-core products with FP32 accumulation: P is
 * stored in FP16, and the FP32 operand is rounded to FP16 after a power-of-two
 * scaling (per aggregate for the coarse input of the prolongation; by the field
 * maximum of each right-hand side for the restriction), about 2^-12 relative
 * error per entry.  n_rhs < 1 or a null pointer: DDAMG_ERR_INVALID_ARG. */
int ddamg_restrict(ddamg_handle* h, const double* fine_in, double* coarse_out, int n_rhs);
int ddamg_prolong(ddamg_handle* h, const double* coarse_in, double* fine_out, int n_rhs);

/* out = D_c in for coarse vectors (Sec. 3.2), V-cycle precision arithmetic (in
 * DDAMG_PREC_HALF: D_c stored in FP16, FP16 tensor-core products, FP32 accumulation). */
int ddamg_apply_Dc(ddamg_handle* h, const double* in, double* out, int n_rhs);

/* out = D_c in, like ddamg_apply_Dc, for callers that must not have this library
 * allocate device memory during the call: a code whose memory pool already owns
 * almost all of the GPU (PyTorch's caching allocator, a serving process with a
 * fixed budget), or a latency-critical loop that cannot pay the implicit device
 * synchronisation of cudaMalloc/cudaFree.  The paper has no counterpart; this is
 * a deployment variant of the coarse-operator application.
 * in, out: DEVICE pointers (coarse-vector layout above, n_rhs vectors, FP64);
 *   host pointers are rejected with DDAMG_ERR_INVALID_ARG.
 * Working memory: a fixed 16 MiB device array inside the library (every GPU that
 *   loads the library holds it until the process exits).  n_rhs is limited to
 *   16 MiB / (2 * coarse sites * 2N * bytes per complex number of the V-cycle
 *   precision, 8 single / 16 double); larger n_rhs fails with
 *   DDAMG_ERR_INVALID_ARG and a message giving the limit.  No cudaMalloc,
 *   cudaFree or other allocating call is made.
 * The handle's device (current when the handle was created) must be the current
 *   device; otherwise DDAMG_ERR_INVALID_ARG.
 * The first call on a device looks the array up with cudaGetSymbolAddress (with
 *   that device current); make that first call before any stream capture.
 * The call is stream-ordered on the handle's stream and returns without waiting
 *   for the GPU: out is complete once that stream reaches the call's last kernel.
 * All calls share the one array and it keeps the last call's contents; calls that
 *   overlap on the GPU (other host threads, other streams) race on it. */
int ddamg_apply_Dc_noalloc(ddamg_handle* h, const double* in, double* out, int n_rhs);

/* Copy the assembled coarse stencil (FP64 as assembled) into out:
 * [coarse site][direction d][row][col] complex with d = 0 self, 1 + 2 mu (+mu),
 * 2 + 2 mu (-mu), rows/cols in the coarse-vector component order. */
int ddamg_get_coarse_stencil(const ddamg_handle* h, double* out);

/* out ~ D_c^{-1} in by the odd-even GMRES of Sec. 6 (V-cycle precision).
 * fixed_iters > 0 runs exactly that many GMRES steps instead of the tolerance. */
int ddamg_coarse_solve(ddamg_handle* h, const double* in, double* out, int n_rhs, int fixed_iters);

/* out = C^(nu) in, one V-cycle (Sec. 4.2).  coarse_fixed_iters > 0 fixes the
 * number of coarse GMRES steps (for reproducible comparisons). */
int ddamg_vcycle(ddamg_handle* h, const double* in, double* out, int n_rhs, int coarse_fixed_iters);

/* Change the mass: D(m0') = D(m0) + (m0' - m0) I, so the site terms, D_c's
 * diagonal blocks (P^H P = I) and the coarse even-site inverses are updated
 * while P is kept (mass re-use, Sec. 6.3). */
int ddamg_set_mass(ddamg_handle* h, double m0);

/* Issue all further work of the handle on this cudaStream_t (NULL = the
 * handle's own stream). */
int ddamg_set_stream(ddamg_handle* h, void* cuda_stream);

/* Geometry of the handle: V, number of coarse sites, 2N. */
int ddamg_info(const ddamg_handle* h, long long* n_sites, long long* n_coarse_sites, int* coarse_dof);

/* Per-kernel timing with CUDA events on the handle's stream (benchmarks).
 * ddamg_profile_enable(h, mask) records the kernel families whose bit is set
 * in mask (bit order as listed by ddamg_profile_families; -1 = all, 0 = off);
 * ddamg_profile_read fills up to max entries (name, launches, total
 * milliseconds, algorithmic bytes moved and flops) and returns the number of families
 * recorded.  ddamg_profile_families writes the comma-separated family names
 * into names (len bytes) and returns their number. */
typedef struct {
    char name[48];
    long long launches;
    double total_ms;
    double bytes;  /* algorithmic bytes moved (every operand read/written once per launch) */
    double flops;  /* algorithmic floating-point operations (0 where not counted) */
} ddamg_kernel_profile;
int ddamg_profile_enable(ddamg_handle* h, int family_mask);
int ddamg_profile_families(char* names, int len);
int ddamg_profile_read(ddamg_handle* h, ddamg_kernel_profile* out, int max);
int ddamg_profile_reset(ddamg_handle* h);

/* Number of kernels this library has launched since load (all handles). */
long long ddamg_launch_count(void);

/* Test hook: make the next n device allocations of the library fail (OOM). */
void ddamg_debug_fail_allocs(int n);

/* ---- Recursion to a third level (Sec. 3: the two-level algorithm formulated again for the coarse
 * system, whose solve then needs only low accuracy; Sec. 6.4: 3 and 4 levels).  The paper prints no
 * algorithm for it; this one is:
 *   level 1 = the handle's coarse lattice and D_1 = D_c; its lattice blocks (block1) are the
 *   level-1 SAP domains and aggregates; P_1 is the ordered orthonormal basis of the level-1 test
 *   vectors on each (block, Gamma5^c half); D_2 = P_1^H D_1 P_1, solved by odd-even GMRES (Sec. 6);
 *   the level-1 V-cycle is x = P_1 D_2^{-1} P_1^H r followed by nu1 SAP iterations on D_1 x = r;
 *   the fine V-cycle's coarse solve becomes FGMRES(inner_kv) on D_1 to inner_tol preconditioned by
 *   the level-1 V-cycle (inner = 0), or one level-1 V-cycle (inner = 1).
 * P_1, D_2 and its inverses are built in FP64; the level-1 and level-2 solves run in the handle's
 * V-cycle precision (FP64 on DOUBLE handles, FP32 on SINGLE and HALF handles, with FP32 copies of
 * D_1, P_1, D_2 and the inverses).  HALF handles also keep FP16 copies: the level-1 SAP reads D_1 and
 * its even inverses in FP16 (FP32 arithmetic), and the coarsest level's GMRES and ddamg_ml_apply_D2
 * apply D_2 (and its even inverses) from FP16 tensor-core fragments, with each right-hand-side entry
 * entering as an FP16 hi + lo pair so that the product is the FP16-rounded matrix times the FP32
 * vector to about 2^-22 (2 n_vec1 divisible by 8; otherwise FP32).  The third level is tied to the coarse operator it was built
 * from: after ddamg_run_setup, ddamg_setup_from_vectors or ddamg_set_mass the calls below return
 * DDAMG_ERR_NOT_READY until ddamg_ml_build runs again.
 * Level-1 vectors use the coarse layout of ddamg_restrict ([n_rhs][coarse sites lex][2N]);
 * level-2 vectors are [n_rhs][level-2 sites lex][2 n_vec1], the level-2 sites being the level-1
 * blocks numbered lexicographically by block coordinates, component h * n_vec1 + j for the j-th
 * vector on the Gamma5^c half h.  Pointers may be host or device memory (as elsewhere). */
typedef struct {
    int block1[4];      /* level-1 block in coarse sites: SAP domain and aggregate (2,2,2,2) */
    int n_vec1;         /* level-1 test vectors N_1 per aggregate half (20) */
    int nu1;            /* SAP iterations of the level-1 V-cycle (2) */
    int mr_steps1;      /* MR steps of its block solver (4) */
    int inner;          /* 0: FGMRES on D_1 with the level-1 V-cycle; 1: one level-1 V-cycle (0) */
    int inner_kv;       /* restart length of that FGMRES (10; at most 64) */
    double inner_tol;   /* its relative residual target (5e-2) */
    int inner_maxiter;  /* cap on its iterations per solve (1000) */
    double coarse_tol;  /* relative residual target of the odd-even GMRES on D_2 (5e-2) */
    int coarse_restart; /* its restart length (30; at most 64) */
    int coarse_maxiter; /* cap on its iterations per solve (1000) */
    int n_inv1;         /* rounds of the level-1 setup of ddamg_ml_setup (6) */
    int setup_update1;  /* ddamg_setup_update of those rounds (DDAMG_SETUP_DDALPHA) */
} ddamg_ml_params;
void ddamg_ml_default_params(ddamg_ml_params* p);

/* Build level 2 from the level-1 test vectors v1 ([n_vec1][coarse sites lex][2N]): P_1, D_2 and the
 * inverses of D_2's even diagonal blocks.  INVALID_ARG: block1 not dividing
 * the coarse lattice into an even number of blocks per direction (with one even extent), or a
 * parameter out of range; RANK: v1 linearly dependent on an aggregate or a singular diagonal block
 * of D_2 (the previous third level is then released). */
int ddamg_ml_build(ddamg_handle* h, const ddamg_ml_params* p, const double* v1);
/* Build level 2 by the adaptive setup on level 1 instead: Algorithm 1's first phase
 * (v_j <- M_SAP^(eta) v_j, eta = 1, 2, 3, with the level-1 SAP) and n_inv1 rounds of Algorithm 2
 * (or of Algorithm 1's update) with the level-1 V-cycle, all n_vec1 vectors as one batch, from the
 * initial vectors v0 ([n_vec1][coarse sites lex][2N], e.g. random); P_1 and D_2 are rebuilt at the
 * start of every round and after the last.  v_out (may be null) receives the final vectors.
 * Errors as ddamg_ml_build. */
int ddamg_ml_setup(ddamg_handle* h, const ddamg_ml_params* p, const double* v0, double* v_out);
/* A fourth (fifth, ...) level: the same construction applied to the current coarsest level, whose
 * odd-even GMRES is then replaced by FGMRES(inner_kv) preconditioned by its own V-cycle (Sec. 6.4
 * runs 2, 3 and 4 levels).  p->block1 and p->n_vec1 refer to the current coarsest level (its sites
 * and 2 n_vec components per site); v holds its test vectors ([n_vec1][its sites lex][its
 * components]): initial ones for the adaptive setup (setup != 0), or the vectors themselves
 * (setup == 0).  v_out (may be null) receives the final vectors.  Errors as ddamg_ml_build;
 * NOT_READY without a third level. */
int ddamg_ml_add_level(ddamg_handle* h, const ddamg_ml_params* p, const double* v, int setup, double* v_out);
/* Number of levels of the hierarchy: 2 without a third level. */
int ddamg_ml_levels(const ddamg_handle* h);
/* Release the levels beyond the second (ddamg_destroy does it too). */
int ddamg_ml_release(ddamg_handle* h);
/* out = M_SAP^(nu) in on level 1 (red-black SAP of D_1 over the level-1 blocks, MR block solves). */
int ddamg_ml_apply_sap1(ddamg_handle* h, const double* in, double* out, int n_rhs, int nu);
/* Level-1 restriction out = P_1^H in (level 1 -> level 2) and prolongation out = P_1 in. */
int ddamg_ml_restrict1(ddamg_handle* h, const double* in, double* out, int n_rhs);
int ddamg_ml_prolong1(ddamg_handle* h, const double* in, double* out, int n_rhs);
/* out = D_2 in on level-2 vectors. */
int ddamg_ml_apply_D2(ddamg_handle* h, const double* in, double* out, int n_rhs);
/* out = the level-1 V-cycle applied to in (level-1 vectors). */
int ddamg_ml_vcycle1(ddamg_handle* h, const double* in, double* out, int n_rhs);
/* out = the fine V-cycle with the recursive coarse solve applied to in (fine spinors);
 * inner_fixed_iters > 0 runs exactly that many FGMRES steps on D_1 instead of stopping at inner_tol. */
int ddamg_ml_vcycle(ddamg_handle* h, const double* in, double* out, int n_rhs, int inner_fixed_iters);
/* Three-level solve: ddamg_solve_batch (same outer scheme, initial guess z, tol, status and
 * stats) with the fine V-cycle's coarse solve replaced by the recursion (coarse_iterations =
 * FGMRES steps on D_1). */
int ddamg_ml_solve(ddamg_handle* h, const double* b, double* z, int n_rhs, double tol, ddamg_stats* st);
/* ddamg_ml_solve from the zero initial guess with z output only (as
 * ddamg_solve_batch_zero_guess). */
int ddamg_ml_solve_zero_guess(ddamg_handle* h, const double* b, double* z, int n_rhs, double tol, ddamg_stats* st);
/* Counters of the last ddamg_ml_solve: out[0] FGMRES steps on D_1, out[1] GMRES steps on D_2,
 * out[2] level-1 V-cycles (per right-hand side). */
int ddamg_ml_counts(const ddamg_handle* h, long long* out);

/* Release every resource of the handle. */
int ddamg_destroy(ddamg_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* DDAMG_H */
