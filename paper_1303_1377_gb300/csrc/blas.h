// Batched vector kernels and the device-side state of the batched (F)GMRES.
#pragma once
#include "common.cuh"

namespace ddamg {

// Per-right-hand-side Arnoldi/Givens state of a batched restarted (F)GMRES(m),
// all on the device.  H[r][i][k] (i <= m, k < m) is the rotated Hessenberg
// matrix, (cs, sn) the Givens rotations, g the rotated right-hand side.
struct KrylovState {
    int nrhs, m;
    cplx<double>* H;   // [nrhs][m+1][m]
    double* cs;        // [nrhs][m]
    cplx<double>* sn;  // [nrhs][m]
    cplx<double>* g;   // [nrhs][m+1]
    int* steps;        // Arnoldi steps taken in the current cycle
    double* resid;     // current residual estimate |g_{k+1}|
    int* active;       // still iterating in this cycle
    int* enabled;      // takes part in this solve at all
    int* flags;        // bit 1: non-finite value met
    double* target;    // absolute residual target tol * ||b||
    double* ctarget;   // target of the current cycle: max(target, cycle_tol * beta of the cycle)
    double cycle_tol;  // 0: a cycle runs to target (or the restart length)
};

template <typename Ta, typename Tb>
int multidot(const cplx<Ta>* A, size_t istride, size_t arstride, int k, const cplx<Tb>* w, size_t wrstride, size_t n, int nrhs,
             cplx<double>* out, int ostride_i, double* scratch, cudaStream_t st);
template <typename To, typename Ta>
int lincomb(cplx<To>* out, size_t ors, double beta, const cplx<Ta>* A, size_t istride, size_t ars, int k, const cplx<double>* coef,
            int cstride_i, size_t n, int nrhs, const int* mask, cudaStream_t st, double alpha = 1.0);
int add_columns(cplx<double>* a, const cplx<double>* b, int n, cudaStream_t st);
// double-word vectors
template <>
int multidot<dwf, dwf>(const cplx<dwf>* A, size_t istride, size_t arstride, int k, const cplx<dwf>* w, size_t wrstride, size_t n,
                       int nrhs, cplx<double>* out, int ostride_i, double* scratch, cudaStream_t st);
int multidot_dw(const cplx<dwf>* A, size_t istride, size_t arstride, int k, const cplx<dwf>* w, size_t wrstride, size_t n, int nrhs,
                cplx<double>* out, int ostride_i, double* scratch, const int* run_flag, cudaStream_t st);
int axpy_norm_dw(cplx<dwf>* w, const cplx<dwf>* A, size_t istride, size_t rstride, int k, const cplx<double>* coef, int cstride_i,
                 size_t n, int nrhs, double alpha, float4* coef_scratch, double* scratch, cplx<double>* norm_out, const int* run_flag,
                 cudaStream_t st);
int dgks(const cplx<double>* before, const cplx<double>* after, const int* active, int nrhs, double eta, int* flag, cudaStream_t st);
int add_columns_flag(cplx<double>* a, const cplx<double>* b, int n, const int* flag, cudaStream_t st);
int lincomb_dw(cplx<dwf>* out, size_t ors, int beta1, const cplx<dwf>* A, size_t istride, size_t ars, int k, const cplx<double>* coef,
               int cstride_i, size_t n, int nrhs, double alpha, float4* coef_scratch, cudaStream_t st);
int xupdate_dw(cplx<double>* x, const cplx<float>* Z, size_t istride, size_t n, int k, const cplx<double>* coef, int nrhs,
               float4* coef_scratch, cudaStream_t st);
// FP32 basis (even n, 16-byte aligned vectors; -1 otherwise).  ticket: nrhs zeroed counters (left
// zeroed), used to let the last CTA of each right-hand side finish the reduction.  copy_last: also
// receives the last of the k products (may be null).
int multidot_f32(const cplx<float>* A, size_t istride, size_t arstride, int k, const cplx<float>* w, size_t wrstride, size_t n, int nrhs,
                 cplx<double>* out, int ostride_i, double* scratch, unsigned* ticket, cplx<double>* copy_last, const int* run_flag,
                 cudaStream_t st);
int axpy_norm_f32(cplx<float>* w, const cplx<float>* A, size_t istride, size_t rstride, int k, const cplx<double>* coef, int cstride_i,
                  size_t n, int nrhs, double alpha, double* scratch, unsigned* ticket, cplx<double>* norm_out, const int* run_flag,
                  cudaStream_t st);
int scale_f32(cplx<float>* w, const cplx<double>* scale, size_t n, int nrhs, cudaStream_t st);
int residual_f32(const cplx<double>* b, const cplx<double>* w, const cplx<float>* t, cplx<float>* out, size_t n, cudaStream_t st);
int split_f64(const cplx<double>* x, cplx<float>* hi, cplx<float>* lo, size_t n, cudaStream_t st);
int convert_d2dw(const double* in, cplx<dwf>* out, size_t nreal, cudaStream_t st);
int convert_dw2f(const cplx<dwf>* in, float* out, size_t nreal, cudaStream_t st);
template <typename To, typename Ti>
int convert(const Ti* in, To* out, size_t n, cudaStream_t st);
template <typename To, typename Ti>
int to_internal(const cplx<Ti>* in, cplx<To>* out, const int* lex_of, int V, int ncomp, int nrhs, cudaStream_t st);
template <typename To, typename Ti>
int from_internal(const cplx<Ti>* in, cplx<To>* out, const int* lex_of, int V, int ncomp, int nrhs, cudaStream_t st);
template <typename To, typename Ti>
int coarse_perm(const cplx<Ti>* in, cplx<To>* out, const int* clex_of, int NB, int nc, int nrhs, int to_int, cudaStream_t st);
int gauge_to_internal(const cplx<double>* in, cplx<double>* out, const int* lex_of, int V, cudaStream_t st);

int arnoldi_start(const KrylovState& s, const cplx<double>* nrm2, cplx<double>* scale, int force_all, cudaStream_t st);
int arnoldi_update(const KrylovState& s, int k, const cplx<double>* hcol, cplx<double>* scale, cudaStream_t st);
int arnoldi_solve(const KrylovState& s, cplx<double>* y, cudaStream_t st);

// scratch size (doubles) needed by multidot for nrhs right-hand sides
inline size_t multidot_scratch_doubles(int nrhs) { return (size_t)(1216 / (nrhs > 0 ? nrhs : 1) + 1) * nrhs * 2 * 32 + 64; }

}  // namespace ddamg
