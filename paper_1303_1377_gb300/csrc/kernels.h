// Host-side declarations of the kernel launchers of libddamg (all return 0 or a
// negative ddamg_status).
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"
#include "../../include/ddamg.h"

namespace ddamg {

template <typename T>
struct FineOp {
    const cplx<T>* U;   // [4][9][V]
    const T* clov;      // [72][V] site term A = (m0+4) I + clover
    const T* clovinv;   // [72][V] A^{-1} (used on even sites)
};

struct FineOpAoS {  // LinksAoS, CloverAoS: common.cuh
    LinksAoS U;
    CloverAoS clov, clovinv;
};
struct FineOpAoS16 {
    LinksAoS16 U;
    CloverAoS16 clov, clovinv;
};

// coarse stencil in storage type S (float, double or __half2 packed as cplx<half>)
template <typename S>
struct CoarseOp {
    const S* B;     // [NB][9][nc(col)][nc(row)] column-major 2N x 2N blocks, d = 0 self, 1 + dir
    const S* Dinv;  // [NB/2][nc][nc] column-major inverse of B_0 on even coarse sites
    const int* cnbr;  // [8][NB] neighbouring coarse site per direction
    int NB;
    int nc;
};

// ---- fine.cu
template <typename T, typename Ts>
int launch_dslash(const Geom& g, const FineOp<T>& op, const cplx<Ts>* in, const cplx<T>* b, cplx<T>* out, int nrhs,
                  cudaStream_t st);
template <typename T>
int launch_sap_colour(const Geom& g, const FineOp<T>& op, const cplx<T>* b, cplx<T>* z, int colour, int nrhs, int mr_steps,
                      cudaStream_t st);
// FP32 SAP sweep reading links and site terms from their per-site copies
int launch_sap_colour_aos(const Geom& g, const FineOpAoS& op, const cplx<float>* b, cplx<float>* z, int colour, int nrhs, int mr_steps,
                          cudaStream_t st);
bool sap_aos_supported(const Geom& g, int nrhs);
int launch_sap_colour_aos16(const Geom& g, const FineOpAoS16& op, const cplx<float>* b, cplx<float>* z, int colour, int nrhs,
                            int mr_steps, cudaStream_t st);
// FP32 [comp][V] -> FP16 per-site copies (links [V][4][3] uint4, site term [V][9] uint4)
int links_to_aos16(const cplx<float>* U, uint4* out, int V, cudaStream_t st);
int clover_to_aos16(const float* cl, uint4* out, int V, cudaStream_t st);
// [comp][V] -> per-site copies (links: 4 x 9 complex -> [V][4][5] float4; site term: 72 -> [V][18] float4)
int links_to_aos(const cplx<float>* U, float4* out, int V, cudaStream_t st);
int clover_to_aos(const float* cl, float4* out, int V, cudaStream_t st);
int upload_gamma_products(const double* gg);
int launch_dslash_dw(const Geom& g, const float4* U, const float2* clov, const cplx<float>* in, void* out, bool out_dw, int nrhs,
                     cudaStream_t st);
int launch_to_dw(const double* in, float2* out, size_t n, cudaStream_t st);
int launch_clover(const Geom& g, const cplx<double>* U, double m0, double csw, double* clov, double* clovinv, cudaStream_t st);

// ---- transfer.cu (P, P^H, Gram-Schmidt, D_c assembly)
template <typename T, typename Tp>
int launch_restrict(const Geom& g, const cplx<Tp>* P, int N, const cplx<T>* in, cplx<T>* out, int nrhs, cudaStream_t st);
template <typename T, typename Tp>
int launch_prolong(const Geom& g, const cplx<Tp>* P, int N, const cplx<T>* in, cplx<T>* out, int nrhs, cudaStream_t st);
// half-precision V-cycle: restriction as FP16 tensor-core products (needs Vb % 16 == 0, N % 4 == 0, N <= 32)
bool restrict_tc_supported(const Geom& g, int N);
// rmax: nrhs ints of device scratch (the field maxima)
int launch_restrict_tc(const Geom& g, const cplx<__half>* P, int N, const cplx<float>* in, cplx<float>* out, int nrhs, int* rmax,
                       cudaStream_t st);
// half-precision V-cycle: prolongation as FP16 tensor-core products (needs Vb % 16 == 0, N <= 32)
bool prolong_tc_supported(const Geom& g, int N);
int launch_prolong_tc(const Geom& g, const cplx<__half>* P, int N, const cplx<float>* in, cplx<float>* out, int nrhs, cudaStream_t st);
int launch_gram_schmidt(const Geom& g, cplx<double>* P, int N, int* rank_fail, cudaStream_t st);
int launch_assemble_T(const Geom& g, const FineOp<double>& op, const cplx<double>* P, int N, int dir, int col0, int ncols, cplx<double>* T,
                      cudaStream_t st);
int launch_block_project(const Geom& g, const cplx<double>* P, int N, const cplx<double>* T, int col0, int ncols, const int* sites,
                         int nsites, double* Bout, size_t site_stride, cudaStream_t st);

// ---- coarse.cu
template <typename T, typename S>
int launch_coarse_full(const CoarseOp<S>& op, const cplx<T>* x, cplx<T>* y, int nrhs, cudaStream_t st);
template <typename T, typename S>
int launch_coarse_even(const CoarseOp<S>& op, const cplx<T>* b_e, size_t b_rs, const cplx<T>* x_o, size_t x_rs, T beta,
                       cplx<T>* out_e, size_t o_rs, int nrhs, cudaStream_t st);
template <typename T, typename S>
int launch_coarse_odd(const CoarseOp<S>& op, const cplx<T>* x_o, size_t x_rs, const cplx<T>* t_e, size_t t_rs, int use_diag,
                      cplx<T>* out_o, size_t o_rs, int nrhs, cudaStream_t st);
int launch_coarse_invert(const double* B, double* Dinv, int NB, int nc, int* fail, cudaStream_t st);

// ---- coarse_tc.cu (half-precision storage, tensor cores)
struct CoarseTC {
    const uint4* Bh;
    const uint4* Dh;
    const int* cnbr;
    int NB, nc, Mt, Kt_all, Kt_hops, Kt_d;
    int* err;       // set to 1 by a kernel whose bulk copy did not complete (read by the solve)
    int split = 0;  // 1: right-hand sides enter as FP16 hi + lo pairs (about FP32 accuracy of the product)
};
int tc_dims(int nc, int* Mt, int* Kt_all, int* Kt_hops, int* Kt_d);
int pack_coarse_tc(const double* B64, const double* Dinv64, uint4* Bh, uint4* Dh, int NB, int nc, cudaStream_t st);
int tc_coarse_full(const CoarseTC& op, const cplx<float>* x, cplx<float>* y, int nrhs, cudaStream_t st);
int tc_coarse_even(const CoarseTC& op, const cplx<float>* b_e, size_t b_rs, const cplx<float>* x_o, size_t x_rs, float beta,
                   cplx<float>* out_e, size_t o_rs, int nrhs, cudaStream_t st);
int tc_coarse_odd(const CoarseTC& op, const cplx<float>* x_o, size_t x_rs, const cplx<float>* t_e, size_t t_rs, int use_diag,
                  cplx<float>* out_o, size_t o_rs, int nrhs, cudaStream_t st);
int convert_to_half(const double* in, void* out, size_t n, cudaStream_t st);

}  // namespace ddamg
