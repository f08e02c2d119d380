// Batched vector kernels for the Krylov solvers: multi-dot products with FP64
// accumulation (deterministic two-stage reduction), linear combinations with
// per-right-hand-side complex coefficients, precision conversion and the
// permutations between the ABI's lexicographic layout and the internal order.
#include "kernels.h"
#include "blas.h"
#include "dw.cuh"

namespace ddamg {

// Basis addressing: vector i of rhs r starts at base + i * istride + r * rstride.
constexpr int kDotThreads = 256;
constexpr int kDotMaxK = 32;

// stage 1: partial[cta][i][r] for i < k over a slice of n
template <typename Ta, typename Tb, int KB>
__global__ void __launch_bounds__(kDotThreads) multidot_kernel(const cplx<Ta>* __restrict__ A, size_t istride, size_t arstride, int k,
                                                               const cplx<Tb>* __restrict__ w, size_t wrstride, size_t n, int nrhs,
                                                               int ctas_per_rhs, double* __restrict__ partial) {
    const int r = blockIdx.x % nrhs;
    const int part = blockIdx.x / nrhs;
    const cplx<Ta>* Ar = A + r * arstride;
    const cplx<Tb>* wr = w + r * wrstride;
    double acc[2 * KB];
#pragma unroll
    for (int q = 0; q < 2 * KB; ++q) acc[q] = 0.0;
    const size_t stride = (size_t)ctas_per_rhs * blockDim.x;
    for (size_t e = (size_t)part * blockDim.x + threadIdx.x; e < n; e += stride) {
        cplx<double> wv = ccast<double>(wr[e]);
#pragma unroll
        for (int i = 0; i < KB; ++i) {
            if (i < k) {
                cplx<double> a = ccast<double>(Ar[i * istride + e]);
                acc[2 * i] = fma(a.re, wv.re, fma(a.im, wv.im, acc[2 * i]));
                acc[2 * i + 1] = fma(a.re, wv.im, fma(-a.im, wv.re, acc[2 * i + 1]));
            }
        }
    }
    __shared__ double red[kDotThreads / 32][2 * KB];
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < 2 * KB; ++q) {
        if (q < 2 * k) {
            double v = warp_sum(acc[q]);
            if (lane == 0) red[wi][q] = v;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * k; q += blockDim.x) {
        double s = 0;
        for (int ww = 0; ww < kDotThreads / 32; ++ww) s += red[ww][q];
        partial[((size_t)blockIdx.x) * 2 * k + q] = s;
    }
}

// stage 2: out[i * ostride_i + r] = sum over the ctas of rhs r
__global__ void multidot_finish(const double* __restrict__ partial, int k, int nrhs, int ctas_per_rhs,
                                cplx<double>* __restrict__ out, int ostride_i, const int* __restrict__ run_flag = nullptr) {
    if (run_flag && !*run_flag) return;
    int q = blockIdx.x * blockDim.x + threadIdx.x;  // q = r * k + i
    if (q >= nrhs * k) return;
    int r = q / k, i = q % k;
    double re = 0, im = 0;
    for (int p = 0; p < ctas_per_rhs; ++p) {
        const double* src = partial + ((size_t)(p * nrhs + r)) * 2 * k;
        re += src[2 * i];
        im += src[2 * i + 1];
    }
    out[(size_t)i * ostride_i + r] = mk(re, im);
}

template <typename Ta, typename Tb>
int multidot(const cplx<Ta>* A, size_t istride, size_t arstride, int k, const cplx<Tb>* w, size_t wrstride, size_t n, int nrhs,
             cplx<double>* out, int ostride_i, double* scratch, cudaStream_t st) {
    int off = 0;
    while (off < k) {
        int kk = k - off;
        if (kk > kDotMaxK) kk = kDotMaxK;
        int ctas = (int)((n + kDotThreads - 1) / kDotThreads);
        int target = 1216 / nrhs;  // about 8 CTAs per SM over all rhs
        if (target < 1) target = 1;
        if (ctas > target) ctas = target;
        const cplx<Ta>* Ab = A + off * istride;
        if (kk <= 1)
            multidot_kernel<Ta, Tb, 1><<<ctas * nrhs, kDotThreads, 0, st>>>(Ab, istride, arstride, kk, w, wrstride, n, nrhs, ctas, scratch);
        else if (kk <= 4)
            multidot_kernel<Ta, Tb, 4><<<ctas * nrhs, kDotThreads, 0, st>>>(Ab, istride, arstride, kk, w, wrstride, n, nrhs, ctas, scratch);
        else if (kk <= 8)
            multidot_kernel<Ta, Tb, 8><<<ctas * nrhs, kDotThreads, 0, st>>>(Ab, istride, arstride, kk, w, wrstride, n, nrhs, ctas, scratch);
        else if (kk <= 16)
            multidot_kernel<Ta, Tb, 16><<<ctas * nrhs, kDotThreads, 0, st>>>(Ab, istride, arstride, kk, w, wrstride, n, nrhs, ctas, scratch);
        else
            multidot_kernel<Ta, Tb, 32><<<ctas * nrhs, kDotThreads, 0, st>>>(Ab, istride, arstride, kk, w, wrstride, n, nrhs, ctas, scratch);
        DD_CHECK_LAUNCH();
        multidot_finish<<<ceil_div((long long)nrhs * kk, 128), 128, 0, st>>>(scratch, kk, nrhs, ctas, out + (size_t)off * ostride_i,
                                                                          ostride_i);
        DD_CHECK_LAUNCH();
        off += kk;
    }
    return 0;
}

// out[r] = beta * out[r] + sum_{i<k} coef[i * cstride_i + r] * A_i[r]   (coef FP64 complex, on the device)
template <typename To, typename Ta>
__global__ void lincomb_kernel(cplx<To>* __restrict__ out, size_t ors, double beta, const cplx<Ta>* __restrict__ A, size_t istride,
                               size_t ars, int k, const cplx<double>* __restrict__ coef, int cstride_i, size_t n, int nrhs,
                               const int* __restrict__ mask, double alpha) {
    const size_t tot = n * nrhs;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(q / n);
        size_t e = q % n;
        if (mask && !mask[r]) continue;
        cplx<double> acc = beta == 0.0 ? czero<double>() : beta * ccast<double>(out[r * ors + e]);
        for (int i = 0; i < k; ++i) cmac(acc, alpha * coef[(size_t)i * cstride_i + r], ccast<double>(A[i * istride + r * ars + e]));
        out[r * ors + e] = ccast<To>(acc);
    }
}

template <typename To, typename Ta>
int lincomb(cplx<To>* out, size_t ors, double beta, const cplx<Ta>* A, size_t istride, size_t ars, int k, const cplx<double>* coef,
            int cstride_i, size_t n, int nrhs, const int* mask, cudaStream_t st, double alpha) {
    long long tot = (long long)n * nrhs;
    int blocks = ceil_div(tot, 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    lincomb_kernel<To, Ta><<<blocks, 256, 0, st>>>(out, ors, beta, A, istride, ars, k, coef, cstride_i, n, nrhs, mask, alpha);
    DD_CHECK_LAUNCH();
    return 0;
}

template <typename To, typename Ti>
__global__ void convert_kernel(const Ti* __restrict__ in, To* __restrict__ out, size_t n) {
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) out[q] = To(in[q]);
}

template <typename To, typename Ti>
int convert(const Ti* in, To* out, size_t n, cudaStream_t st) {
    int blocks = ceil_div((long long)n, 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    convert_kernel<To, Ti><<<blocks, 256, 0, st>>>(in, out, n);
    DD_CHECK_LAUNCH();
    return 0;
}

// ABI lexicographic field [nrhs][V][ncomp] <-> internal [nrhs][ncomp][V];  lex_of[i] = lexicographic site of internal i
template <typename To, typename Ti>
__global__ void to_internal_kernel(const cplx<Ti>* __restrict__ in, cplx<To>* __restrict__ out, const int* __restrict__ lex_of, int V,
                                   int ncomp, int nrhs) {
    const size_t tot = (size_t)V * nrhs;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(q / V), i = (int)(q % V);
        const cplx<Ti>* src = in + ((size_t)r * V + lex_of[i]) * ncomp;
        cplx<To>* dst = out + (size_t)r * ncomp * V + i;
        for (int k = 0; k < ncomp; ++k) dst[(size_t)k * V] = ccast<To>(src[k]);
    }
}

template <typename To, typename Ti>
__global__ void from_internal_kernel(const cplx<Ti>* __restrict__ in, cplx<To>* __restrict__ out, const int* __restrict__ lex_of,
                                     int V, int ncomp, int nrhs) {
    const size_t tot = (size_t)V * nrhs;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(q / V), i = (int)(q % V);
        const cplx<Ti>* src = in + (size_t)r * ncomp * V + i;
        cplx<To>* dst = out + ((size_t)r * V + lex_of[i]) * ncomp;
        for (int k = 0; k < ncomp; ++k) dst[k] = ccast<To>(src[(size_t)k * V]);
    }
}

template <typename To, typename Ti>
int to_internal(const cplx<Ti>* in, cplx<To>* out, const int* lex_of, int V, int ncomp, int nrhs, cudaStream_t st) {
    int blocks = ceil_div((long long)V * nrhs, 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    to_internal_kernel<To, Ti><<<blocks, 256, 0, st>>>(in, out, lex_of, V, ncomp, nrhs);
    DD_CHECK_LAUNCH();
    return 0;
}
template <typename To, typename Ti>
int from_internal(const cplx<Ti>* in, cplx<To>* out, const int* lex_of, int V, int ncomp, int nrhs, cudaStream_t st) {
    int blocks = ceil_div((long long)V * nrhs, 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    from_internal_kernel<To, Ti><<<blocks, 256, 0, st>>>(in, out, lex_of, V, ncomp, nrhs);
    DD_CHECK_LAUNCH();
    return 0;
}

// coarse vectors: ABI [nrhs][NB lex][nc] <-> internal [nrhs][NB internal][nc]
template <typename To, typename Ti>
__global__ void coarse_perm_kernel(const cplx<Ti>* __restrict__ in, cplx<To>* __restrict__ out, const int* __restrict__ clex_of,
                                   int NB, int nc, int nrhs, int to_int) {
    const size_t tot = (size_t)NB * nc * nrhs;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
        int k = (int)(q % nc);
        size_t t = q / nc;
        int c = (int)(t % NB), r = (int)(t / NB);
        size_t a = ((size_t)r * NB + c) * nc + k;
        size_t b = ((size_t)r * NB + clex_of[c]) * nc + k;
        if (to_int) out[a] = ccast<To>(in[b]);
        else out[b] = ccast<To>(in[a]);
    }
}
template <typename To, typename Ti>
int coarse_perm(const cplx<Ti>* in, cplx<To>* out, const int* clex_of, int NB, int nc, int nrhs, int to_int, cudaStream_t st) {
    int blocks = ceil_div((long long)NB * nc * nrhs, 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    coarse_perm_kernel<To, Ti><<<blocks, 256, 0, st>>>(in, out, clex_of, NB, nc, nrhs, to_int);
    DD_CHECK_LAUNCH();
    return 0;
}

// gauge field: ABI [V lex][4][3][3] FP64 -> internal [4][9][V] FP64
__global__ void gauge_to_internal_kernel(const cplx<double>* __restrict__ in, cplx<double>* __restrict__ out,
                                         const int* __restrict__ lex_of, int V) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)V; i += (size_t)gridDim.x * blockDim.x) {
        const cplx<double>* src = in + (size_t)lex_of[i] * 36;
        for (int q = 0; q < 36; ++q) out[(size_t)q * V + i] = src[q];
    }
}
int gauge_to_internal(const cplx<double>* in, cplx<double>* out, const int* lex_of, int V, cudaStream_t st) {
    int blocks = ceil_div(V, 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    gauge_to_internal_kernel<<<blocks, 256, 0, st>>>(in, out, lex_of, V);
    DD_CHECK_LAUNCH();
    return 0;
}

// Hessenberg bookkeeping of batched (F)GMRES: one thread per right-hand side (the update: one warp).
// Column k of H arrives in hcol[i * nrhs + r] (i <= k) with ||w||^2 in hcol[(k+1) * nrhs + r].re.
// One warp per right-hand side: the lanes fetch the new Hessenberg column and the stored rotations
// side by side into shared memory, lane 0 applies the rotations in order (the only sequential part),
// and the lanes write the column back.
constexpr int kArnoldiMaxM = 64;
__global__ void __launch_bounds__(32) arnoldi_update_kernel(KrylovState s, int k, const cplx<double>* __restrict__ hcol,
                                                            cplx<double>* __restrict__ scale) {
    const int r = blockIdx.x, lane = threadIdx.x;
    const int m = s.m;
    cplx<double>* H = s.H + (size_t)r * (m + 1) * m;  // H[i * m + k]
    if (!s.active[r]) {
        if (lane == 0) scale[r] = mk(0.0, 0.0);
        return;
    }
    __shared__ cplx<double> col[kArnoldiMaxM + 1], sn_s[kArnoldiMaxM];
    __shared__ double cs_s[kArnoldiMaxM];
    for (int i = lane; i <= k + 1; i += 32) col[i] = hcol[(size_t)i * s.nrhs + r];
    for (int i = lane; i < k; i += 32) {
        cs_s[i] = s.cs[r * m + i];
        sn_s[i] = s.sn[r * m + i];
    }
    __syncwarp();
    if (lane == 0) {
        const double hk = sqrt(col[k + 1].re);
        // apply the previous rotations
        for (int i = 0; i < k; ++i) {
            const double c = cs_s[i];
            const cplx<double> sn = sn_s[i];
            const cplx<double> a = col[i], b = col[i + 1];
            col[i] = c * a + sn * b;
            col[i + 1] = c * b - conj(sn) * a;
        }
        const cplx<double> a = col[k];
        const double na = sqrt(norm2(a));
        const double den = sqrt(na * na + hk * hk);
        double c;
        cplx<double> sn;
        if (den == 0.0) {
            c = 1.0;
            sn = mk(0.0, 0.0);
        } else if (na == 0.0) {
            c = 0.0;
            sn = mk(1.0, 0.0);
        } else {
            c = na / den;
            sn = (hk / (na * den)) * a;  // (a/|a|) conj(hk)/den, hk real
        }
        s.cs[r * m + k] = c;
        s.sn[r * m + k] = sn;
        col[k] = c * a + hk * sn;
        const cplx<double> gk = s.g[r * (m + 1) + k];
        s.g[r * (m + 1) + k + 1] = -1.0 * (conj(sn) * gk);
        s.g[r * (m + 1) + k] = c * gk;
        const double est = sqrt(norm2(s.g[r * (m + 1) + k + 1]));
        s.steps[r] = k + 1;
        s.resid[r] = est;
        const bool nonfinite = !(est == est) || !(hk == hk);
        if (nonfinite) s.flags[r] |= 2;
        if (est <= s.ctarget[r] || nonfinite) s.active[r] = 0;
        scale[r] = (hk > 0.0 && s.active[r]) ? mk(1.0 / hk, 0.0) : mk(0.0, 0.0);
    }
    __syncwarp();
    for (int i = lane; i <= k; i += 32) H[i * m + k] = col[i];
}

// y = H^{-1} g (upper triangular, steps[r] columns); y stored as coef[i * nrhs + r]
__global__ void arnoldi_solve_kernel(KrylovState s, cplx<double>* __restrict__ y) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= s.nrhs) return;
    const int m = s.m;
    const cplx<double>* H = s.H + (size_t)r * (m + 1) * m;
    int n = s.steps[r];
    for (int i = m - 1; i >= n; --i) y[(size_t)i * s.nrhs + r] = mk(0.0, 0.0);
    for (int i = n - 1; i >= 0; --i) {
        cplx<double> t = s.g[r * (m + 1) + i];
        for (int j = i + 1; j < n; ++j) t = t - H[i * m + j] * y[(size_t)j * s.nrhs + r];
        cplx<double> d = H[i * m + i];
        double dn = norm2(d);
        y[(size_t)i * s.nrhs + r] = dn > 0 ? t * mk(d.re / dn, -d.im / dn) : mk(0.0, 0.0);
    }
}

// start of a cycle: beta = sqrt(nrm2[r]); g = (beta, 0...); active = beta > target; scale = 1/beta
__global__ void arnoldi_start_kernel(KrylovState s, const cplx<double>* __restrict__ nrm2, cplx<double>* __restrict__ scale,
                                     int force_all) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= s.nrhs) return;
    const int m = s.m;
    double beta = sqrt(nrm2[r].re);
    for (int i = 0; i <= m; ++i) s.g[r * (m + 1) + i] = mk(0.0, 0.0);
    s.g[r * (m + 1)] = mk(beta, 0.0);
    s.steps[r] = 0;
    s.resid[r] = beta;
    bool nonfinite = !(beta == beta) || beta > 1e300;
    if (nonfinite) s.flags[r] |= 2;
    s.active[r] = (s.enabled[r] && !nonfinite && (force_all || beta > s.target[r])) ? 1 : 0;
    s.ctarget[r] = fmax(s.target[r], s.cycle_tol * beta);
    scale[r] = (s.active[r] && beta > 0) ? mk(1.0 / beta, 0.0) : mk(0.0, 0.0);
}

int arnoldi_start(const KrylovState& s, const cplx<double>* nrm2, cplx<double>* scale, int force_all, cudaStream_t st) {
    arnoldi_start_kernel<<<ceil_div(s.nrhs, 64), 64, 0, st>>>(s, nrm2, scale, force_all);
    DD_CHECK_LAUNCH();
    return 0;
}
int arnoldi_update(const KrylovState& s, int k, const cplx<double>* hcol, cplx<double>* scale, cudaStream_t st) {
    if (s.m > kArnoldiMaxM || k >= s.m) return DDAMG_ERR_INVALID_ARG;
    arnoldi_update_kernel<<<s.nrhs, 32, 0, st>>>(s, k, hcol, scale);
    DD_CHECK_LAUNCH();
    return 0;
}
int arnoldi_solve(const KrylovState& s, cplx<double>* y, cudaStream_t st) {
    arnoldi_solve_kernel<<<ceil_div(s.nrhs, 64), 64, 0, st>>>(s, y);
    DD_CHECK_LAUNCH();
    return 0;
}

// ---------------------------------------------------------------------------
// double-word basis vectors (cplx<dwf>, one float4 per complex number)
// ---------------------------------------------------------------------------
__device__ __forceinline__ cdw ld4(const cplx<dwf>* p) {
    float4 v = *reinterpret_cast<const float4*>(p);
    return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ void st4(cplx<dwf>* p, const cdw& a) {
    dw re = dw_norm(a.re), im = dw_norm(a.im);
    *reinterpret_cast<float4*>(p) = make_float4(re.h, re.l, im.h, im.l);
}

template <int KB>
__global__ void __launch_bounds__(kDotThreads) multidot_dw_kernel(const cplx<dwf>* __restrict__ A, size_t istride, size_t arstride, int k,
                                                                  const cplx<dwf>* __restrict__ w, size_t wrstride, size_t n, int nrhs,
                                                                  int ctas_per_rhs, double* __restrict__ partial,
                                                                  const int* __restrict__ run_flag) {
    if (run_flag && !*run_flag) return;
    const int r = blockIdx.x % nrhs;
    const int part = blockIdx.x / nrhs;
    const cplx<dwf>* Ar = A + r * arstride;
    const cplx<dwf>* wr = w + r * wrstride;
    cdw acc[KB];
#pragma unroll
    for (int q = 0; q < KB; ++q) acc[q] = cdw_zero();
    const size_t stride = (size_t)ctas_per_rhs * blockDim.x;
    for (size_t e = (size_t)part * blockDim.x + threadIdx.x; e < n; e += stride) {
        cdw wv = ld4(wr + e);
#pragma unroll
        for (int i = 0; i < KB; ++i)
            if (i < k) cdw_mac_conj(acc[i], ld4(Ar + i * istride + e), wv);
    }
    __shared__ double red[kDotThreads / 32][2 * KB];
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < KB; ++i) {
        if (i < k) {
            double vr = warp_sum(dw_to_double(acc[i].re));
            double vi = warp_sum(dw_to_double(acc[i].im));
            if (lane == 0) {
                red[wi][2 * i] = vr;
                red[wi][2 * i + 1] = vi;
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * k; q += blockDim.x) {
        double s = 0;
        for (int ww = 0; ww < kDotThreads / 32; ++ww) s += red[ww][q];
        partial[((size_t)blockIdx.x) * 2 * k + q] = s;
    }
}

int multidot_dw(const cplx<dwf>* A, size_t istride, size_t arstride, int k, const cplx<dwf>* w, size_t wrstride, size_t n, int nrhs,
                cplx<double>* out, int ostride_i, double* scratch, const int* run_flag, cudaStream_t st) {
    int off = 0;
    while (off < k) {
        int kk = k - off;
        if (kk > 16) kk = 16;
        int ctas = (int)((n + kDotThreads - 1) / kDotThreads);
        int target = 1216 / nrhs;
        if (target < 1) target = 1;
        if (ctas > target) ctas = target;
        const cplx<dwf>* Ab = A + off * istride;
        if (kk <= 1)
            multidot_dw_kernel<1><<<ctas * nrhs, kDotThreads, 0, st>>>(Ab, istride, arstride, kk, w, wrstride, n, nrhs, ctas, scratch, run_flag);
        else if (kk <= 4)
            multidot_dw_kernel<4><<<ctas * nrhs, kDotThreads, 0, st>>>(Ab, istride, arstride, kk, w, wrstride, n, nrhs, ctas, scratch, run_flag);
        else if (kk <= 8)
            multidot_dw_kernel<8><<<ctas * nrhs, kDotThreads, 0, st>>>(Ab, istride, arstride, kk, w, wrstride, n, nrhs, ctas, scratch, run_flag);
        else
            multidot_dw_kernel<16><<<ctas * nrhs, kDotThreads, 0, st>>>(Ab, istride, arstride, kk, w, wrstride, n, nrhs, ctas, scratch, run_flag);
        DD_CHECK_LAUNCH();
        multidot_finish<<<ceil_div((long long)nrhs * kk, 128), 128, 0, st>>>(scratch, kk, nrhs, ctas, out + (size_t)off * ostride_i,
                                                                          ostride_i, run_flag);
        DD_CHECK_LAUNCH();
        off += kk;
    }
    return 0;
}

template <>
int multidot<dwf, dwf>(const cplx<dwf>* A, size_t istride, size_t arstride, int k, const cplx<dwf>* w, size_t wrstride, size_t n,
                       int nrhs, cplx<double>* out, int ostride_i, double* scratch, cudaStream_t st) {
    return multidot_dw(A, istride, arstride, k, w, wrstride, n, nrhs, out, ostride_i, scratch, nullptr, st);
}

// coefficients alpha * coef[i][r] (FP64 complex) -> double-word pairs
__global__ void coef_to_dw_kernel(const cplx<double>* __restrict__ coef, int cstride_i, int k, int nrhs, double alpha,
                                  float4* __restrict__ out, const int* __restrict__ run_flag) {
    if (run_flag && !*run_flag) return;
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= k * nrhs) return;
    int i = q / nrhs, r = q % nrhs;
    cplx<double> c = coef[(size_t)i * cstride_i + r];
    dw re = dw_from_double(alpha * c.re), im = dw_from_double(alpha * c.im);
    out[q] = make_float4(re.h, re.l, im.h, im.l);
}

// out[r] = beta * out[r] + sum_i cdw[i][r] * A_i[r]  (beta 0 or 1), double-word arithmetic
template <int KB>
__global__ void lincomb_dw_kernel(cplx<dwf>* __restrict__ out, size_t ors, int beta1, const cplx<dwf>* __restrict__ A, size_t istride,
                                  size_t ars, int k, const float4* __restrict__ cdwv, size_t n, int nrhs) {
    const size_t tot = n * nrhs;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(q / n);
        size_t e = q % n;
        cdw acc = beta1 ? ld4(out + r * ors + e) : cdw_zero();
#pragma unroll 4
        for (int i = 0; i < k; ++i) {
            float4 c = __ldg(cdwv + (size_t)i * nrhs + r);
            cdw cc = {{c.x, c.y}, {c.z, c.w}};
            cdw_mac(acc, cc, ld4(A + i * istride + r * ars + e));
        }
        st4(out + r * ors + e, acc);
    }
}

int lincomb_dw(cplx<dwf>* out, size_t ors, int beta1, const cplx<dwf>* A, size_t istride, size_t ars, int k, const cplx<double>* coef,
               int cstride_i, size_t n, int nrhs, double alpha, float4* coef_scratch, cudaStream_t st) {
    coef_to_dw_kernel<<<ceil_div((long long)k * nrhs, 128), 128, 0, st>>>(coef, cstride_i, k, nrhs, alpha, coef_scratch, nullptr);
    DD_CHECK_LAUNCH();
    long long tot = (long long)n * nrhs;
    int blocks = ceil_div(tot, 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    lincomb_dw_kernel<1><<<blocks, 256, 0, st>>>(out, ors, beta1, A, istride, ars, k, coef_scratch, n, nrhs);
    DD_CHECK_LAUNCH();
    return 0;
}

// w[r] += sum_i cdw[i][r] * A_i[r] in place, with ||w[r]||^2 of the result accumulated
// per CTA (partial[cta], one rhs per CTA); skipped entirely when *run_flag == 0.
constexpr int kAxpyThreads = 256;
__global__ void __launch_bounds__(kAxpyThreads) axpy_norm_dw_kernel(cplx<dwf>* __restrict__ wv, const cplx<dwf>* __restrict__ A,
                                                                    size_t istride, size_t rstride, int k, const float4* __restrict__ cdwv,
                                                                    size_t n, int nrhs, int ctas_per_rhs, double* __restrict__ partial,
                                                                    const int* __restrict__ run_flag) {
    if (run_flag && !*run_flag) return;
    const int r = blockIdx.x % nrhs;
    const int part = blockIdx.x / nrhs;
    cplx<dwf>* wr = wv + r * rstride;
    const cplx<dwf>* Ar = A + r * rstride;
    double nrm = 0.0;
    const size_t stride = (size_t)ctas_per_rhs * blockDim.x;
    for (size_t e = (size_t)part * blockDim.x + threadIdx.x; e < n; e += stride) {
        cdw acc = ld4(wr + e);
        for (int i = 0; i < k; ++i) {
            float4 c = __ldg(cdwv + (size_t)i * nrhs + r);
            cdw cc = {{c.x, c.y}, {c.z, c.w}};
            cdw_mac(acc, cc, ld4(Ar + i * istride + e));
        }
        st4(wr + e, acc);
        double re = dw_to_double(acc.re), im = dw_to_double(acc.im);
        nrm = fma(re, re, fma(im, im, nrm));
    }
    __shared__ double red[kAxpyThreads / 32];
    nrm = warp_sum(nrm);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int q = 0; q < kAxpyThreads / 32; ++q) s += red[q];
        partial[blockIdx.x * 2] = s;
        partial[blockIdx.x * 2 + 1] = 0.0;
    }
}

int axpy_norm_dw(cplx<dwf>* w, const cplx<dwf>* A, size_t istride, size_t rstride, int k, const cplx<double>* coef, int cstride_i,
                 size_t n, int nrhs, double alpha, float4* coef_scratch, double* scratch, cplx<double>* norm_out, const int* run_flag,
                 cudaStream_t st) {
    coef_to_dw_kernel<<<ceil_div((long long)k * nrhs, 128), 128, 0, st>>>(coef, cstride_i, k, nrhs, alpha, coef_scratch, run_flag);
    DD_CHECK_LAUNCH();
    int ctas = (int)((n + kAxpyThreads - 1) / kAxpyThreads);
    int target = 1216 / nrhs;
    if (target < 1) target = 1;
    if (ctas > target) ctas = target;
    axpy_norm_dw_kernel<<<ctas * nrhs, kAxpyThreads, 0, st>>>(w, A, istride, rstride, k, coef_scratch, n, nrhs, ctas, scratch, run_flag);
    DD_CHECK_LAUNCH();
    multidot_finish<<<ceil_div((long long)nrhs, 128), 128, 0, st>>>(scratch, 1, nrhs, ctas, norm_out, nrhs, run_flag);
    DD_CHECK_LAUNCH();
    return 0;
}

// ---------------------------------------------------------------------------
// FP32 basis vectors (the inner cycles of the refinement scheme).  A thread
// handles two complex numbers (one float4) per step; products and short sums
// are FP32, flushed into FP64 accumulators every kFlush steps, so that FP64
// arithmetic stays a small fraction of the work.  Requires even n and
// 16-byte aligned vectors (every fine vector is 12 V complex numbers).
// ---------------------------------------------------------------------------
constexpr int kFlush = 32;

// The CTAs of one right-hand side leave their partial sums in `partial`; the last of them to finish
// (counted by ticket[r]) adds them up in CTA order, so the result is the same as a separate
// reduction launch (deterministic) without that launch.
__device__ __forceinline__ bool last_cta_of_rhs(unsigned* ticket, int r, int ctas_per_rhs) {
    __shared__ bool last;
    __threadfence();  // every partial of this CTA is visible before the ticket is taken
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket + r, 1u) == (unsigned)ctas_per_rhs - 1u;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Reduce-scatter of NV = 2 KB per-lane FP32 values across a warp (NV a power of two, <= 32): on
// return v[0] of lane l holds the sum over the 32 lanes of value (l mod NV).  Each halving step
// sends the half of the live values that the partner lane keeps, so the whole reduction costs
// NV - 1 shuffles (plus log2(32 / NV) for the lanes beyond NV) instead of 5 NV.
template <int NV>
__device__ __forceinline__ void warp_reduce_scatter(float (&v)[NV], int lane) {
#pragma unroll
    for (int s = NV / 2; s >= 1; s >>= 1) {
        const bool upper = lane & s;
#pragma unroll
        for (int j = 0; j < s; ++j) {
            const float send = upper ? v[j] : v[j + s];
            const float keep = upper ? v[j + s] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
#pragma unroll
    for (int s = NV; s < 32; s <<= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], s);
}

template <int KB>
__global__ void __launch_bounds__(kDotThreads) multidot_f32_kernel(const float4* __restrict__ A, size_t istride4, size_t arstride4, int k,
                                                                   const float4* __restrict__ w, size_t wrstride4, size_t n4, int nrhs,
                                                                   int ctas_per_rhs, double* __restrict__ partial, unsigned* __restrict__ ticket,
                                                                   cplx<double>* __restrict__ out, int ostride_i, cplx<double>* __restrict__ copy_last,
                                                                   const int* __restrict__ run_flag) {
    if (run_flag && !*run_flag) return;
    constexpr int NV = 2 * KB;  // (re, im) of each product, interleaved: v[2 i], v[2 i + 1]
    const int r = blockIdx.x % nrhs;
    const int part = blockIdx.x / nrhs;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const float4* Ar = A + r * arstride4;
    const float4* wr = w + r * wrstride4;
    // every kFlush steps the warp's FP32 sums are reduce-scattered and lane (q mod NV) adds the sum of
    // value q to its one FP64 accumulator: FP64 state is one register per lane, whatever KB
    float f[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) f[q] = 0.f;
    double acc = 0.0;
    const size_t stride = (size_t)ctas_per_rhs * blockDim.x;
    const size_t e0 = (size_t)part * blockDim.x + threadIdx.x;
    // the trip count is uniform across the warp (the flush needs all 32 lanes): lanes past the end
    // run the last trips with zero products
    const size_t base = e0 - lane;
    const size_t trips = base < n4 ? (n4 - base + stride - 1) / stride : 0;
    for (size_t t = 0; t < trips;) {
        const size_t tend = t + kFlush < trips ? t + kFlush : trips;
        for (; t < tend; ++t) {
            const size_t e = e0 + t * stride;
            if (e < n4) {
                const float4 wv = wr[e];
#pragma unroll
                for (int i = 0; i < KB; ++i) {
                    if (i < k) {
                        const float4 a = Ar[i * istride4 + e];  // conj(a) w for both complex numbers
                        // two independent products per component keep the accumulator chain two FMAs deep
                        f[2 * i] += fmaf(a.x, wv.x, a.y * wv.y) + fmaf(a.z, wv.z, a.w * wv.w);
                        f[2 * i + 1] += fmaf(a.x, wv.y, -a.y * wv.x) + fmaf(a.z, wv.w, -a.w * wv.z);
                    }
                }
            }
        }
        warp_reduce_scatter<NV>(f, lane);
        acc += (double)f[0];
#pragma unroll
        for (int q = 0; q < NV; ++q) f[q] = 0.f;
    }
    __shared__ double red[kDotThreads / 32][NV];
    if (lane < NV) red[wi][lane] = acc;
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * k; q += blockDim.x) {
        double s = 0;
        for (int ww = 0; ww < kDotThreads / 32; ++ww) s += red[ww][q];
        partial[((size_t)blockIdx.x) * 2 * k + q] = s;
    }
    if (!last_cta_of_rhs(ticket, r, ctas_per_rhs)) return;
    // one warp per product: its lanes read the CTAs' partial sums side by side (fixed order, so the
    // result does not depend on which CTA finished last)
    for (int i = wi; i < k; i += kDotThreads / 32) {
        double re = 0, im = 0;
        for (int p = lane; p < ctas_per_rhs; p += 32) {
            const double* src = partial + ((size_t)(p * nrhs + r)) * 2 * k;
            re += __ldcg(src + 2 * i);
            im += __ldcg(src + 2 * i + 1);
        }
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) {
            out[(size_t)i * ostride_i + r] = mk(re, im);
            if (copy_last && i == k - 1) copy_last[r] = mk(re, im);
        }
    }
    if (threadIdx.x == 0) ticket[r] = 0u;
}

static bool f32_layout_ok(const void* A, size_t istride, size_t arstride, const void* w, size_t wrstride, size_t n) {
    return n % 2 == 0 && istride % 2 == 0 && arstride % 2 == 0 && wrstride % 2 == 0 && ((uintptr_t)A & 15) == 0 &&
           ((uintptr_t)w & 15) == 0;
}

// CTAs per right-hand side of the FP32 basis kernels: about four resident CTAs per SM over all
// right-hand sides (608 on 152 SMs) as long as every thread has a float4 to work on; short vectors
// (the coarsest level) are spread thin rather than left to one CTA per right-hand side
static int f32_ctas(size_t n4, int nrhs, int threads) {
    const long long target = std::max(1, 608 / nrhs);
    const long long by_len = (long long)((n4 + threads - 1) / threads);
    return (int)std::max(1LL, std::min(target, by_len));
}

int multidot_f32(const cplx<float>* A, size_t istride, size_t arstride, int k, const cplx<float>* w, size_t wrstride, size_t n, int nrhs,
                 cplx<double>* out, int ostride_i, double* scratch, unsigned* ticket, cplx<double>* copy_last, const int* run_flag,
                 cudaStream_t st) {
    if (!f32_layout_ok(A, istride, arstride, w, wrstride, n)) return -1;
    const size_t n4 = n / 2;
    int off = 0;
    while (off < k) {
        int kk = k - off;
        if (kk > 16) kk = 16;
        const int ctas = f32_ctas(n4, nrhs, kDotThreads);
        const float4* Ab = reinterpret_cast<const float4*>(A + off * istride);
        const float4* w4 = reinterpret_cast<const float4*>(w);
        const unsigned grid = ctas * nrhs;
        cplx<double>* o = out + (size_t)off * ostride_i;
        cplx<double>* cl = off + kk == k ? copy_last : nullptr;
        if (kk <= 1)
            multidot_f32_kernel<1><<<grid, kDotThreads, 0, st>>>(Ab, istride / 2, arstride / 2, kk, w4, wrstride / 2, n4, nrhs, ctas, scratch,
                                                                 ticket, o, ostride_i, cl, run_flag);
        else if (kk <= 8)
            multidot_f32_kernel<8><<<grid, kDotThreads, 0, st>>>(Ab, istride / 2, arstride / 2, kk, w4, wrstride / 2, n4, nrhs, ctas, scratch,
                                                                 ticket, o, ostride_i, cl, run_flag);
        else
            multidot_f32_kernel<16><<<grid, kDotThreads, 0, st>>>(Ab, istride / 2, arstride / 2, kk, w4, wrstride / 2, n4, nrhs, ctas, scratch,
                                                                  ticket, o, ostride_i, cl, run_flag);
        DD_CHECK_LAUNCH();
        off += kk;
    }
    return 0;
}

// w[r] += sum_i alpha c[i][r] * A_i[r] in place (FP32; the coefficients are rounded to FP32 in the
// kernel), with ||w[r]||^2 of the result (FP64 sum) in norm_out[r].re
constexpr int kAxpyMaxK = 64;
__global__ void __launch_bounds__(kAxpyThreads) axpy_norm_f32_kernel(float4* __restrict__ wv, const float4* __restrict__ A, size_t istride4,
                                                                     size_t rstride4, int k, const cplx<double>* __restrict__ coef,
                                                                     int cstride_i, double alpha, size_t n4, int nrhs, int ctas_per_rhs,
                                                                     double* __restrict__ partial, unsigned* __restrict__ ticket,
                                                                     cplx<double>* __restrict__ norm_out, const int* __restrict__ run_flag) {
    if (run_flag && !*run_flag) return;
    const int r = blockIdx.x % nrhs;
    const int part = blockIdx.x / nrhs;
    __shared__ float2 cs[kAxpyMaxK];
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const cplx<double> c = coef[(size_t)i * cstride_i + r];
        cs[i] = make_float2((float)(alpha * c.re), (float)(alpha * c.im));
    }
    __syncthreads();
    float4* wr = wv + r * rstride4;
    const float4* Ar = A + r * rstride4;
    double nrm = 0.0;
    const size_t stride = (size_t)ctas_per_rhs * blockDim.x;
    for (size_t e = (size_t)part * blockDim.x + threadIdx.x; e < n4; e += stride) {
        float4 acc = wr[e];
#pragma unroll 4
        for (int i = 0; i < k; ++i) {
            const float2 c = cs[i];
            const float4 a = Ar[i * istride4 + e];
            acc.x = fmaf(c.x, a.x, fmaf(-c.y, a.y, acc.x));
            acc.y = fmaf(c.x, a.y, fmaf(c.y, a.x, acc.y));
            acc.z = fmaf(c.x, a.z, fmaf(-c.y, a.w, acc.z));
            acc.w = fmaf(c.x, a.w, fmaf(c.y, a.z, acc.w));
        }
        wr[e] = acc;
        nrm += (double)(acc.x * acc.x + acc.y * acc.y) + (double)(acc.z * acc.z + acc.w * acc.w);
    }
    __shared__ double red[kAxpyThreads / 32];
    nrm = warp_sum(nrm);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int q = 0; q < kAxpyThreads / 32; ++q) s += red[q];
        partial[blockIdx.x] = s;
    }
    if (!last_cta_of_rhs(ticket, r, ctas_per_rhs)) return;
    if (threadIdx.x == 0) {
        double s = 0;
        for (int p = 0; p < ctas_per_rhs; ++p) s += __ldcg(partial + (size_t)p * nrhs + r);
        norm_out[r] = mk(s, 0.0);
        ticket[r] = 0u;
    }
}

int axpy_norm_f32(cplx<float>* w, const cplx<float>* A, size_t istride, size_t rstride, int k, const cplx<double>* coef, int cstride_i,
                  size_t n, int nrhs, double alpha, double* scratch, unsigned* ticket, cplx<double>* norm_out, const int* run_flag,
                  cudaStream_t st) {
    if (!f32_layout_ok(A, istride, rstride, w, rstride, n) || k > kAxpyMaxK) return -1;
    const size_t n4 = n / 2;
    const int ctas = f32_ctas(n4, nrhs, kAxpyThreads);
    axpy_norm_f32_kernel<<<ctas * nrhs, kAxpyThreads, 0, st>>>(reinterpret_cast<float4*>(w), reinterpret_cast<const float4*>(A), istride / 2,
                                                               rstride / 2, k, coef, cstride_i, alpha, n4, nrhs, ctas, scratch, ticket,
                                                               norm_out, run_flag);
    DD_CHECK_LAUNCH();
    return 0;
}

// w[r] *= scale[r] (real part) for an FP32 basis vector; one float4 (two complex numbers) per step
__global__ void scale_f32_kernel(float4* __restrict__ w, const cplx<double>* __restrict__ scale, size_t n4, int nrhs) {
    const int r = blockIdx.y;
    const float a = (float)scale[r].re;
    float4* wr = w + (size_t)r * n4;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n4; e += (size_t)gridDim.x * blockDim.x) {
        float4 v = wr[e];
        v.x *= a, v.y *= a, v.z *= a, v.w *= a;
        wr[e] = v;
    }
}
int scale_f32(cplx<float>* w, const cplx<double>* scale, size_t n, int nrhs, cudaStream_t st) {
    if (n % 2 || ((uintptr_t)w & 15)) return -1;
    const size_t n4 = n / 2;
    int bx = (int)std::min<size_t>((n4 + 255) / 256, (size_t)std::max(1, 152 * 8 / nrhs));
    scale_f32_kernel<<<dim3(bx, nrhs), 256, 0, st>>>(reinterpret_cast<float4*>(w), scale, n4, nrhs);
    DD_CHECK_LAUNCH();
    return 0;
}

// x = hi + lo with hi = fl32(x), lo = fl32(x - hi): the pair holds x to about 2^-48 relative
__global__ void split_f64_kernel(const double2* __restrict__ x, float2* __restrict__ hi, float2* __restrict__ lo, size_t n) {
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const double2 v = x[q];
        const float hr = (float)v.x, hm = (float)v.y;
        hi[q] = make_float2(hr, hm);
        lo[q] = make_float2((float)(v.x - (double)hr), (float)(v.y - (double)hm));
    }
}
int split_f64(const cplx<double>* x, cplx<float>* hi, cplx<float>* lo, size_t n, cudaStream_t st) {
    int blocks = ceil_div((long long)n, 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    split_f64_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const double2*>(x), reinterpret_cast<float2*>(hi),
                                             reinterpret_cast<float2*>(lo), n);
    DD_CHECK_LAUNCH();
    return 0;
}

// Reorthogonalisation test of classical Gram-Schmidt (the DGKS criterion with
// threshold eta): request a second pass when, for any active right-hand side,
// ||w after||^2 < eta^2 ||w before||^2.
__global__ void dgks_kernel(const cplx<double>* __restrict__ before, const cplx<double>* __restrict__ after,
                            const int* __restrict__ active, int nrhs, double eta2, int* __restrict__ flag) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int f = 0;
        for (int r = 0; r < nrhs; ++r)
            if (active[r] && after[r].re < eta2 * before[r].re) f = 1;
        *flag = f;
    }
}
int dgks(const cplx<double>* before, const cplx<double>* after, const int* active, int nrhs, double eta, int* flag, cudaStream_t st) {
    dgks_kernel<<<1, 32, 0, st>>>(before, after, active, nrhs, eta * eta, flag);
    DD_CHECK_LAUNCH();
    return 0;
}
__global__ void add_columns_flag_kernel(cplx<double>* __restrict__ a, const cplx<double>* __restrict__ b, int n, const int* __restrict__ flag) {
    if (!*flag) return;
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) a[q] = a[q] + b[q];
}
int add_columns_flag(cplx<double>* a, const cplx<double>* b, int n, const int* flag, cudaStream_t st) {
    add_columns_flag_kernel<<<ceil_div(n, 128), 128, 0, st>>>(a, b, n, flag);
    DD_CHECK_LAUNCH();
    return 0;
}

// x[r] += sum_i y[i][r] Z_i[r] for an FP64 iterate and FP32 preconditioned vectors: the sum is
// formed in double-word arithmetic (exact FP32 products, ~2^-48 accumulation) and added once in FP64.
// Grid: blockIdx.y = right-hand side.
__global__ void xupdate_kernel(cplx<double>* __restrict__ x, const cplx<float>* __restrict__ Z, size_t istride, size_t n, int k,
                               const float4* __restrict__ cdwv, int nrhs) {
    const int r = blockIdx.y;
    cplx<double>* xr = x + (size_t)r * n;
    const cplx<float>* Zr = Z + (size_t)r * n;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        cdw acc = cdw_zero();
#pragma unroll 4
        for (int i = 0; i < k; ++i) {
            const float4 c = __ldg(cdwv + (size_t)i * nrhs + r);
            const cplx<float> zv = Zr[i * istride + e];
            const dw cr = {c.x, c.y}, ci = {c.z, c.w};
            dw_macf(acc.re, cr, zv.re);
            dw_macf(acc.re, dw_neg(ci), zv.im);
            dw_macf(acc.im, cr, zv.im);
            dw_macf(acc.im, ci, zv.re);
        }
        const cplx<double> xv = xr[e];
        xr[e] = mk(xv.re + dw_to_double(acc.re), xv.im + dw_to_double(acc.im));
    }
}
int xupdate_dw(cplx<double>* x, const cplx<float>* Z, size_t istride, size_t n, int k, const cplx<double>* coef, int nrhs,
               float4* coef_scratch, cudaStream_t st) {
    coef_to_dw_kernel<<<ceil_div((long long)k * nrhs, 128), 128, 0, st>>>(coef, nrhs, k, nrhs, 1.0, coef_scratch, nullptr);
    DD_CHECK_LAUNCH();
    int bx = (int)std::min<size_t>((n + 255) / 256, (size_t)std::max(1, 152 * 16 / nrhs));
    xupdate_kernel<<<dim3(bx, nrhs), 256, 0, st>>>(x, Z, istride, n, k, coef_scratch, nrhs);
    DD_CHECK_LAUNCH();
    return 0;
}

// V0 = fl32(b - (w + t)) for an FP64 w and an FP32 t (the true residual of the refinement cycles)
__global__ void residual_f32_kernel(const double2* __restrict__ b, const double2* __restrict__ w, const float2* __restrict__ t,
                                    float2* __restrict__ out, size_t n) {
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const double2 bv = b[q], wv = w[q];
        const float2 tv = t[q];
        out[q] = make_float2((float)(bv.x - (wv.x + (double)tv.x)), (float)(bv.y - (wv.y + (double)tv.y)));
    }
}
int residual_f32(const cplx<double>* b, const cplx<double>* w, const cplx<float>* t, cplx<float>* out, size_t n, cudaStream_t st) {
    int blocks = ceil_div((long long)n, 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    residual_f32_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const double2*>(b), reinterpret_cast<const double2*>(w),
                                                reinterpret_cast<const float2*>(t), reinterpret_cast<float2*>(out), n);
    DD_CHECK_LAUNCH();
    return 0;
}

// FP64 <-> double-word vectors and double-word -> FP32 (the V-cycle input)
__global__ void d2dw_kernel(const double* __restrict__ in, float2* __restrict__ out, size_t n) {
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        dw v = dw_from_double(in[q]);
        out[q] = make_float2(v.h, v.l);
    }
}
__global__ void dw2f_kernel(const float2* __restrict__ in, float* __restrict__ out, size_t n) {
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        float2 v = in[q];
        out[q] = v.x + v.y;
    }
}
int convert_d2dw(const double* in, cplx<dwf>* out, size_t nreal, cudaStream_t st) {
    int blocks = ceil_div((long long)nreal, 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    d2dw_kernel<<<blocks, 256, 0, st>>>(in, reinterpret_cast<float2*>(out), nreal);
    DD_CHECK_LAUNCH();
    return 0;
}
int convert_dw2f(const cplx<dwf>* in, float* out, size_t nreal, cudaStream_t st) {
    int blocks = ceil_div((long long)nreal, 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    dw2f_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const float2*>(in), out, nreal);
    DD_CHECK_LAUNCH();
    return 0;
}

__global__ void add_columns_kernel(cplx<double>* __restrict__ a, const cplx<double>* __restrict__ b, int n) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) a[q] = a[q] + b[q];
}
int add_columns(cplx<double>* a, const cplx<double>* b, int n, cudaStream_t st) {
    add_columns_kernel<<<ceil_div(n, 128), 128, 0, st>>>(a, b, n);
    DD_CHECK_LAUNCH();
    return 0;
}

// explicit instantiations
#define DD_INST_DOT(Ta, Tb)                                                                                                   \
    template int multidot<Ta, Tb>(const cplx<Ta>*, size_t, size_t, int, const cplx<Tb>*, size_t, size_t, int, cplx<double>*, \
                                  int, double*, cudaStream_t);
DD_INST_DOT(double, double)
DD_INST_DOT(float, float)
#define DD_INST_LC(To, Ta)                                                                                                  \
    template int lincomb<To, Ta>(cplx<To>*, size_t, double, const cplx<Ta>*, size_t, size_t, int, const cplx<double>*, int, \
                                 size_t, int, const int*, cudaStream_t, double);
DD_INST_LC(double, double)
DD_INST_LC(double, float)
DD_INST_LC(float, float)
DD_INST_LC(float, double)
template int convert<float, double>(const double*, float*, size_t, cudaStream_t);
template int convert<double, float>(const float*, double*, size_t, cudaStream_t);
template int to_internal<double, double>(const cplx<double>*, cplx<double>*, const int*, int, int, int, cudaStream_t);
template int to_internal<float, double>(const cplx<double>*, cplx<float>*, const int*, int, int, int, cudaStream_t);
template int to_internal<float, float>(const cplx<float>*, cplx<float>*, const int*, int, int, int, cudaStream_t);
template int from_internal<double, double>(const cplx<double>*, cplx<double>*, const int*, int, int, int, cudaStream_t);
template int from_internal<double, float>(const cplx<float>*, cplx<double>*, const int*, int, int, int, cudaStream_t);
template int from_internal<float, float>(const cplx<float>*, cplx<float>*, const int*, int, int, int, cudaStream_t);
template int coarse_perm<double, double>(const cplx<double>*, cplx<double>*, const int*, int, int, int, int, cudaStream_t);
template int coarse_perm<float, double>(const cplx<double>*, cplx<float>*, const int*, int, int, int, int, cudaStream_t);
template int coarse_perm<double, float>(const cplx<float>*, cplx<double>*, const int*, int, int, int, int, cudaStream_t);

}  // namespace ddamg
