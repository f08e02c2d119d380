// Coarse operator kernels: D_c = P^H D P as a 9-point stencil of dense 2N x 2N
// blocks on the coarse torus (Sec. 3.2), its odd-even Schur complement pieces
// (Sec. 6) and the inverses of the diagonal blocks on even coarse sites.
//
// Storage: B[c][d][col][row] (column-major blocks), d = 0 self, 1 + dir for the
// fine directions dir = 2 mu + (backward); Dinv[c][col][row] for even c.
// Coarse sites in internal order: even (red) sites first, then odd.
// Vectors: cplx[nrhs][sites][nc] addressed through (pointer, rhs stride,
// first site) so that half vectors and full vectors share one kernel.
#include "kernels.h"

namespace ddamg {

template <typename T>
struct CVec {
    cplx<T>* p;
    size_t rstride;  // elements between right-hand sides
    int site0;       // coarse site stored at p[0]
};

// pairs of consecutive complex matrix entries (rows 2p, 2p+1 of one column)
__device__ __forceinline__ void load_pair(const float* p, cplx<float>& a, cplx<float>& b) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    a = mk(v.x, v.y);
    b = mk(v.z, v.w);
}
__device__ __forceinline__ void load_pair(const double* p, cplx<double>& a, cplx<double>& b) {
    double2 v0 = __ldg(reinterpret_cast<const double2*>(p));
    double2 v1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
    a = mk(v0.x, v0.y);
    b = mk(v1.x, v1.y);
}

// acc[2][NRP] += sum over columns q in [q0, q1) of M(q)[2p..2p+1] * xs[q][0..NRP);
// column q of the stacked matrices starts at first + q * nc complex entries (slots are
// contiguous nc x nc column-major blocks).
template <typename T, typename S, int NRP>
__device__ __forceinline__ void gemm_slice(const S* first, int nc, int p, int q0, int q1, const cplx<T>* xs,
                                           cplx<T> (&acc)[2][NRP]) {
    const S* bp = first + 2 * ((size_t)q0 * nc + 2 * p);
    const cplx<T>* xq = xs + (size_t)q0 * NRP;
#pragma unroll 2
    for (int q = q0; q < q1; ++q, bp += 2 * nc, xq += NRP) {
        cplx<T> b0, b1;
        load_pair(bp, b0, b1);
#pragma unroll
        for (int r = 0; r < NRP; ++r) {
            cplx<T> xv = xq[r];
            cmac(acc[0][r], b0, xv);
            cmac(acc[1][r], b1, xv);
        }
    }
}

// One CTA per coarse site c = site_begin + blockIdx.x.  Thread (p, g): rows 2p, 2p+1,
// k-group g of the 8 or 9 (direction, column) slices; partial sums are reduced in
// shared memory.  acc = self + hop_sign * sum_{d=1..8} B_d(c) xin[nbr_d(c)] with
//   self = 0 (self_mode 0), B_0(c) xself[c] (1) or xself[c] (2);  out = apply_inv ? Dinv acc : acc.
template <typename T, typename S, int NRP>
__global__ void __launch_bounds__(128) coarse_stencil_kernel(CoarseOp<S> op, int site_begin, CVec<T> xin, CVec<T> xself,
                                                             int self_mode, T hop_sign, int apply_inv, CVec<T> out, int nrhs) {
    extern __shared__ unsigned char smem_raw[];
    const int nc = op.nc, RP = nc / 2;
    const int KG = blockDim.x / RP;
    cplx<T>* xs = reinterpret_cast<cplx<T>*>(smem_raw);  // [slots][nc][NRP], later reused for partial sums
    const int c = site_begin + blockIdx.x;
    const bool use_hops = hop_sign != T(0);
    const int slot0 = (self_mode == 1) ? 0 : 1;      // slot 0 = B_0 x_self
    const int nslots = use_hops ? 9 - slot0 : 1 - slot0;
    const S* first = op.B + ((size_t)(c * 9 + slot0) * nc) * nc * 2;
    // stage the vectors: slot sl holds direction d = slot0 + sl
    for (int q = threadIdx.x; q < nslots * nc * NRP; q += blockDim.x) {
        int r = q % NRP, col = (q / NRP) % nc, d = slot0 + q / (NRP * nc);
        cplx<T> v = czero<T>();
        if (r < nrhs) {
            if (d == 0) {
                v = xself.p[r * xself.rstride + (size_t)(c - xself.site0) * nc + col];
            } else {
                int n = __ldg(op.cnbr + (d - 1) * op.NB + c);
                v = hop_sign * xin.p[r * xin.rstride + (size_t)(n - xin.site0) * nc + col];
            }
        }
        xs[q] = v;
    }
    __syncthreads();
    const int p = threadIdx.x % RP, g = threadIdx.x / RP;
    const bool act = g < KG;
    cplx<T> acc[2][NRP];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = 0; r < NRP; ++r) acc[h][r] = czero<T>();
    const int Kt = nslots * nc;
    if (act && nslots > 0) gemm_slice<T, S, NRP>(first, nc, p, (g * Kt) / KG, ((g + 1) * Kt) / KG, xs, acc);
    __syncthreads();
    // reduce the KG partial sums: red[g][row][r]
    cplx<T>* red = xs;
    if (act)
#pragma unroll
        for (int r = 0; r < NRP; ++r) {
            red[((size_t)g * nc + 2 * p) * NRP + r] = acc[0][r];
            red[((size_t)g * nc + 2 * p + 1) * NRP + r] = acc[1][r];
        }
    __syncthreads();
    cplx<T>* vsum = red + (size_t)KG * nc * NRP;  // [nc][NRP]
    for (int o = threadIdx.x; o < nc * NRP; o += blockDim.x) {
        cplx<T> s = czero<T>();
        for (int gg = 0; gg < KG; ++gg) s = s + red[(size_t)gg * nc * NRP + o];
        if (self_mode == 2) {
            int row = o / NRP, r = o % NRP;
            if (r < nrhs) s = s + xself.p[r * xself.rstride + (size_t)(c - xself.site0) * nc + row];
        }
        vsum[o] = s;
    }
    __syncthreads();
    if (apply_inv) {
        const S* dfirst = op.Dinv + ((size_t)c * nc) * nc * 2;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int r = 0; r < NRP; ++r) acc[h][r] = czero<T>();
        if (act) gemm_slice<T, S, NRP>(dfirst, nc, p, (g * nc) / KG, ((g + 1) * nc) / KG, vsum, acc);
        __syncthreads();
        if (act)
#pragma unroll
            for (int r = 0; r < NRP; ++r) {
                red[((size_t)g * nc + 2 * p) * NRP + r] = acc[0][r];
                red[((size_t)g * nc + 2 * p + 1) * NRP + r] = acc[1][r];
            }
        __syncthreads();
        for (int o = threadIdx.x; o < nc * NRP; o += blockDim.x) {
            cplx<T> s = czero<T>();
            for (int gg = 0; gg < KG; ++gg) s = s + red[(size_t)gg * nc * NRP + o];
            vsum[o] = s;
        }
        __syncthreads();
    }
    for (int o = threadIdx.x; o < nc * NRP; o += blockDim.x) {
        int row = o / NRP, r = o % NRP;
        if (r < nrhs) out.p[r * out.rstride + (size_t)(c - out.site0) * nc + row] = vsum[o];
    }
}

template <typename T, typename S, int NRP>
static int launch_stencil_nrp(const CoarseOp<S>& op, int site_begin, int nsites, CVec<T> xin, CVec<T> xself, int self_mode,
                              T hop_sign, int apply_inv, CVec<T> out, int nrhs, cudaStream_t st) {
    const int RP = op.nc / 2;
    int KG = 128 / RP;
    if (KG < 1) KG = 1;
    const int nt = KG * RP;
    size_t stage = (size_t)9 * op.nc * NRP * sizeof(cplx<T>);
    size_t reduce = (size_t)(KG + 1) * op.nc * NRP * sizeof(cplx<T>);
    size_t smem = stage > reduce ? stage : reduce;
    // set once per kernel instance (a function-local static initialiser is thread safe)
    static const bool attr = [] {
        cudaFuncSetAttribute(coarse_stencil_kernel<T, S, NRP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        return true;
    }();
    (void)attr;
    coarse_stencil_kernel<T, S, NRP><<<nsites, nt, smem, st>>>(op, site_begin, xin, xself, self_mode, hop_sign, apply_inv, out, nrhs);
    DD_CHECK_LAUNCH();
    return 0;
}

// batch of up to kMaxCoarseBatch right-hand sides per launch; larger batches are split
template <typename T, typename S>
static int launch_stencil(const CoarseOp<S>& op, int site_begin, int nsites, CVec<T> xin, CVec<T> xself, int self_mode,
                          T hop_sign, int apply_inv, CVec<T> out, int nrhs, cudaStream_t st) {
    while (nrhs > 0) {
        int n = nrhs;
        int rc;
        int cap = (sizeof(T) == 8 || op.nc > 48) ? 16 : 24;
        if (n > cap) n = cap;
        if (n == 1) rc = launch_stencil_nrp<T, S, 1>(op, site_begin, nsites, xin, xself, self_mode, hop_sign, apply_inv, out, n, st);
        else if (n == 2) rc = launch_stencil_nrp<T, S, 2>(op, site_begin, nsites, xin, xself, self_mode, hop_sign, apply_inv, out, n, st);
        else if (n <= 4) rc = launch_stencil_nrp<T, S, 4>(op, site_begin, nsites, xin, xself, self_mode, hop_sign, apply_inv, out, n, st);
        else if (n <= 8) rc = launch_stencil_nrp<T, S, 8>(op, site_begin, nsites, xin, xself, self_mode, hop_sign, apply_inv, out, n, st);
        else if (n <= 12) rc = launch_stencil_nrp<T, S, 12>(op, site_begin, nsites, xin, xself, self_mode, hop_sign, apply_inv, out, n, st);
        else if (n <= 16) rc = launch_stencil_nrp<T, S, 16>(op, site_begin, nsites, xin, xself, self_mode, hop_sign, apply_inv, out, n, st);
        else rc = launch_stencil_nrp<T, S, 24>(op, site_begin, nsites, xin, xself, self_mode, hop_sign, apply_inv, out, n, st);
        if (rc) return rc;
        nrhs -= n;
        xin.p += n * xin.rstride;
        xself.p += n * xself.rstride;
        out.p += n * out.rstride;
    }
    return 0;
}

// y = D_c x on full vectors [nrhs][NB][nc]
template <typename T, typename S>
int launch_coarse_full(const CoarseOp<S>& op, const cplx<T>* x, cplx<T>* y, int nrhs, cudaStream_t st) {
    size_t rs = (size_t)op.NB * op.nc;
    CVec<T> xv{const_cast<cplx<T>*>(x), rs, 0}, yv{y, rs, 0};
    return launch_stencil<T, S>(op, 0, op.NB, xv, xv, 1, T(1), 0, yv, nrhs, st);
}

// even sites: out_e = Dinv (b_e + beta * sum_d B_d x_o[nbr]) (b_e may be null: then 0).
// Each half vector is given by its pointer to the first even/odd site and its rhs stride.
template <typename T, typename S>
int launch_coarse_even(const CoarseOp<S>& op, const cplx<T>* b_e, size_t b_rs, const cplx<T>* x_o, size_t x_rs, T beta,
                       cplx<T>* out_e, size_t o_rs, int nrhs, cudaStream_t st) {
    const int H = op.NB / 2;
    CVec<T> xv{const_cast<cplx<T>*>(x_o ? x_o : out_e), x_o ? x_rs : o_rs, H};
    CVec<T> bv{const_cast<cplx<T>*>(b_e ? b_e : out_e), b_e ? b_rs : o_rs, 0};
    CVec<T> ov{out_e, o_rs, 0};
    return launch_stencil<T, S>(op, 0, H, xv, bv, b_e ? 2 : 0, x_o ? beta : T(0), 1, ov, nrhs, st);
}

// odd sites: out_o = (use_diag ? B_0 x_o : x_o) - sum_d B_d t_e[nbr]
template <typename T, typename S>
int launch_coarse_odd(const CoarseOp<S>& op, const cplx<T>* x_o, size_t x_rs, const cplx<T>* t_e, size_t t_rs, int use_diag,
                      cplx<T>* out_o, size_t o_rs, int nrhs, cudaStream_t st) {
    const int H = op.NB / 2;
    CVec<T> tv{const_cast<cplx<T>*>(t_e), t_rs, 0}, xv{const_cast<cplx<T>*>(x_o), x_rs, H}, ov{out_o, o_rs, H};
    return launch_stencil<T, S>(op, H, H, tv, xv, use_diag ? 1 : 2, T(-1), 0, ov, nrhs, st);
}

#define DD_INST_COARSE(T, S)                                                                                          \
    template int launch_coarse_full<T, S>(const CoarseOp<S>&, const cplx<T>*, cplx<T>*, int, cudaStream_t);           \
    template int launch_coarse_even<T, S>(const CoarseOp<S>&, const cplx<T>*, size_t, const cplx<T>*, size_t, T,      \
                                          cplx<T>*, size_t, int, cudaStream_t);                                       \
    template int launch_coarse_odd<T, S>(const CoarseOp<S>&, const cplx<T>*, size_t, const cplx<T>*, size_t, int,     \
                                         cplx<T>*, size_t, int, cudaStream_t);
DD_INST_COARSE(double, double)
DD_INST_COARSE(float, float)

// ---------------------------------------------------------------------------
// inverses of the diagonal blocks on even coarse sites: Gauss-Jordan with
// partial pivoting on [B_0 | I] in shared memory, FP64.  CTA = even site.
// ---------------------------------------------------------------------------
__global__ void coarse_invert_kernel(const cplx<double>* __restrict__ B, cplx<double>* __restrict__ Dinv, int nc,
                                     int* __restrict__ fail) {
    extern __shared__ unsigned char smem_raw[];
    cplx<double>* M = reinterpret_cast<cplx<double>*>(smem_raw);  // [nc][2nc] row-major
    __shared__ int piv_s;
    __shared__ cplx<double> pv_s;
    const int c = blockIdx.x;
    const int w2 = 2 * nc;
    const cplx<double>* B0 = B + (size_t)c * 9 * nc * nc;
    for (int q = threadIdx.x; q < nc * w2; q += blockDim.x) {
        int i = q / w2, j = q % w2;
        M[q] = (j < nc) ? B0[(size_t)j * nc + i] : mk(j - nc == i ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    for (int p = 0; p < nc; ++p) {
        if (threadIdx.x == 0) {
            int best = p;
            double bv = norm2(M[p * w2 + p]);
            for (int i = p + 1; i < nc; ++i)
                if (norm2(M[i * w2 + p]) > bv) {
                    bv = norm2(M[i * w2 + p]);
                    best = i;
                }
            if (!(bv > 0.0)) atomicExch(fail, 1);
            piv_s = best;
        }
        __syncthreads();
        const int pr = piv_s;
        if (pr != p)
            for (int j = threadIdx.x; j < w2; j += blockDim.x) {
                cplx<double> t = M[p * w2 + j];
                M[p * w2 + j] = M[pr * w2 + j];
                M[pr * w2 + j] = t;
            }
        __syncthreads();
        if (threadIdx.x == 0) {
            cplx<double> a = M[p * w2 + p];
            double dn = norm2(a);
            pv_s = dn > 0 ? mk(a.re / dn, -a.im / dn) : mk(0.0, 0.0);
        }
        __syncthreads();
        const cplx<double> inv = pv_s;
        for (int j = threadIdx.x; j < w2; j += blockDim.x) M[p * w2 + j] = M[p * w2 + j] * inv;
        __syncthreads();
        // eliminate column p from all other rows; factors read before any update
        for (int q = threadIdx.x; q < nc * w2; q += blockDim.x) {
            int i = q / w2, j = q % w2;
            if (i == p || j == p) continue;
            M[q] = M[q] - M[i * w2 + p] * M[p * w2 + j];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nc; i += blockDim.x)
            if (i != p) M[i * w2 + p] = mk(0.0, 0.0);
        __syncthreads();
    }
    cplx<double>* D = Dinv + (size_t)c * nc * nc;
    for (int q = threadIdx.x; q < nc * nc; q += blockDim.x) {
        int col = q / nc, row = q % nc;
        D[q] = M[row * w2 + nc + col];
    }
}

int launch_coarse_invert(const double* B, double* Dinv, int NB, int nc, int* fail, cudaStream_t st) {
    size_t smem = (size_t)nc * 2 * nc * sizeof(cplx<double>);
    cudaFuncSetAttribute(coarse_invert_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    coarse_invert_kernel<<<NB / 2, 256, smem, st>>>(reinterpret_cast<const cplx<double>*>(B), reinterpret_cast<cplx<double>*>(Dinv),
                                                   nc, fail);
    DD_CHECK_LAUNCH();
    return 0;
}

}  // namespace ddamg
