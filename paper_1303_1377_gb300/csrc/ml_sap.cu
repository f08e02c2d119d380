// Level-1 SAP colour step as one kernel (Sec. 2.3 and the odd-even MR block solver of Sec. 6,
// applied to D_1 = D_c on the lattice of the fine aggregates; the recursion of Sec. 3).
//
// One CTA per (level-1 block of the colour, group of up to 12 right-hand sides).  It forms the
// residual r = b - D_1 z on the block's sites, runs the MR steps on the block's odd-site Schur
// complement S = A_oo - A_oe A_ee^{-1} A_eo with every MR vector in shared memory, back-substitutes
// the even sites and adds the correction to z.  The same arithmetic as the functor sequence of
// ml_sap (ml_ops.cuh), which is kept for other shapes and for the host check; this kernel replaces
// its 27 launches per colour and their round trips of every MR vector through global memory.
//
// Thread (group h, slot s, row a) owns component a of the block's s-th even site and of its s-th odd
// site, for the right-hand sides 4h..4h+3 of the CTA (three groups: three times the warps of one
// thread per row, and a third of the accumulators per thread).  A block of D_1 is read by its nc row threads as one
// coalesced column per step (the second group finds it in L1); the vector it multiplies is read
// from shared memory, one broadcast per column and right-hand-side pair.
#include "kernels.h"
#include "ml_ops.cuh"

namespace ddamg {

namespace {

constexpr int kR = 12;  // right-hand sides per CTA
constexpr int kT = 4;   // right-hand sides per thread (kR / kT thread groups)
constexpr int kG = kR / kT;

// shared-memory vector of one half block: [slot][component][kR]
struct HalfVec {
    cplx<float>* p;
    int nc;
    __device__ __forceinline__ cplx<float>* at(int s, int a) const { return p + ((size_t)s * nc + a) * kR; }
};

// the operator's entries: FP32 complex, or FP16 (re, im) pairs on half-precision handles
template <bool H16>
struct OpRef {
    const void* B;
    const void* Dinv;
    __device__ __forceinline__ cplx<float> at(const void* base, size_t q) const {
        if constexpr (H16) {
            const float2 f = __half22float2(__ldg(reinterpret_cast<const __half2*>(base) + q));
            return mk(f.x, f.y);
        } else {
            return ldg_c(reinterpret_cast<const cplx<float>*>(base) + q);
        }
    }
};

// acc[j] += sum_col B[col][row] v[col][q0 + j] for the column-major nc x nc block at entry `first` of
// `base` (global) and the shared-memory vector v ([nc][kR]), j < kT
template <bool H16>
__device__ __forceinline__ void row_times(cplx<float> (&acc)[kT], const OpRef<H16>& op, const void* base, size_t first, int nc, int row,
                                          const cplx<float>* v, int q0, float sign = 1.f) {
    const size_t bp = first + row;
#pragma unroll 4
    for (int col = 0; col < nc; ++col) {
        const cplx<float> bv0 = op.at(base, bp + (size_t)col * nc);
        const cplx<float> bv = mk(sign * bv0.re, sign * bv0.im);
        const float4* v4 = reinterpret_cast<const float4*>(v + (size_t)col * kR + q0);
#pragma unroll
        for (int q = 0; q < kT / 2; ++q) {
            const float4 x = v4[q];
            cmac(acc[2 * q], bv, mk(x.x, x.y));
            cmac(acc[2 * q + 1], bv, mk(x.z, x.w));
        }
    }
}

__device__ __forceinline__ void zero(cplx<float> (&acc)[kT]) {
#pragma unroll
    for (int r = 0; r < kT; ++r) acc[r] = czero<float>();
}

}  // namespace

template <bool H16>
__global__ void __launch_bounds__(1024, 1) ml_sap_fused_kernel(MLView<float> v, const cplx<float>* __restrict__ b,
                                                              cplx<float>* __restrict__ z, int nrhs, int colour, int mr_steps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nc = v.nc, He = v.Vb1e, Vb = v.Vb1;
    const size_t fs = (size_t)v.NB * nc;
    const int c2 = colour * (v.NB2 / 2) + blockIdx.x;
    const int r0 = blockIdx.y * kR;
    const int nr = min(kR, nrhs - r0);
    const int t = threadIdx.x;
    const bool act = t < kG * He * nc;
    const int hg = act ? t / (He * nc) : 0, tt = act ? t % (He * nc) : 0;
    const int s = tt / nc, row = tt % nc;
    const int q0 = hg * kT;  // this thread's first right-hand side within the CTA
    const OpRef<H16> op{H16 ? v.B1h : (const void*)v.B1, H16 ? v.Dinv1h : (const void*)v.Dinv1};
    const size_t nn = (size_t)nc * nc;
    auto blk = [&](int c, int d) { return ((size_t)c * 9 + d) * nn; };  // first entry of block d of site c

    // shared memory: six half-block vectors, site tables, MR step sizes
    const size_t hv = (size_t)He * nc * kR;
    cplx<float>* base = reinterpret_cast<cplx<float>*>(smem_raw);
    const HalfVec Re{base, nc}, Te{base + hv, nc}, Rho{base + 2 * hv, nc}, Xo{base + 3 * hv, nc}, So{base + 4 * hv, nc},
        Stg{base + 5 * hv, nc};
    cplx<float>* alpha = base + 6 * hv;                              // [kR]
    int* site = reinterpret_cast<int*>(alpha + kR);                  // [Vb] level-1 site of local index l
    int* nbl = site + Vb;                                            // [Vb][8] local index of the in-block neighbour, or -1

    for (int l = t; l < Vb; l += blockDim.x) site[l] = v.sites[(size_t)c2 * Vb + l];
    __syncthreads();
    for (int q = t; q < Vb * 8; q += blockDim.x) {
        const int l = q / 8, d = q % 8, c = site[l];
        nbl[q] = v.same[(size_t)d * v.NB + c] ? v.loc_of[v.nbr1[(size_t)d * v.NB + c]] : -1;
    }
    __syncthreads();
    const int ce = site[s], co = site[He + s];  // this thread's even and odd site

    cplx<float> acc[kT];
    // ---- residual r = b - D_1 z on the even (pass 0) and odd (pass 1) sites of the block; z of
    // out-of-block neighbours belongs to blocks of the other colour, which this launch leaves alone
    for (int pass = 0; pass < 2; ++pass) {
        const int off = pass ? He : 0;
        zero(acc);
        for (int d = 0; d < 9; ++d) {
            for (int q = t; q < He * kR * nc; q += blockDim.x) {  // Stg[ss][col][r] = z at the d-neighbour of site off + ss
                const int col = q % nc, r = (q / nc) % kR, ss = q / (nc * kR);
                const int c = site[off + ss];
                const int n = d == 0 ? c : v.nbr1[(size_t)(d - 1) * v.NB + c];
                Stg.at(ss, col)[r] = r < nr ? z[(size_t)(r0 + r) * fs + (size_t)n * nc + col] : czero<float>();
            }
            __syncthreads();
            if (act) row_times(acc, op, op.B, blk(pass ? co : ce, d), nc, row, Stg.at(s, 0), q0);
            __syncthreads();
        }
        if (act) {
            const HalfVec& dst = pass ? So : Re;  // r_o parks in So until rho is formed
            const int c = pass ? co : ce;
            cplx<float>* o = dst.at(s, row) + q0;
#pragma unroll
            for (int j = 0; j < kT; ++j)
                o[j] = q0 + j < nr ? b[(size_t)(r0 + q0 + j) * fs + (size_t)c * nc + row] - acc[j] : czero<float>();
        }
    }
    __syncthreads();
    // ---- t_e = A_ee^{-1} r_e
    if (act) {
        zero(acc);
        row_times(acc, op, op.Dinv, (size_t)ce * nn, nc, row, Re.at(s, 0), q0);
        cplx<float>* o = Te.at(s, row) + q0;
#pragma unroll
        for (int j = 0; j < kT; ++j) o[j] = acc[j];
    }
    __syncthreads();
    // ---- rho = r_o - A_oe t_e; x_o = 0
    if (act) {
        zero(acc);
        for (int d = 0; d < 8; ++d) {
            const int n = nbl[(He + s) * 8 + d];
            if (n >= 0) row_times(acc, op, op.B, blk(co, 1 + d), nc, row, Te.at(n, 0), q0, -1.f);
        }
        const cplx<float>* ro = So.at(s, row) + q0;
        cplx<float>* o = Rho.at(s, row) + q0;
        cplx<float>* xo = Xo.at(s, row) + q0;
#pragma unroll
        for (int j = 0; j < kT; ++j) {
            o[j] = ro[j] + acc[j];
            xo[j] = czero<float>();
        }
    }
    __syncthreads();
    // ---- MR steps on S rho
    for (int it = 0; it < mr_steps; ++it) {
        if (act) {  // u_e = A_eo rho (parked in So)
            zero(acc);
            for (int d = 0; d < 8; ++d) {
                const int n = nbl[s * 8 + d];
                if (n >= 0) row_times(acc, op, op.B, blk(ce, 1 + d), nc, row, Rho.at(n - He, 0), q0);
            }
            cplx<float>* o = So.at(s, row) + q0;
#pragma unroll
            for (int j = 0; j < kT; ++j) o[j] = acc[j];
        }
        __syncthreads();
        if (act) {  // t_e = A_ee^{-1} u_e
            zero(acc);
            row_times(acc, op, op.Dinv, (size_t)ce * nn, nc, row, So.at(s, 0), q0);
            cplx<float>* o = Te.at(s, row) + q0;
#pragma unroll
            for (int j = 0; j < kT; ++j) o[j] = acc[j];
        }
        __syncthreads();
        if (act) {  // s_o = A_oo rho - A_oe t_e
            zero(acc);
            row_times(acc, op, op.B, blk(co, 0), nc, row, Rho.at(s, 0), q0);
            for (int d = 0; d < 8; ++d) {
                const int n = nbl[(He + s) * 8 + d];
                if (n >= 0) row_times(acc, op, op.B, blk(co, 1 + d), nc, row, Te.at(n, 0), q0, -1.f);
            }
            cplx<float>* o = So.at(s, row) + q0;
#pragma unroll
            for (int j = 0; j < kT; ++j) o[j] = acc[j];
        }
        __syncthreads();
        {  // alpha_r = <s, rho> / <s, s> over the block's odd sites: warp w sums right-hand side r = w, w + nwarps, ...
            const int w = t >> 5, lane = t & 31, nw = blockDim.x >> 5;
            for (int r = w; r < kR; r += nw) {
                float nre = 0.f, nim = 0.f, den = 0.f;
                for (int q = lane; q < He * nc; q += 32) {
                    const cplx<float> sv = So.p[(size_t)q * kR + r], rv = Rho.p[(size_t)q * kR + r];
                    nre += sv.re * rv.re + sv.im * rv.im;
                    nim += sv.re * rv.im - sv.im * rv.re;
                    den += sv.re * sv.re + sv.im * sv.im;
                }
                nre = warp_sum(nre);
                nim = warp_sum(nim);
                den = warp_sum(den);
                if (lane == 0) alpha[r] = den > ml_den_floor<float>() ? mk(nre / den, nim / den) : czero<float>();
            }
        }
        __syncthreads();
        if (act) {  // x_o += alpha rho; rho -= alpha s
            cplx<float>* xo = Xo.at(s, row) + q0;
            cplx<float>* ro = Rho.at(s, row) + q0;
            const cplx<float>* so = So.at(s, row) + q0;
#pragma unroll
            for (int j = 0; j < kT; ++j) {
                const cplx<float> a = alpha[q0 + j];
                cmac(xo[j], a, ro[j]);
                ro[j] = ro[j] - a * so[j];
            }
        }
        __syncthreads();
    }
    // ---- x_e = A_ee^{-1} (r_e - A_eo x_o); z += x on the block
    if (act) {
        zero(acc);
        for (int d = 0; d < 8; ++d) {
            const int n = nbl[s * 8 + d];
            if (n >= 0) row_times(acc, op, op.B, blk(ce, 1 + d), nc, row, Xo.at(n - He, 0), q0, -1.f);
        }
        const cplx<float>* re = Re.at(s, row) + q0;
        cplx<float>* o = So.at(s, row) + q0;
#pragma unroll
        for (int j = 0; j < kT; ++j) o[j] = re[j] + acc[j];
    }
    __syncthreads();
    if (act) {
        zero(acc);
        row_times(acc, op, op.Dinv, (size_t)ce * nn, nc, row, So.at(s, 0), q0);
        const cplx<float>* xo = Xo.at(s, row) + q0;
#pragma unroll
        for (int j = 0; j < kT; ++j) {
            if (q0 + j < nr) {
                cplx<float>* ze = z + (size_t)(r0 + q0 + j) * fs + (size_t)ce * nc + row;
                cplx<float>* zo = z + (size_t)(r0 + q0 + j) * fs + (size_t)co * nc + row;
                *ze = *ze + acc[j];
                *zo = *zo + xo[j];
            }
        }
    }
}

static size_t ml_sap_fused_smem(const MLView<float>& v) {
    return (size_t)6 * v.Vb1e * v.nc * kR * sizeof(cplx<float>) + kR * sizeof(cplx<float>) + (size_t)v.Vb1 * 9 * sizeof(int);
}

bool ml_sap_fused_supported(const MLView<float>& v) {
    return v.Vb1 == 2 * v.Vb1e && kG * v.Vb1e * v.nc <= 1024 && v.nc % 2 == 0 && ml_sap_fused_smem(v) <= 227 * 1024;
}

int launch_ml_sap_fused(const MLView<float>& v, const cplx<float>* b, cplx<float>* z, int nrhs, int colour, int mr_steps,
                        cudaStream_t st) {
    const size_t smem = ml_sap_fused_smem(v);
    static const bool attr = [] {
        cudaFuncSetAttribute(ml_sap_fused_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        cudaFuncSetAttribute(ml_sap_fused_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        return true;
    }();
    (void)attr;
    const int threads = ((kG * v.Vb1e * v.nc + 31) / 32) * 32;
    const dim3 grid((unsigned)(v.NB2 / 2), (unsigned)((nrhs + kR - 1) / kR));
    if (v.B1h && v.Dinv1h)
        ml_sap_fused_kernel<true><<<grid, threads, smem, st>>>(v, b, z, nrhs, colour, mr_steps);
    else
        ml_sap_fused_kernel<false><<<grid, threads, smem, st>>>(v, b, z, nrhs, colour, mr_steps);
    DD_CHECK_LAUNCH();
    return 0;
}

}  // namespace ddamg
