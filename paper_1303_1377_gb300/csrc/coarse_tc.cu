// Coarse stencil on tensor cores with FP16 storage and FP32 accumulation (the
// half-precision mode of the V-cycle).  For one coarse site c the operator is
// y = sum_d B_d(c) x_{c+d} (Sec. 3.2).  Complex blocks are written as two real
// planes, A_c = [Re B ; Im B] (2nc rows), and the right-hand sides as two real
// column groups [Re X | Im X]; one real GEMM P = A_c X gives
//   Re y = P[0:nc, 0:NR] - P[nc:2nc, NR:2NR],  Im y = P[nc:2nc, 0:NR] + P[0:nc, NR:2NR],
// so the complex matrix is stored once (2 halves per entry) without the 2x2
// real embedding.  The nine directions are stacked along K, the eight hops first
// (8 nc columns: a multiple of 16 for any N) and the self block last, so the
// Schur-complement kernels that use only the hops read a 16-aligned K range.
//
// Storage: A_c is pre-arranged in the register-fragment order of
// mma.sync.m16n8k16 (A row-major): for each (m-tile, k-tile) the 32 lanes' four
// 32-bit registers are 512 contiguous bytes, so each warp streams the matrix
// with one coalesced 16-byte load per lane and k-tile.  The right-hand sides are
// staged in shared memory as FP16 (k contiguous per column).
//
// Why mma.sync here: each coarse site owns a distinct 2nc x 9nc matrix (M = 80
// rows at N_v = 20) multiplied by a thin 9nc x 2 n_rhs block, and the kernel
// streams every matrix byte once, so it is bound by HBM.  A warp-level m16
// tile matches the 80-row per-site blocks without padding.
#include <cuda_fp16.h>

#include "bulk.cuh"
#include "kernels.h"

namespace ddamg {

__device__ __forceinline__ __half elem_of(const double* M, size_t base, int nc, int m, int col) {
    // M: complex column-major nc x nc block at base (doubles), m < nc: real plane, else imaginary plane
    int row = m < nc ? m : m - nc;
    return __float2half_rn((float)M[base + 2 * ((size_t)col * nc + row) + (m < nc ? 0 : 1)]);
}

__device__ __forceinline__ unsigned pack2(__half lo, __half hi) {
    __half2 v = __halves2half2(lo, hi);
    return *reinterpret_cast<unsigned*>(&v);
}

// A_c[m][kk] for the stencil matrix
__device__ __forceinline__ __half stencil_elem(const double* B64, int c, int nc, int m, int kk) {
    int d, col;
    if (kk < 8 * nc) {
        d = 1 + kk / nc;
        col = kk % nc;
    } else if (kk < 9 * nc) {
        d = 0;
        col = kk - 8 * nc;
    } else {
        return __float2half_rn(0.f);
    }
    return elem_of(B64, (((size_t)c * 9 + d) * nc) * nc * 2, nc, m, col);
}

__global__ void pack_stencil_kernel(const double* __restrict__ B64, uint4* __restrict__ Bh, int NB, int nc, int Mt, int Kt) {
    const size_t tot = (size_t)NB * Mt * Kt * 32;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
        int L = (int)(q % 32);
        int kt = (int)((q / 32) % Kt);
        int mt = (int)((q / 32 / Kt) % Mt);
        int c = (int)(q / ((size_t)32 * Kt * Mt));
        int g = L >> 2, t = L & 3;
        int r0 = mt * 16 + g, r1 = r0 + 8, k0 = kt * 16 + 2 * t, k1 = k0 + 8;
        uint4 v;
        v.x = pack2(stencil_elem(B64, c, nc, r0, k0), stencil_elem(B64, c, nc, r0, k0 + 1));
        v.y = pack2(stencil_elem(B64, c, nc, r1, k0), stencil_elem(B64, c, nc, r1, k0 + 1));
        v.z = pack2(stencil_elem(B64, c, nc, r0, k1), stencil_elem(B64, c, nc, r0, k1 + 1));
        v.w = pack2(stencil_elem(B64, c, nc, r1, k1), stencil_elem(B64, c, nc, r1, k1 + 1));
        Bh[q] = v;
    }
}

__device__ __forceinline__ __half dinv_elem(const double* D64, int c, int nc, int m, int kk) {
    if (kk >= nc) return __float2half_rn(0.f);
    return elem_of(D64, (size_t)c * nc * nc * 2, nc, m, kk);
}

__global__ void pack_dinv_kernel(const double* __restrict__ D64, uint4* __restrict__ Dh, int NH, int nc, int Mt, int Kt) {
    const size_t tot = (size_t)NH * Mt * Kt * 32;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
        int L = (int)(q % 32);
        int kt = (int)((q / 32) % Kt);
        int mt = (int)((q / 32 / Kt) % Mt);
        int c = (int)(q / ((size_t)32 * Kt * Mt));
        int g = L >> 2, t = L & 3;
        int r0 = mt * 16 + g, r1 = r0 + 8, k0 = kt * 16 + 2 * t, k1 = k0 + 8;
        uint4 v;
        v.x = pack2(dinv_elem(D64, c, nc, r0, k0), dinv_elem(D64, c, nc, r0, k0 + 1));
        v.y = pack2(dinv_elem(D64, c, nc, r1, k0), dinv_elem(D64, c, nc, r1, k0 + 1));
        v.z = pack2(dinv_elem(D64, c, nc, r0, k1), dinv_elem(D64, c, nc, r0, k1 + 1));
        v.w = pack2(dinv_elem(D64, c, nc, r1, k1), dinv_elem(D64, c, nc, r1, k1 + 1));
        Dh[q] = v;
    }
}

int tc_dims(int nc, int* Mt, int* Kt_all, int* Kt_hops, int* Kt_d) {
    if (nc % 8) return DDAMG_ERR_INVALID_ARG;
    *Mt = nc / 8;
    *Kt_hops = (8 * nc) / 16;
    *Kt_d = (nc + 15) / 16;
    *Kt_all = *Kt_hops + *Kt_d;
    return 0;
}

int pack_coarse_tc(const double* B64, const double* Dinv64, uint4* Bh, uint4* Dh, int NB, int nc, cudaStream_t st) {
    int Mt, Kta, Kth, Ktd;
    if (tc_dims(nc, &Mt, &Kta, &Kth, &Ktd)) {
        set_error("half precision needs 2N divisible by 8");
        return DDAMG_ERR_INVALID_ARG;
    }
    pack_stencil_kernel<<<152 * 8, 256, 0, st>>>(B64, Bh, NB, nc, Mt, Kta);
    DD_CHECK_LAUNCH();
    pack_dinv_kernel<<<152 * 8, 256, 0, st>>>(Dinv64, Dh, NB / 2, nc, Mt, Ktd);
    DD_CHECK_LAUNCH();
    return 0;
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint4& a, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

template <typename T>
struct CVecT {
    cplx<T>* p;
    size_t rstride;
    int site0;
};

// One CTA per coarse site with two warps per m-tile: warp w < Mt owns m-tile w (rows 16w..16w+15 of
// [Re; Im]) in the tensor-core product; all 2 Mt warps gather and convert the right-hand sides and
// write the result.
// SPLIT: each right-hand-side entry x is staged as two FP16 numbers, hi = fp16(x) and
// lo = fp16(2^11 (x - hi)), and multiplied by both (P = A hi + 2^-11 A lo), so the product is that of
// the FP16-rounded matrix with x to about 2^-22 relative instead of 2^-11.  The operator then stays
// one fixed linear map, which a Krylov solver on an ill-conditioned coarsest level needs: with the
// inputs rounded to FP16 its residual estimate and the true residual drift apart.
//   acc = self + hop_sign * sum_{d=1..8} B_d(c) xin[nbr_d(c)]; self = 0 / B_0 xself / xself;
//   out = apply_inv ? Dinv acc : acc       (same modes as the CUDA-core kernel)
// The site's FP16 matrix (the k-tiles this call uses, and D_ee^{-1} when applied) is brought into
// shared memory by bulk copies issued first, so that HBM streams it while the CTA gathers the
// right-hand sides of the neighbouring sites (L2 hits) and converts them to FP16.
constexpr float kLoScale = 2048.f;  // 2^11: the low FP16 part of a split entry, scaled into the normal range

// x -> (hi, lo) for the SPLIT staging of two values
__device__ __forceinline__ void split_half2(float a, float b, __half2& hi, __half2& lo) {
    hi = __floats2half2_rn(a, b);
    const float2 h = __half22float2(hi);
    lo = __floats2half2_rn((a - h.x) * kLoScale, (b - h.y) * kLoScale);
}

template <int NRP, bool SPLIT>
__global__ void __launch_bounds__(512, 2) coarse_tc_kernel(CoarseTC op, int site_begin, CVecT<float> xin, CVecT<float> xself, int self_mode,
                                                          float hop_sign, int apply_inv, CVecT<float> out, int nrhs) {
    constexpr int NT = NRP / 4;  // n-tiles of 8 columns over [Re X | Im X] (2 NRP columns)
    constexpr int NPL = SPLIT ? 2 : 1;  // staged planes: hi (and lo)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nc = op.nc, Mt = op.Mt;
    const int Kp = op.Kt_all * 16;
    const int LDX = Kp + 8;  // halves per staged column (bank offset)
    const bool hops = hop_sign != 0.f;
    const int kt0 = hops ? 0 : op.Kt_hops;
    const int kt1 = self_mode == 1 ? op.Kt_all : op.Kt_hops;
    const int nkt = kt1 - kt0;
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw);
    int* snb = reinterpret_cast<int*>(smem_raw + 8);                       // [8] neighbouring sites
    uint4* As = reinterpret_cast<uint4*>(smem_raw + 64);                    // [Mt][nkt][32]
    uint4* Ds = As + (size_t)Mt * nkt * 32;                                 // [Mt][Kt_d][32]
    __half* XT = reinterpret_cast<__half*>(Ds + (apply_inv ? (size_t)Mt * op.Kt_d * 32 : 0));  // [NPL][2 NRP][LDX]
    __half* XL = XT + (size_t)2 * NRP * LDX;                                // the lo plane (SPLIT)
    float* Cs = reinterpret_cast<float*>(XT + (size_t)NPL * 2 * NRP * LDX);  // [2nc][2 NRP]
    cplx<float>* Vs = reinterpret_cast<cplx<float>*>(Cs + (size_t)2 * nc * 2 * NRP);  // [nc][NRP]
    const int c = site_begin + blockIdx.x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    if (threadIdx.x == 0) mbar_init(bar, 1);
    if (threadIdx.x < 8) snb[threadIdx.x] = __ldg(op.cnbr + threadIdx.x * op.NB + c);
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned abytes = (unsigned)nkt * 512u, dbytes = apply_inv ? (unsigned)(Mt * op.Kt_d) * 512u : 0u;
        mbar_arrive_expect_tx(bar, abytes * Mt + dbytes);
        if (abytes)
            for (int m = 0; m < Mt; ++m)
                bulk_g2s(As + (size_t)m * nkt * 32, op.Bh + (((size_t)c * Mt + m) * op.Kt_all + kt0) * 32, abytes, bar);
        if (dbytes) bulk_g2s(Ds, op.Dh + ((size_t)c * Mt * op.Kt_d) * 32, dbytes, bar);
    }
    // 1. stage [Re X | Im X]^T for the used K range, two complex entries (one float4) at a time; the
    //    loads of a batch are all issued before the first conversion, so their latencies overlap
    {
        constexpr int GB = 8;
        const int k0 = kt0 * 16, kh = nkt * 8, tot = NRP * kh;
        for (int q0 = 0; q0 < tot; q0 += GB * blockDim.x) {
            float4 v[GB];
#pragma unroll
            for (int j = 0; j < GB; ++j) {
                const int q = q0 + j * blockDim.x + threadIdx.x;
                v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (q < tot) {
                    const int kk = k0 + 2 * (q % kh), r = q / kh;
                    if (r < nrhs) {
                        if (kk < 8 * nc) {
                            const int d = kk / nc, col = kk - d * nc;  // nc even: kk, kk + 1 share the direction
                            v[j] = __ldg(reinterpret_cast<const float4*>(xin.p + r * xin.rstride + (size_t)(snb[d] - xin.site0) * nc + col));
                        } else if (kk < 9 * nc && self_mode == 1) {
                            v[j] = __ldg(reinterpret_cast<const float4*>(xself.p + r * xself.rstride + (size_t)(c - xself.site0) * nc +
                                                                         (kk - 8 * nc)));
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < GB; ++j) {
                const int q = q0 + j * blockDim.x + threadIdx.x;
                if (q < tot) {
                    const int kk = k0 + 2 * (q % kh), r = q / kh;
                    const float sg = kk < 8 * nc ? hop_sign : 1.f;
                    if constexpr (SPLIT) {
                        __half2 h, l;
                        split_half2(sg * v[j].x, sg * v[j].z, h, l);
                        *reinterpret_cast<__half2*>(XT + (size_t)r * LDX + kk) = h;
                        *reinterpret_cast<__half2*>(XL + (size_t)r * LDX + kk) = l;
                        split_half2(sg * v[j].y, sg * v[j].w, h, l);
                        *reinterpret_cast<__half2*>(XT + (size_t)(NRP + r) * LDX + kk) = h;
                        *reinterpret_cast<__half2*>(XL + (size_t)(NRP + r) * LDX + kk) = l;
                    } else {
                        *reinterpret_cast<__half2*>(XT + (size_t)r * LDX + kk) = __floats2half2_rn(sg * v[j].x, sg * v[j].z);
                        *reinterpret_cast<__half2*>(XT + (size_t)(NRP + r) * LDX + kk) = __floats2half2_rn(sg * v[j].y, sg * v[j].w);
                    }
                }
            }
        }
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(!ok)) {  // the copy never completed: flag it, let it drain, leave
        if (threadIdx.x == 0) {
            atomicExch(op.err, 1);
            mbar_wait_bounded(bar, 0);
        }
        return;
    }
    float acc[NT][4], acl[NT][4];
#pragma unroll
    for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = acl[n][0] = acl[n][1] = acl[n][2] = acl[n][3] = 0.f;
    const bool mma_warp = w < Mt;
    // P += A X for the A fragments in As (k-tiles [ka, kb), staged columns from kx0 on); the lo plane
    // goes to acl and is folded in by fold()
    auto gemm = [&](const uint4* Ab, int nk, int kx0) {
#pragma unroll 4
        for (int kt = 0; kt < nk; ++kt) {
            const uint4 a = Ab[(size_t)kt * 32];
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const size_t xo = (size_t)(n * 8 + g) * LDX + (kx0 + kt) * 16 + 2 * t;
                mma16816(acc[n], a, *reinterpret_cast<const unsigned*>(XT + xo), *reinterpret_cast<const unsigned*>(XT + xo + 8));
                if constexpr (SPLIT)
                    mma16816(acl[n], a, *reinterpret_cast<const unsigned*>(XL + xo), *reinterpret_cast<const unsigned*>(XL + xo + 8));
            }
        }
    };
    auto fold = [&]() {
        if constexpr (SPLIT) {
#pragma unroll
            for (int n = 0; n < NT; ++n)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    acc[n][i] += acl[n][i] * (1.f / kLoScale);
                    acl[n][i] = 0.f;
                }
        }
    };
    if (mma_warp) {
        gemm(As + (size_t)w * nkt * 32 + lane, nkt, kt0);
        fold();
    }
    // 2. recombine the planes into complex rows (+ identity self term)
    auto store_acc = [&]() {
        if (!mma_warp) return;
#pragma unroll
        for (int n = 0; n < NT; ++n) {
            int r0 = w * 16 + g, col = n * 8 + 2 * t;
            Cs[(size_t)r0 * 2 * NRP + col] = acc[n][0];
            Cs[(size_t)r0 * 2 * NRP + col + 1] = acc[n][1];
            Cs[(size_t)(r0 + 8) * 2 * NRP + col] = acc[n][2];
            Cs[(size_t)(r0 + 8) * 2 * NRP + col + 1] = acc[n][3];
        }
    };
    store_acc();
    __syncthreads();
    for (int q = threadIdx.x; q < nc * NRP; q += blockDim.x) {
        int row = q / NRP, r = q % NRP;
        float re = Cs[(size_t)row * 2 * NRP + r] - Cs[(size_t)(nc + row) * 2 * NRP + NRP + r];
        float im = Cs[(size_t)(nc + row) * 2 * NRP + r] + Cs[(size_t)row * 2 * NRP + NRP + r];
        cplx<float> v = mk(re, im);
        if (self_mode == 2 && r < nrhs) v = v + xself.p[r * xself.rstride + (size_t)(c - xself.site0) * nc + row];
        Vs[q] = v;
    }
    __syncthreads();
    if (apply_inv) {
        const int Kd = op.Kt_d * 16;
        for (int q = threadIdx.x; q < NRP * Kd; q += blockDim.x) {
            int kk = q % Kd, r = q / Kd;
            cplx<float> v = kk < nc ? Vs[kk * NRP + r] : czero<float>();
            const __half hr = __float2half_rn(v.re), hi = __float2half_rn(v.im);
            XT[(size_t)r * LDX + kk] = hr;
            XT[(size_t)(NRP + r) * LDX + kk] = hi;
            if constexpr (SPLIT) {
                XL[(size_t)r * LDX + kk] = __float2half_rn((v.re - __half2float(hr)) * kLoScale);
                XL[(size_t)(NRP + r) * LDX + kk] = __float2half_rn((v.im - __half2float(hi)) * kLoScale);
            }
        }
        __syncthreads();
#pragma unroll
        for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
        if (mma_warp) {
            gemm(Ds + (size_t)w * op.Kt_d * 32 + lane, op.Kt_d, 0);
            fold();
        }
        store_acc();
        __syncthreads();
        for (int q = threadIdx.x; q < nc * NRP; q += blockDim.x) {
            int row = q / NRP, r = q % NRP;
            float re = Cs[(size_t)row * 2 * NRP + r] - Cs[(size_t)(nc + row) * 2 * NRP + NRP + r];
            float im = Cs[(size_t)(nc + row) * 2 * NRP + r] + Cs[(size_t)row * 2 * NRP + NRP + r];
            Vs[q] = mk(re, im);
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < nc * NRP; q += blockDim.x) {
        int row = q / NRP, r = q % NRP;
        if (r < nrhs) out.p[r * out.rstride + (size_t)(c - out.site0) * nc + row] = Vs[q];
    }
}

// dynamic shared memory of coarse_tc_kernel<NRP> for one call
static size_t tc_smem(const CoarseTC& op, int nrp, int self_mode, float hop_sign, int apply_inv) {
    const int Kp = op.Kt_all * 16;
    const int nkt = (self_mode == 1 ? op.Kt_all : op.Kt_hops) - (hop_sign != 0.f ? 0 : op.Kt_hops);
    return 64 + (size_t)op.Mt * (nkt + (apply_inv ? op.Kt_d : 0)) * 512 + (size_t)(op.split ? 2 : 1) * 2 * nrp * (Kp + 8) * sizeof(__half) +
           (size_t)2 * op.nc * 2 * nrp * sizeof(float) + (size_t)op.nc * nrp * sizeof(cplx<float>);
}
constexpr size_t kTcSmemMax = 227 * 1024;

template <int NRP>
static int launch_tc_nrp(const CoarseTC& op, int site_begin, int nsites, CVecT<float> xin, CVecT<float> xself, int self_mode,
                         float hop_sign, int apply_inv, CVecT<float> out, int nrhs, cudaStream_t st) {
    const size_t smem = tc_smem(op, NRP, self_mode, hop_sign, apply_inv);
    // set once per kernel instance (a function-local static initialiser is thread safe)
    static const bool attr = [] {
        cudaFuncSetAttribute(coarse_tc_kernel<NRP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax);
        if constexpr (NRP <= 12) cudaFuncSetAttribute(coarse_tc_kernel<NRP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax);
        return true;
    }();
    (void)attr;
    if constexpr (NRP <= 12) {  // split staging: at most 12 right-hand sides per launch (no register spills)
        if (op.split) {
            coarse_tc_kernel<NRP, true><<<nsites, 64 * op.Mt, smem, st>>>(op, site_begin, xin, xself, self_mode, hop_sign, apply_inv, out,
                                                                          nrhs);
            DD_CHECK_LAUNCH();
            return 0;
        }
    }
    coarse_tc_kernel<NRP, false><<<nsites, 64 * op.Mt, smem, st>>>(op, site_begin, xin, xself, self_mode, hop_sign, apply_inv, out, nrhs);
    DD_CHECK_LAUNCH();
    return 0;
}

static int launch_tc(const CoarseTC& op, int site_begin, int nsites, CVecT<float> xin, CVecT<float> xself, int self_mode,
                     float hop_sign, int apply_inv, CVecT<float> out, int nrhs, cudaStream_t st) {
    // right-hand sides per launch: up to 24, fewer where the site's matrix and the staged vectors
    // would not fit in shared memory
    int cap = op.split ? 12 : 24;
    while (cap > 4 && tc_smem(op, cap, self_mode, hop_sign, apply_inv) > kTcSmemMax) cap = cap > 16 ? 16 : cap > 12 ? 12 : cap - 4;
    if (tc_smem(op, 4, self_mode, hop_sign, apply_inv) > kTcSmemMax) {
        set_error("coarse stencil: the per-site FP16 matrix does not fit in shared memory (2N too large for half precision)");
        return DDAMG_ERR_INVALID_ARG;
    }
    while (nrhs > 0) {
        int n = nrhs > cap ? cap : nrhs;
        int rc;
        if (n <= 4) rc = launch_tc_nrp<4>(op, site_begin, nsites, xin, xself, self_mode, hop_sign, apply_inv, out, n, st);
        else if (n <= 8) rc = launch_tc_nrp<8>(op, site_begin, nsites, xin, xself, self_mode, hop_sign, apply_inv, out, n, st);
        else if (n <= 12) rc = launch_tc_nrp<12>(op, site_begin, nsites, xin, xself, self_mode, hop_sign, apply_inv, out, n, st);
        else if (n <= 16) rc = launch_tc_nrp<16>(op, site_begin, nsites, xin, xself, self_mode, hop_sign, apply_inv, out, n, st);
        else rc = launch_tc_nrp<24>(op, site_begin, nsites, xin, xself, self_mode, hop_sign, apply_inv, out, n, st);
        if (rc) return rc;
        nrhs -= n;
        xin.p += n * xin.rstride;
        xself.p += n * xself.rstride;
        out.p += n * out.rstride;
    }
    return 0;
}

int tc_coarse_full(const CoarseTC& op, const cplx<float>* x, cplx<float>* y, int nrhs, cudaStream_t st) {
    size_t rs = (size_t)op.NB * op.nc;
    CVecT<float> xv{const_cast<cplx<float>*>(x), rs, 0}, yv{y, rs, 0};
    return launch_tc(op, 0, op.NB, xv, xv, 1, 1.f, 0, yv, nrhs, st);
}

int tc_coarse_even(const CoarseTC& op, const cplx<float>* b_e, size_t b_rs, const cplx<float>* x_o, size_t x_rs, float beta,
                   cplx<float>* out_e, size_t o_rs, int nrhs, cudaStream_t st) {
    const int H = op.NB / 2;
    CVecT<float> xv{const_cast<cplx<float>*>(x_o ? x_o : out_e), x_o ? x_rs : o_rs, H};
    CVecT<float> bv{const_cast<cplx<float>*>(b_e ? b_e : out_e), b_e ? b_rs : o_rs, 0};
    CVecT<float> ov{out_e, o_rs, 0};
    return launch_tc(op, 0, H, xv, bv, b_e ? 2 : 0, x_o ? beta : 0.f, 1, ov, nrhs, st);
}

int tc_coarse_odd(const CoarseTC& op, const cplx<float>* x_o, size_t x_rs, const cplx<float>* t_e, size_t t_rs, int use_diag,
                  cplx<float>* out_o, size_t o_rs, int nrhs, cudaStream_t st) {
    const int H = op.NB / 2;
    CVecT<float> tv{const_cast<cplx<float>*>(t_e), t_rs, 0}, xv{const_cast<cplx<float>*>(x_o), x_rs, H}, ov{out_o, o_rs, H};
    return launch_tc(op, H, H, tv, xv, use_diag ? 1 : 2, -1.f, 0, ov, nrhs, st);
}

// P (FP64) -> FP16 copy for the half-precision restriction / prolongation
__global__ void to_half_kernel(const double* __restrict__ in, __half* __restrict__ out, size_t n) {
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        out[q] = __float2half_rn((float)in[q]);
}
int convert_to_half(const double* in, void* out, size_t n, cudaStream_t st) {
    int blocks = ceil_div((long long)n, 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    to_half_kernel<<<blocks, 256, 0, st>>>(in, reinterpret_cast<__half*>(out), n);
    DD_CHECK_LAUNCH();
    return 0;
}

}  // namespace ddamg
