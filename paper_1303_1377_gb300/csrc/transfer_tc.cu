// Prolongation on tensor cores for the half-precision V-cycle (Sec. 3.1):
//   y[r][k][x] = sum_j P_j[k][x] e[r][c(x)][h(k) N + j]
// For one aggregate half (block c, spins {2h, 2h+1}) this is a complex product
// Y (6 Vb x n_rhs) = P_{c,h} (6 Vb x N) E_{c,h} (N x n_rhs).  It runs as real
// mma.sync.m16n8k16 products (FP16 operands, FP32 accumulation):
//   A: 16 sites of one spin-colour component k, K = j (N padded to 32); the real
//      and the imaginary plane of P are two A tiles of the same rows;
//   B: columns (r, re/im) interleaved, so a lane's accumulator holds the real and
//      imaginary parts of one right-hand side and the complex result
//        Re y = ReP.Re e - ImP.Im e,  Im y = ReP.Im e + ImP.Re e
//      is formed in registers.
// P is read straight from its FP16 [N][12][V] array: for a fixed j the eight rows
// of a fragment are eight consecutive sites (one 32-byte sector).  E is staged in
// shared memory as FP16 after scaling each right-hand side of the aggregate by a
// power of two of its largest entry (exact to undo), so FP16 range never limits it.
#include <cuda_fp16.h>

#include "kernels.h"

namespace ddamg {

__device__ __forceinline__ void mma16816_tr(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                            unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned as_u32(__half2 v) { return *reinterpret_cast<unsigned*>(&v); }

constexpr int kProTCWarps = 8;
constexpr int kProKPad = 32;  // K = j padded to two k-tiles

// CTA = aggregate c, NT n-tiles of four right-hand sides (r0 .. r0 + 4 NT - 1).
template <int NT>
__global__ void __launch_bounds__(kProTCWarps * 32) prolong_tc_kernel(Geom g, const __half2* __restrict__ P, int N,
                                                                       const cplx<float>* __restrict__ in, cplx<float>* __restrict__ out,
                                                                       int nrhs, int r0) {
    constexpr int NC = 8 * NT;           // B columns: (r, re/im)
    constexpr int LDK = 2 * kProKPad + 8; // halves per staged column: both halves h, padded
    __shared__ __align__(16) __half Es[NC * LDK];
    __shared__ float inv_scale[4 * NT];
    const int c = blockIdx.x;
    const int nc = 2 * N;
    // 1. per right-hand side: scale 2^-e with 2^e >= max |e|, then stage E as FP16 [col][h*32 + j]
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int rr = w; rr < 4 * NT; rr += kProTCWarps) {
        const int r = r0 + rr;
        float m = 0.f;
        if (r < nrhs)
            for (int q = lane; q < nc; q += 32) {
                const cplx<float> v = in[((size_t)r * g.NB + c) * nc + q];
                m = fmaxf(m, fmaxf(fabsf(v.re), fabsf(v.im)));
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        int ex = 0;
        if (m > 0.f) frexpf(m, &ex);                       // m < 2^ex
        const float s = ldexpf(1.f, -ex), is = ldexpf(1.f, ex);
        if (lane == 0) inv_scale[rr] = is;
        for (int q = lane; q < 2 * kProKPad; q += 32) {
            const int h = q / kProKPad, j = q % kProKPad;
            cplx<float> v = czero<float>();
            if (r < nrhs && j < N) v = in[((size_t)r * g.NB + c) * nc + h * N + j];
            Es[(2 * rr) * LDK + q] = __float2half_rn(v.re * s);
            Es[(2 * rr + 1) * LDK + q] = __float2half_rn(v.im * s);
        }
    }
    __syncthreads();
    const int gq = lane >> 2, t = lane & 3;
    // 2. tasks: (h, component k within the half, group of 16 sites)
    const int sg = g.Vb / 16;
    const int ntask = 2 * 6 * sg;
    for (int task = w; task < ntask; task += kProTCWarps) {
        const int h = task / (6 * sg), kc = (task / sg) % 6, s0 = (task % sg) * 16;
        const int k = 6 * h + kc;
        const size_t site0 = (size_t)c * g.Vb + s0;
        float accR[NT][4], accI[NT][4];
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int q = 0; q < 4; ++q) accR[n][q] = accI[n][q] = 0.f;
#pragma unroll
        for (int kt = 0; kt < 2; ++kt) {
            // A rows gq, gq+8 (sites), cols 2t, 2t+1, 2t+8, 2t+9 (j)
            __half2 v[4][2];  // [j slot][row]
#pragma unroll
            for (int js = 0; js < 4; ++js) {
                const int j = 16 * kt + 2 * t + (js & 1) + (js >> 1) * 8;
#pragma unroll
                for (int rw = 0; rw < 2; ++rw) {
                    __half2 x = __float2half2_rn(0.f);
                    if (j < N) x = __ldg(P + ((size_t)j * 12 + k) * g.V + site0 + gq + 8 * rw);
                    v[js][rw] = x;
                }
            }
            // real plane fragments (.x) and imaginary plane fragments (.y)
            const unsigned ar0 = as_u32(__lows2half2(v[0][0], v[1][0])), ar1 = as_u32(__lows2half2(v[0][1], v[1][1]));
            const unsigned ar2 = as_u32(__lows2half2(v[2][0], v[3][0])), ar3 = as_u32(__lows2half2(v[2][1], v[3][1]));
            const unsigned ai0 = as_u32(__highs2half2(v[0][0], v[1][0])), ai1 = as_u32(__highs2half2(v[0][1], v[1][1]));
            const unsigned ai2 = as_u32(__highs2half2(v[2][0], v[3][0])), ai3 = as_u32(__highs2half2(v[2][1], v[3][1]));
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const __half* bc = Es + (size_t)(n * 8 + gq) * LDK + h * kProKPad + kt * 16 + 2 * t;
                const unsigned b0 = *reinterpret_cast<const unsigned*>(bc);
                const unsigned b1 = *reinterpret_cast<const unsigned*>(bc + 8);
                mma16816_tr(accR[n], ar0, ar1, ar2, ar3, b0, b1);
                mma16816_tr(accI[n], ai0, ai1, ai2, ai3, b0, b1);
            }
        }
        // lane holds rows gq, gq+8 and columns 2t (Re e_r), 2t+1 (Im e_r) of r = r0 + 4n + t
#pragma unroll
        for (int n = 0; n < NT; ++n) {
            const int rr = 4 * n + t, r = r0 + rr;
            if (r >= nrhs) continue;
            const float is = inv_scale[rr];
            cplx<float>* o = out + ((size_t)r * 12 + k) * g.V + site0 + gq;
            o[0] = mk((accR[n][0] - accI[n][1]) * is, (accR[n][1] + accI[n][0]) * is);
            o[8] = mk((accR[n][2] - accI[n][3]) * is, (accR[n][3] + accI[n][2]) * is);
        }
    }
}

// ---------------------------------------------------------------------------
// Restriction e[r][c][h N + j] = sum_{x in c, k in half h} conj(P_j[k][x]) in[r][k][x]
// as FP16 tensor-core products with FP32 accumulation: per aggregate half,
//   C = A B,  A rows (r, re/im): row g = Re x_r, row g + 8 = Im x_r (8 right-hand
//   sides per m-tile), K = (component, site) in steps of 16 sites of one component,
//   B columns (j, re/im) of P.  A lane then holds, for one (r, j),
//     c0 = ReX.ReP, c1 = ReX.ImP, c2 = ImX.ReP, c3 = ImX.ImP  and
//     e = (c0 + c3) + i (c2 - c1).
// The warps of a CTA split the K range; their partial sums meet in shared memory.
// Each right-hand side is scaled by a power of two that maps its largest entry on
// the whole field below 2^14 before it is rounded to FP16: an FP16 normal number
// keeps 11 significant bits over 29 binades, so only entries 2^28 below that
// maximum lose precision (a separate pass finds the maxima).
// ---------------------------------------------------------------------------
constexpr int kResTCWarps = 8;

template <int NTN>  // n-tiles over (j, re/im): N = 4 NTN test vectors
__global__ void __launch_bounds__(kResTCWarps * 32) restrict_tc_kernel(Geom g, const __half2* __restrict__ P, int N,
                                                                        const cplx<float>* __restrict__ in, cplx<float>* __restrict__ out,
                                                                        int nrhs, int r0, const int* __restrict__ rmax) {
    constexpr int MT = 2;  // 16 right-hand sides per launch group
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* red = reinterpret_cast<float*>(smem_raw);  // [warps][32 lanes][MT * NTN * 4]
    __shared__ float scale[8 * MT], inv_scale[8 * MT];
    const int c = blockIdx.x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, t = lane & 3;
    const size_t blk0 = (size_t)c * g.Vb;
    // 1. per right-hand side: power-of-two scale of its largest entry on the whole field
    if (threadIdx.x < 8 * MT) {
        const int r = r0 + threadIdx.x;
        int ex = 0;
        const float mm = r < nrhs ? __int_as_float(rmax[r]) : 0.f;
        if (mm > 0.f) frexpf(mm, &ex);
        scale[threadIdx.x] = ldexpf(1.f, 14 - ex);  // largest entry maps below 2^14
        inv_scale[threadIdx.x] = ldexpf(1.f, ex - 14);
    }
    __syncthreads();
    const int sg = g.Vb / 16;
    for (int h = 0; h < 2; ++h) {
        float acc[MT][NTN][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int n = 0; n < NTN; ++n)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[mt][n][q] = 0.f;
        float sc[MT];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) sc[mt] = scale[8 * mt + gq];
        // 2. this warp's share of the k-tiles (component kc, 16 sites from s0)
#pragma unroll 2
        for (int kt = w; kt < 6 * sg; kt += kResTCWarps) {
            const int k = 6 * h + kt / sg, s0 = (kt % sg) * 16;
            const size_t site = blk0 + s0 + 2 * t;
            unsigned a[MT][4];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                const int r = r0 + 8 * mt + gq;
                float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
                if (r < nrhs) {
                    const float4* xr = reinterpret_cast<const float4*>(in + ((size_t)r * 12 + k) * g.V + site);
                    lo = __ldg(xr);      // sites 2t, 2t+1
                    hi = __ldg(xr + 4);  // sites 2t+8, 2t+9
                }
                const float f = sc[mt];
                a[mt][0] = as_u32(__floats2half2_rn(lo.x * f, lo.z * f));  // row g (Re), K 2t, 2t+1
                a[mt][1] = as_u32(__floats2half2_rn(lo.y * f, lo.w * f));  // row g+8 (Im)
                a[mt][2] = as_u32(__floats2half2_rn(hi.x * f, hi.z * f));  // row g, K 2t+8, 2t+9
                a[mt][3] = as_u32(__floats2half2_rn(hi.y * f, hi.w * f));
            }
            const int plane = gq & 1;
#pragma unroll
            for (int n = 0; n < NTN; ++n) {
                const int j = 4 * n + (gq >> 1);
                const uint2* pj = reinterpret_cast<const uint2*>(P + ((size_t)j * 12 + k) * g.V + site);
                const uint2 v0 = __ldg(pj), v1 = __ldg(pj + 4);  // sites 2t, 2t+1 and 2t+8, 2t+9
                const __half2 p00 = *reinterpret_cast<const __half2*>(&v0.x), p01 = *reinterpret_cast<const __half2*>(&v0.y);
                const __half2 p10 = *reinterpret_cast<const __half2*>(&v1.x), p11 = *reinterpret_cast<const __half2*>(&v1.y);
                const unsigned b0 = as_u32(plane ? __highs2half2(p00, p01) : __lows2half2(p00, p01));
                const unsigned b1 = as_u32(plane ? __highs2half2(p10, p11) : __lows2half2(p10, p11));
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) mma16816_tr(acc[mt][n], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
            }
        }
        // 3. sum the warps' partial tiles and form e
        float* my = red + ((size_t)w * 32 + lane) * (MT * NTN * 4);
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int n = 0; n < NTN; ++n)
#pragma unroll
                for (int q = 0; q < 4; ++q) my[(mt * NTN + n) * 4 + q] = acc[mt][n][q];
        __syncthreads();
        for (int q = threadIdx.x; q < 32 * MT * NTN; q += blockDim.x) {
            const int ln = q % 32, tile = q / 32;  // tile = mt * NTN + n
            float cc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int ww = 0; ww < kResTCWarps; ++ww) {
                const float* src = red + ((size_t)ww * 32 + ln) * (MT * NTN * 4) + tile * 4;
                cc[0] += src[0], cc[1] += src[1], cc[2] += src[2], cc[3] += src[3];
            }
            const int mt = tile / NTN, n = tile % NTN, rr = 8 * mt + (ln >> 2), j = 4 * n + (ln & 3), r = r0 + rr;
            if (r < nrhs && j < N) {
                const float is = inv_scale[rr];
                out[((size_t)r * g.NB + c) * (2 * N) + h * N + j] = mk((cc[0] + cc[3]) * is, (cc[2] - cc[1]) * is);
            }
        }
        __syncthreads();
    }
}

// rmax[r] = bits of max |Re|, |Im| over the field of right-hand side r (non-negative floats
// order like their bit patterns, so an integer atomicMax finds the largest)
__global__ void field_absmax_kernel(const float4* __restrict__ in, size_t n4, int* __restrict__ rmax) {
    const int r = blockIdx.y;
    const float4* x = in + (size_t)r * n4;
    float m = 0.f;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (size_t)gridDim.x * blockDim.x) {
        const float4 v = __ldg(x + q);
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(rmax + r, __float_as_int(m));
}

bool restrict_tc_supported(const Geom& g, int N) { return g.Vb % 16 == 0 && N % 4 == 0 && N <= 32; }

int launch_restrict_tc(const Geom& g, const cplx<__half>* P, int N, const cplx<float>* in, cplx<float>* out, int nrhs, int* rmax,
                       cudaStream_t st) {
    const __half2* P2 = reinterpret_cast<const __half2*>(P);
    const int NTN = N / 4;
    const size_t sm = (size_t)kResTCWarps * 32 * 2 * NTN * 4 * sizeof(float);
    const size_t n4 = (size_t)12 * g.V / 2;  // float4 = two complex numbers; 12 V is even
    DD_CUDA(cudaMemsetAsync(rmax, 0, sizeof(int) * nrhs, st));
    const int bx = (int)std::min<size_t>((n4 + 255) / 256, (size_t)std::max(1, 152 * 8 / nrhs));
    field_absmax_kernel<<<dim3(bx, nrhs), 256, 0, st>>>(reinterpret_cast<const float4*>(in), n4, rmax);
    DD_CHECK_LAUNCH();
    for (int r0 = 0; r0 < nrhs; r0 += 16) {
        switch (NTN) {
#define DD_RES_TC(n)                                                                                                   \
    case n:                                                                                                            \
        if (sm + 1024 > 48 * 1024) /* dynamic + static beyond the default 48 KB needs the opt-in */                           \
            cudaFuncSetAttribute(restrict_tc_kernel<n>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);               \
        restrict_tc_kernel<n><<<g.NB, kResTCWarps * 32, sm, st>>>(g, P2, N, in, out, nrhs, r0, rmax);                \
        break;
            DD_RES_TC(1)
            DD_RES_TC(2)
            DD_RES_TC(3)
            DD_RES_TC(4)
            DD_RES_TC(5)
            DD_RES_TC(6)
            DD_RES_TC(7)
            DD_RES_TC(8)
#undef DD_RES_TC
            default:
                return DDAMG_ERR_INVALID_ARG;
        }
        DD_CHECK_LAUNCH();
    }
    return 0;
}

bool prolong_tc_supported(const Geom& g, int N) { return g.Vb % 16 == 0 && N <= kProKPad; }

int launch_prolong_tc(const Geom& g, const cplx<__half>* P, int N, const cplx<float>* in, cplx<float>* out, int nrhs, cudaStream_t st) {
    const __half2* P2 = reinterpret_cast<const __half2*>(P);
    for (int r0 = 0; r0 < nrhs; r0 += 12) {
        const int nr = std::min(12, nrhs - r0);
        const int nt = (nr + 3) / 4;
        if (nt == 3)
            prolong_tc_kernel<3><<<g.NB, kProTCWarps * 32, 0, st>>>(g, P2, N, in, out, nrhs, r0);
        else if (nt == 2)
            prolong_tc_kernel<2><<<g.NB, kProTCWarps * 32, 0, st>>>(g, P2, N, in, out, nrhs, r0);
        else
            prolong_tc_kernel<1><<<g.NB, kProTCWarps * 32, 0, st>>>(g, P2, N, in, out, nrhs, r0);
        DD_CHECK_LAUNCH();
    }
    return 0;
}

}  // namespace ddamg
