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
