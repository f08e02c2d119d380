// Aggregation-based transfer operators (Sec. 3.1-3.2): restriction P^H,
// prolongation P, the local orthonormalisation of the test vectors on every
// aggregate, and the assembly of the coarse stencil D_c = P^H D P.
//
// P is stored as N fine spinor fields P_j [N][12][V] (internal order): column
// (c, h, j) of P is P_j restricted to block c and spins {2h, 2h+1}.
// Coarse vectors: cplx[nrhs][NB][2N], component h*N + j.
#include <cuda_fp16.h>

#include "kernels.h"
#include "dirac.cuh"

namespace ddamg {

// ---------------------------------------------------------------------------
// restriction out[r][c][h*N + j] = sum_{x in c, k in half h} conj(P_j[k][x]) in[r][k][x]
// CTA = (block c, rhs r), one thread per site of the block.
// ---------------------------------------------------------------------------
template <typename T, typename Tp>
__global__ void restrict_kernel(Geom g, const cplx<Tp>* __restrict__ P, int N, const cplx<T>* __restrict__ in,
                                cplx<T>* __restrict__ out, int nrhs) {
    // accumulation in the V-cycle precision T (FP64 arithmetic is a small fraction of FP32 on GB300)
    extern __shared__ unsigned char smem_raw[];
    T* red = reinterpret_cast<T*>(smem_raw);  // [nwarps][4N]
    const int r = blockIdx.x % nrhs;
    const int c = blockIdx.x / nrhs;
    const int l = threadIdx.x;
    const bool act = l < g.Vb;
    const int i = c * g.Vb + l;
    const cplx<T>* inr = in + (size_t)r * 12 * g.V;
    cplx<T> x[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) x[k] = act ? inr[(size_t)k * g.V + i] : czero<T>();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = 0; j < N; ++j) {
        cplx<T> s0 = czero<T>(), s1 = czero<T>();
        if (act) {
            const cplx<Tp>* pj = P + (size_t)j * 12 * g.V;
#pragma unroll
            for (int k = 0; k < 6; ++k) cmac_conj(s0, ccast<T>(pj[(size_t)k * g.V + i]), x[k]);
#pragma unroll
            for (int k = 6; k < 12; ++k) cmac_conj(s1, ccast<T>(pj[(size_t)k * g.V + i]), x[k]);
        }
        s0.re = warp_sum(s0.re);
        s0.im = warp_sum(s0.im);
        s1.re = warp_sum(s1.re);
        s1.im = warp_sum(s1.im);
        if (lane == 0) {
            T* q = red + (size_t)w * 4 * N + 4 * j;
            q[0] = s0.re;
            q[1] = s0.im;
            q[2] = s1.re;
            q[3] = s1.im;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 4 * N; q += blockDim.x) {
        T s = 0;
        for (int ww = 0; ww < nw; ++ww) s += red[(size_t)ww * 4 * N + q];
        int j = q >> 2, h = (q >> 1) & 1, im = q & 1;  // q = 4 j + 2 h + im
        T* o = reinterpret_cast<T*>(out + ((size_t)r * g.NB + c) * (2 * N) + h * N + j);
        o[im] = s;
    }
}

template <typename T, typename Tp>
int launch_restrict(const Geom& g, const cplx<Tp>* P, int N, const cplx<T>* in, cplx<T>* out, int nrhs, cudaStream_t st) {
    const int nt = ((g.Vb + 31) / 32) * 32;
    const long long nblk = (long long)g.NB * nrhs;
    size_t sm = (size_t)(nt / 32) * 4 * N * sizeof(T);
    if (sm > 48 * 1024) cudaFuncSetAttribute(restrict_kernel<T, Tp>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    restrict_kernel<T, Tp><<<(unsigned)nblk, nt, sm, st>>>(g, P, N, in, out, nrhs);
    DD_CHECK_LAUNCH();
    return 0;
}

// ---------------------------------------------------------------------------
// prolongation out[r][k][x] = sum_j P_j[k][x] in[r][c(x)][h(k)*N + j]
// ---------------------------------------------------------------------------
template <typename T, typename Tp>
__global__ void prolong_kernel(Geom g, const cplx<Tp>* __restrict__ P, int N, const cplx<T>* __restrict__ in,
                               cplx<T>* __restrict__ out, int nrhs) {
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* e = reinterpret_cast<cplx<T>*>(smem_raw);  // [2N]
    const int r = blockIdx.x % nrhs;
    const int c = blockIdx.x / nrhs;
    const cplx<T>* src = in + ((size_t)r * g.NB + c) * (2 * N);
    for (int q = threadIdx.x; q < 2 * N; q += blockDim.x) e[q] = src[q];
    __syncthreads();
    const int l = threadIdx.x;
    if (l >= g.Vb) return;
    const int i = c * g.Vb + l;
    cplx<T> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = czero<T>();
    for (int j = 0; j < N; ++j) {
        const cplx<Tp>* pj = P + (size_t)j * 12 * g.V;
        cplx<T> e0 = e[j], e1 = e[N + j];
#pragma unroll
        for (int k = 0; k < 6; ++k) cmac(acc[k], ccast<T>(pj[(size_t)k * g.V + i]), e0);
#pragma unroll
        for (int k = 6; k < 12; ++k) cmac(acc[k], ccast<T>(pj[(size_t)k * g.V + i]), e1);
    }
    cplx<T>* o = out + (size_t)r * 12 * g.V;
#pragma unroll
    for (int k = 0; k < 12; ++k) o[(size_t)k * g.V + i] = acc[k];
}

template <typename T, typename Tp>
int launch_prolong(const Geom& g, const cplx<Tp>* P, int N, const cplx<T>* in, cplx<T>* out, int nrhs, cudaStream_t st) {
    const int nt = ((g.Vb + 31) / 32) * 32;
    const long long nblk = (long long)g.NB * nrhs;
    prolong_kernel<T, Tp><<<(unsigned)nblk, nt, 2 * N * sizeof(cplx<T>), st>>>(g, P, N, in, out, nrhs);
    DD_CHECK_LAUNCH();
    return 0;
}

template int launch_restrict<double, double>(const Geom&, const cplx<double>*, int, const cplx<double>*, cplx<double>*, int,
                                             cudaStream_t);
template int launch_restrict<float, float>(const Geom&, const cplx<float>*, int, const cplx<float>*, cplx<float>*, int,
                                           cudaStream_t);
template int launch_restrict<float, __half>(const Geom&, const cplx<__half>*, int, const cplx<float>*, cplx<float>*, int,
                                            cudaStream_t);
template int launch_prolong<float, __half>(const Geom&, const cplx<__half>*, int, const cplx<float>*, cplx<float>*, int,
                                           cudaStream_t);
template int launch_prolong<double, double>(const Geom&, const cplx<double>*, int, const cplx<double>*, cplx<double>*, int,
                                            cudaStream_t);
template int launch_prolong<float, float>(const Geom&, const cplx<float>*, int, const cplx<float>*, cplx<float>*, int,
                                          cudaStream_t);

// ---------------------------------------------------------------------------
// local orthonormalisation (Sec. 3.1): modified Gram-Schmidt of P_1..P_N on every
// aggregate (block c, half h), in place, FP64.  CTA = (c, h), thread = site.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum_d(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0;
    for (int q = 0; q < nw; ++q) s += red[q];
    return s;
}

__global__ void gram_schmidt_kernel(Geom g, cplx<double>* __restrict__ P, int N, int* __restrict__ fail) {
    __shared__ double red[32];
    const int c = blockIdx.x >> 1, h = blockIdx.x & 1;
    const int l = threadIdx.x;
    const bool act = l < g.Vb;
    const int i = c * g.Vb + l;
    for (int j = 0; j < N; ++j) {
        cplx<double>* pj = P + (size_t)j * 12 * g.V;
        double orig = 0;
        if (act)
            for (int k = 6 * h; k < 6 * h + 6; ++k) orig += norm2(pj[(size_t)k * g.V + i]);
        orig = block_sum_d(orig, red);
        for (int q = 0; q < j; ++q) {
            const cplx<double>* pq = P + (size_t)q * 12 * g.V;
            cplx<double> d = czero<double>();
            if (act)
                for (int k = 6 * h; k < 6 * h + 6; ++k) cmac_conj(d, pq[(size_t)k * g.V + i], pj[(size_t)k * g.V + i]);
            d.re = block_sum_d(d.re, red);
            d.im = block_sum_d(d.im, red);
            if (act)
                for (int k = 6 * h; k < 6 * h + 6; ++k) pj[(size_t)k * g.V + i] = pj[(size_t)k * g.V + i] - d * pq[(size_t)k * g.V + i];
        }
        double nn = 0;
        if (act)
            for (int k = 6 * h; k < 6 * h + 6; ++k) nn += norm2(pj[(size_t)k * g.V + i]);
        nn = block_sum_d(nn, red);
        if (!(nn > 1e-24 * orig) || !(orig > 0)) {
            if (threadIdx.x == 0) atomicExch(fail, 1);
            nn = 1.0;
        }
        double inv = 1.0 / sqrt(nn);
        if (act)
            for (int k = 6 * h; k < 6 * h + 6; ++k) pj[(size_t)k * g.V + i] = inv * pj[(size_t)k * g.V + i];
    }
}

int launch_gram_schmidt(const Geom& g, cplx<double>* P, int N, int* fail, cudaStream_t st) {
    const int nt = ((g.Vb + 31) / 32) * 32;
    gram_schmidt_kernel<<<2 * g.NB, nt, 0, st>>>(g, P, N, fail);
    DD_CHECK_LAUNCH();
    return 0;
}

// ---------------------------------------------------------------------------
// D_c assembly.  For a direction dir (0 = self, 1 + d = hop in fine direction d
// leaving the block) and every column (h, j):
//   T_(h,j) = D_block P_j^(h)            (dir = 0: site term + hops inside the block)
//   T_(h,j) = H_d P_j^(h) on face sites  (dir = 1 + d)
// with P_j^(h) = P_j restricted to spins {2h, 2h+1}.  Then
//   B_dir(c)[(h',j')][(h,j)] = sum_{x in c, k in half h'} conj(P_j'[k][x]) T_(h,j)[k][x].
// ---------------------------------------------------------------------------

// masked load: P_j at site x with only the spins of half h kept
__device__ __forceinline__ void load_half(Spinor<double>& s, const cplx<double>* __restrict__ pj, int V, int x, int h) {
#pragma unroll
    for (int k = 0; k < 12; ++k) s.v[k] = ((k / 6) == h) ? pj[(size_t)k * V + x] : czero<double>();
}

template <int MU>
__device__ __forceinline__ void asm_hop_dir(const Geom& g, const cplx<double>* __restrict__ U, const cplx<double>* __restrict__ pj,
                                            int h, int i, int nb, bool fwd, Spinor<double>& acc) {
    cplx<double> W[9];
    Spinor<double> pn;
    load_half(pn, pj, g.V, nb, h);
    if (fwd) {
        load_link(W, U, g.V, MU, i);
        hop_acc<MU, true>(acc, pn, W);
    } else {
        load_link(W, U, g.V, MU, nb);
        hop_acc<MU, false>(acc, pn, W);
    }
}

__device__ __forceinline__ void asm_hop(const Geom& g, const cplx<double>* __restrict__ U, const cplx<double>* __restrict__ pj,
                                        int h, int i, int nb, int d, Spinor<double>& acc) {
    const bool fwd = (d & 1) == 0;
    switch (d >> 1) {
        case 0: asm_hop_dir<0>(g, U, pj, h, i, nb, fwd, acc); break;
        case 1: asm_hop_dir<1>(g, U, pj, h, i, nb, fwd, acc); break;
        case 2: asm_hop_dir<2>(g, U, pj, h, i, nb, fwd, acc); break;
        default: asm_hop_dir<3>(g, U, pj, h, i, nb, fwd, acc); break;
    }
}

__global__ void assemble_T_kernel(Geom g, FineOp<double> op, const cplx<double>* __restrict__ P, int N, int dir,
                                  cplx<double>* __restrict__ Tout) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)g.V * 2 * N) return;
    const int i = (int)(tid % g.V);
    const int col = (int)(tid / g.V);
    const int h = col / N, j = col % N;
    const cplx<double>* pj = P + (size_t)j * 12 * g.V;
    const int c = block_of(g, i);
    const int l = i - c * g.Vb;
    Spinor<double> acc;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc.v[k] = czero<double>();
    Spinor<double> out;
    if (dir == 0) {
        for (int d = 0; d < 8; ++d) {
            int e = __ldg(g.lnbr + d * g.Vb + l);
            if (e >> 16) continue;
            asm_hop(g, op.U, pj, h, i, c * g.Vb + (e & 0xffff), d, acc);
        }
        Spinor<double> x;
        load_half(x, pj, g.V, i, h);
        herm_apply(op.clov, g.V, i, x, out);
#pragma unroll
        for (int k = 0; k < 12; ++k) out.v[k] = out.v[k] - 0.5 * acc.v[k];
    } else {
        const int d = dir - 1;
        int e = __ldg(g.lnbr + d * g.Vb + l);
        if (e >> 16) asm_hop(g, op.U, pj, h, i, fine_nbr(g, i, d), d, acc);
#pragma unroll
        for (int k = 0; k < 12; ++k) out.v[k] = -0.5 * acc.v[k];
    }
    cplx<double>* o = Tout + (size_t)col * 12 * g.V;
#pragma unroll
    for (int k = 0; k < 12; ++k) o[(size_t)k * g.V + i] = out.v[k];
}

int launch_assemble_T(const Geom& g, const FineOp<double>& op, const cplx<double>* P, int N, int dir, cplx<double>* T,
                      cudaStream_t st) {
    const long long n = (long long)g.V * 2 * N;
    assemble_T_kernel<<<ceil_div(n, 128), 128, 0, st>>>(g, op, P, N, dir, T);
    DD_CHECK_LAUNCH();
    return 0;
}

// B_dir(c) = P_c^H T on the listed local sites (all sites for dir 0, the face for dir > 0).
// CTA = (c, output tile); outputs column-major: o = col * nc + row.
constexpr int kProjThreads = 256;
constexpr int kProjPerThread = 8;

__global__ void __launch_bounds__(kProjThreads) block_project_kernel(Geom g, const cplx<double>* __restrict__ P, int N,
                                                                     const cplx<double>* __restrict__ Tin,
                                                                     const int* __restrict__ sites, int nsites, int CH,
                                                                     double* __restrict__ Bout, size_t site_stride) {
    extern __shared__ unsigned char smem_raw[];
    const int nc = 2 * N;
    cplx<double>* Pc = reinterpret_cast<cplx<double>*>(smem_raw);  // [N][12][CH]
    cplx<double>* Tc = Pc + (size_t)N * 12 * CH;                      // [2N][12][CH]
    const int c = blockIdx.x;
    const int o0 = blockIdx.y * kProjThreads * kProjPerThread;
    cplx<double> acc[kProjPerThread];
#pragma unroll
    for (int m = 0; m < kProjPerThread; ++m) acc[m] = czero<double>();
    for (int s0 = 0; s0 < nsites; s0 += CH) {
        __syncthreads();
        for (int q = threadIdx.x; q < N * 12 * CH; q += blockDim.x) {
            int s = q % CH, k = (q / CH) % 12, j = q / (12 * CH);
            cplx<double> v = czero<double>();
            if (s0 + s < nsites) v = P[((size_t)j * 12 + k) * g.V + (size_t)c * g.Vb + sites[s0 + s]];
            Pc[q] = v;
        }
        for (int q = threadIdx.x; q < nc * 12 * CH; q += blockDim.x) {
            int s = q % CH, k = (q / CH) % 12, col = q / (12 * CH);
            cplx<double> v = czero<double>();
            if (s0 + s < nsites) v = Tin[((size_t)col * 12 + k) * g.V + (size_t)c * g.Vb + sites[s0 + s]];
            Tc[q] = v;
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < kProjPerThread; ++m) {
            int o = o0 + m * kProjThreads + threadIdx.x;
            if (o >= nc * nc) break;
            int col = o / nc, row = o % nc;
            int hp = row / N, jp = row % N;
            const cplx<double>* pr = Pc + ((size_t)jp * 12 + 6 * hp) * CH;
            const cplx<double>* tc = Tc + ((size_t)col * 12 + 6 * hp) * CH;
            for (int q = 0; q < 6 * CH; ++q) cmac_conj(acc[m], pr[q], tc[q]);
        }
    }
#pragma unroll
    for (int m = 0; m < kProjPerThread; ++m) {
        int o = o0 + m * kProjThreads + threadIdx.x;
        if (o >= nc * nc) break;
        double* b = Bout + ((size_t)c * site_stride + o) * 2;
        b[0] = acc[m].re;
        b[1] = acc[m].im;
    }
}

int launch_block_project(const Geom& g, const cplx<double>* P, int N, const cplx<double>* T, const int* sites, int nsites,
                         double* Bout, size_t site_stride, cudaStream_t st) {
    const int nc = 2 * N;
    int CH = (int)((160 * 1024) / ((size_t)3 * N * 12 * sizeof(cplx<double>)));
    if (CH > 8) CH = 8;
    if (CH < 1) CH = 1;
    size_t smem = (size_t)3 * N * 12 * CH * sizeof(cplx<double>);
    cudaFuncSetAttribute(block_project_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    dim3 grid(g.NB, ceil_div((long long)nc * nc, kProjThreads * kProjPerThread));
    block_project_kernel<<<grid, kProjThreads, smem, st>>>(g, P, N, T, sites, nsites, CH, Bout, site_stride);
    DD_CHECK_LAUNCH();
    return 0;
}

}  // namespace ddamg
