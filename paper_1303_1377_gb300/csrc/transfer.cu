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
// CTA = (block c, group of R right-hand sides), one thread per site of the block:
// every P_j entry loaded once serves R right-hand sides.  The 4R partial sums of one
// j are reduced over the warp by recursive halving (each lane keeps half of its
// values and trades the other half with its partner, so 4R values cost about 4R
// shuffles, not 4R log2(32)), then over the warps through shared memory.
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ int bitrev_idx(int lane) {
    // value index held by a lane after the halving levels 1, 2, ..., K/2
    int q = 0;
#pragma unroll
    for (int m = 1, b = K >> 1; m < K; m <<= 1, b >>= 1)
        if (lane & m) q |= b;
    return q;
}

template <typename T, int K>
__device__ __forceinline__ T warp_transpose_sum(T (&v)[K], int lane) {
    // on return lane l holds the warp sum of value bitrev_idx<K>(l & (K-1))
#pragma unroll
    for (int m = 1, half = K >> 1; half >= 1; m <<= 1, half >>= 1) {
        const bool up = lane & m;
#pragma unroll
        for (int q = 0; q < half; ++q) {
            T send = up ? v[q] : v[q + half];
            T keep = up ? v[q + half] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
    }
    T s = v[0];
#pragma unroll
    for (int m = K; m < 32; m <<= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    return s;
}

template <typename T, typename Tp, int R>
__global__ void restrict_kernel(Geom g, const cplx<Tp>* __restrict__ P, int N, const cplx<T>* __restrict__ in,
                                cplx<T>* __restrict__ out, int r0, int ngroups) {
    // accumulation in the V-cycle precision T (FP64 arithmetic is a small fraction of FP32 on GB300)
    constexpr int K = 4 * R;
    extern __shared__ unsigned char smem_raw[];
    T* red = reinterpret_cast<T*>(smem_raw);  // [nwarps][N][K]
    const int rb = r0 + (blockIdx.x % ngroups) * R;
    const int c = blockIdx.x / ngroups;
    const int l = threadIdx.x;
    const bool act = l < g.Vb;
    const int i = c * g.Vb + l;
    cplx<T> x[R][12];
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const cplx<T>* inr = in + (size_t)(rb + u) * 12 * g.V;
#pragma unroll
        for (int k = 0; k < 12; ++k) x[u][k] = act ? inr[(size_t)k * g.V + i] : czero<T>();
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int myq = bitrev_idx<K>(lane & (K - 1));
#pragma unroll 2
    for (int j = 0; j < N; ++j) {
        T v[K];
#pragma unroll
        for (int q = 0; q < K; ++q) v[q] = 0;
        if (act) {
            const cplx<Tp>* pj = P + (size_t)j * 12 * g.V;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const cplx<T> p = ccast<T>(pj[(size_t)k * g.V + i]);
                const int o = k < 6 ? 0 : 2;
#pragma unroll
                for (int u = 0; u < R; ++u) {
                    // conj(p) * x
                    v[4 * u + o] += p.re * x[u][k].re + p.im * x[u][k].im;
                    v[4 * u + o + 1] += p.re * x[u][k].im - p.im * x[u][k].re;
                }
            }
        }
        T s = warp_transpose_sum<T, K>(v, lane);
        if (lane < K) red[((size_t)w * N + j) * K + myq] = s;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < K * N; q += blockDim.x) {
        T s = 0;
        for (int ww = 0; ww < nw; ++ww) s += red[(size_t)ww * K * N + q];
        const int j = q / K, t = q % K;
        const int u = t >> 2, h = (t >> 1) & 1, im = t & 1;  // t = 4 u + 2 h + im
        T* o = reinterpret_cast<T*>(out + ((size_t)(rb + u) * g.NB + c) * (2 * N) + h * N + j);
        o[im] = s;
    }
}

template <typename T, typename Tp, int R>
static int launch_restrict_r(const Geom& g, const cplx<Tp>* P, int N, const cplx<T>* in, cplx<T>* out, int r0, int ngroups,
                             cudaStream_t st) {
    const int nt = ((g.Vb + 31) / 32) * 32;
    const long long nblk = (long long)g.NB * ngroups;
    size_t sm = (size_t)(nt / 32) * 4 * R * N * sizeof(T);
    if (sm > 48 * 1024) cudaFuncSetAttribute(restrict_kernel<T, Tp, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    restrict_kernel<T, Tp, R><<<(unsigned)nblk, nt, sm, st>>>(g, P, N, in, out, r0, ngroups);
    DD_CHECK_LAUNCH();
    return 0;
}

// FP32 (and half-P) restriction takes 2 right-hand sides per CTA, FP64 one (register budget)
template <typename T, typename Tp>
int launch_restrict(const Geom& g, const cplx<Tp>* P, int N, const cplx<T>* in, cplx<T>* out, int nrhs, cudaStream_t st) {
    int r0 = 0;
    if constexpr (sizeof(T) == 4) if (nrhs >= 2) {
        { int e_ = (launch_restrict_r<T, Tp, 2>(g, P, N, in, out, 0, nrhs / 2, st)); if (e_) return e_; }
        r0 = nrhs / 2 * 2;
    }
    if (r0 < nrhs) { int e_ = (launch_restrict_r<T, Tp, 1>(g, P, N, in, out, r0, nrhs - r0, st)); if (e_) return e_; }
    return 0;
}

// ---------------------------------------------------------------------------
// prolongation out[r][k][x] = sum_j P_j[k][x] in[r][c(x)][h(k)*N + j]
// CTA = (block c, group of R right-hand sides); every P_j entry loaded once serves R.
// ---------------------------------------------------------------------------
template <typename T, typename Tp, int R>
__global__ void prolong_kernel(Geom g, const cplx<Tp>* __restrict__ P, int N, const cplx<T>* __restrict__ in,
                               cplx<T>* __restrict__ out, int r0, int ngroups) {
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* e = reinterpret_cast<cplx<T>*>(smem_raw);  // [R][2N]
    const int rb = r0 + (blockIdx.x % ngroups) * R;
    const int c = blockIdx.x / ngroups;
    for (int q = threadIdx.x; q < 2 * N * R; q += blockDim.x) {
        const int u = q / (2 * N), t = q % (2 * N);
        e[q] = in[((size_t)(rb + u) * g.NB + c) * (2 * N) + t];
    }
    __syncthreads();
    const int l = threadIdx.x;
    if (l >= g.Vb) return;
    const int i = c * g.Vb + l;
    cplx<T> acc[R][12];
#pragma unroll
    for (int u = 0; u < R; ++u)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[u][k] = czero<T>();
    for (int j = 0; j < N; ++j) {
        const cplx<Tp>* pj = P + (size_t)j * 12 * g.V;
        cplx<T> e0[R], e1[R];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            e0[u] = e[u * 2 * N + j];
            e1[u] = e[u * 2 * N + N + j];
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const cplx<T> p = ccast<T>(pj[(size_t)k * g.V + i]);
#pragma unroll
            for (int u = 0; u < R; ++u) cmac(acc[u][k], p, k < 6 ? e0[u] : e1[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < R; ++u) {
        cplx<T>* o = out + (size_t)(rb + u) * 12 * g.V;
#pragma unroll
        for (int k = 0; k < 12; ++k) o[(size_t)k * g.V + i] = acc[u][k];
    }
}

template <typename T, typename Tp, int R>
static int launch_prolong_r(const Geom& g, const cplx<Tp>* P, int N, const cplx<T>* in, cplx<T>* out, int r0, int ngroups,
                            cudaStream_t st) {
    const int nt = ((g.Vb + 31) / 32) * 32;
    const long long nblk = (long long)g.NB * ngroups;
    prolong_kernel<T, Tp, R><<<(unsigned)nblk, nt, 2 * N * R * sizeof(cplx<T>), st>>>(g, P, N, in, out, r0, ngroups);
    DD_CHECK_LAUNCH();
    return 0;
}

template <typename T, typename Tp>
int launch_prolong(const Geom& g, const cplx<Tp>* P, int N, const cplx<T>* in, cplx<T>* out, int nrhs, cudaStream_t st) {
    int r0 = 0;
    if constexpr (sizeof(T) == 4) if (nrhs >= 4) {
        { int e_ = (launch_prolong_r<T, Tp, 4>(g, P, N, in, out, 0, nrhs / 4, st)); if (e_) return e_; }
        r0 = nrhs / 4 * 4;
    }
    if (r0 < nrhs) { int e_ = (launch_prolong_r<T, Tp, 1>(g, P, N, in, out, r0, nrhs - r0, st)); if (e_) return e_; }
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

__global__ void assemble_T_kernel(Geom g, FineOp<double> op, const cplx<double>* __restrict__ P, int N, int dir, int col0, int ncols,
                                  cplx<double>* __restrict__ Tout) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)g.V * ncols) return;
    const int i = (int)(tid % g.V);
    const int col = col0 + (int)(tid / g.V);
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
    cplx<double>* o = Tout + (size_t)(col - col0) * 12 * g.V;
#pragma unroll
    for (int k = 0; k < 12; ++k) o[(size_t)k * g.V + i] = out.v[k];
}

// T[col - col0] = (the part of D in direction dir) applied to column col of P (split by chirality
// half), for the columns col0 .. col0 + ncols - 1 of the 2N
int launch_assemble_T(const Geom& g, const FineOp<double>& op, const cplx<double>* P, int N, int dir, int col0, int ncols,
                      cplx<double>* T, cudaStream_t st) {
    const long long n = (long long)g.V * ncols;
    assemble_T_kernel<<<ceil_div(n, 128), 128, 0, st>>>(g, op, P, N, dir, col0, ncols, T);
    DD_CHECK_LAUNCH();
    return 0;
}

// B_dir(c) = P_c^H T on the listed local sites (all sites for dir 0, the face for dir > 0).
// CTA = (c, output tile); outputs column-major: o = col * nc + row.
constexpr int kProjThreads = 256;
constexpr int kProjPerThread = 8;

__global__ void __launch_bounds__(kProjThreads) block_project_kernel(Geom g, const cplx<double>* __restrict__ P, int N,
                                                                     const cplx<double>* __restrict__ Tin, int col0, int ncols,
                                                                     const int* __restrict__ sites, int nsites, int CH,
                                                                     double* __restrict__ Bout, size_t site_stride) {
    extern __shared__ unsigned char smem_raw[];
    const int nc = 2 * N;
    cplx<double>* Pc = reinterpret_cast<cplx<double>*>(smem_raw);  // [N][12][CH]
    cplx<double>* Tc = Pc + (size_t)N * 12 * CH;                      // [ncols][12][CH]
    const int c = blockIdx.x;
    // outputs o = (col - col0) * nc + row of this launch's columns
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
        for (int q = threadIdx.x; q < ncols * 12 * CH; q += blockDim.x) {
            int s = q % CH, k = (q / CH) % 12, col = q / (12 * CH);
            cplx<double> v = czero<double>();
            if (s0 + s < nsites) v = Tin[((size_t)col * 12 + k) * g.V + (size_t)c * g.Vb + sites[s0 + s]];
            Tc[q] = v;
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < kProjPerThread; ++m) {
            int o = o0 + m * kProjThreads + threadIdx.x;
            if (o >= ncols * nc) break;
            int col = o / nc, row = o % nc;  // col relative to col0
            int hp = row / N, jp = row % N;
            const cplx<double>* pr = Pc + ((size_t)jp * 12 + 6 * hp) * CH;
            const cplx<double>* tc = Tc + ((size_t)col * 12 + 6 * hp) * CH;
            for (int q = 0; q < 6 * CH; ++q) cmac_conj(acc[m], pr[q], tc[q]);
        }
    }
#pragma unroll
    for (int m = 0; m < kProjPerThread; ++m) {
        int o = o0 + m * kProjThreads + threadIdx.x;
        if (o >= ncols * nc) break;
        double* b = Bout + ((size_t)c * site_stride + (size_t)col0 * nc + o) * 2;
        b[0] = acc[m].re;
        b[1] = acc[m].im;
    }
}

int launch_block_project(const Geom& g, const cplx<double>* P, int N, const cplx<double>* T, int col0, int ncols, const int* sites,
                         int nsites, double* Bout, size_t site_stride, cudaStream_t st) {
    const int nc = 2 * N;
    int CH = (int)((160 * 1024) / ((size_t)(N + ncols) * 12 * sizeof(cplx<double>)));
    if (CH > 8) CH = 8;
    if (CH < 1) CH = 1;
    size_t smem = (size_t)(N + ncols) * 12 * CH * sizeof(cplx<double>);
    cudaFuncSetAttribute(block_project_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    dim3 grid(g.NB, ceil_div((long long)ncols * nc, kProjThreads * kProjPerThread));
    block_project_kernel<<<grid, kProjThreads, smem, st>>>(g, P, N, T, col0, ncols, sites, nsites, CH, Bout, site_stride);
    DD_CHECK_LAUNCH();
    return 0;
}

}  // namespace ddamg
