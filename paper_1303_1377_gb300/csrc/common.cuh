// Shared device-side definitions of libddamg: complex arithmetic, the internal
// lattice ordering, launch bookkeeping and block reductions.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>

namespace ddamg {

// ---------------------------------------------------------------------------
// complex numbers (interleaved re, im; 8 bytes for float, 16 for double)
// ---------------------------------------------------------------------------
template <typename T>
struct alignas(2 * sizeof(T)) cplx {
    T re, im;
};

// double-word FP32 number h + l used as a storage type (FP64-like precision at FP32 speed)
struct dwf {
    float h, l;
};

template <typename T>
__host__ __device__ __forceinline__ cplx<T> mk(T r, T i) {
    cplx<T> z;
    z.re = r;
    z.im = i;
    return z;
}
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return mk(s * a.re, s * a.im); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> conj(cplx<T> a) { return mk(a.re, -a.im); }
// a += b * c
template <typename T>
__host__ __device__ __forceinline__ void cmac(cplx<T>& a, cplx<T> b, cplx<T> c) {
    a.re = fma(b.re, c.re, a.re);
    a.re = fma(-b.im, c.im, a.re);
    a.im = fma(b.re, c.im, a.im);
    a.im = fma(b.im, c.re, a.im);
}
// a += conj(b) * c
template <typename T>
__host__ __device__ __forceinline__ void cmac_conj(cplx<T>& a, cplx<T> b, cplx<T> c) {
    a.re = fma(b.re, c.re, a.re);
    a.re = fma(b.im, c.im, a.re);
    a.im = fma(b.re, c.im, a.im);
    a.im = fma(-b.im, c.re, a.im);
}
template <typename T>
__host__ __device__ __forceinline__ T norm2(cplx<T> a) { return a.re * a.re + a.im * a.im; }
// multiply by i^p (p = 0..3): 1, i, -1, -i
template <int P, typename T>
__host__ __device__ __forceinline__ cplx<T> ipow(cplx<T> a) {
    if (P == 0) return a;
    if (P == 1) return mk(-a.im, a.re);
    if (P == 2) return mk(-a.re, -a.im);
    return mk(a.im, -a.re);
}
template <typename T>
__host__ __device__ __forceinline__ cplx<T> czero() { return mk<T>(T(0), T(0)); }

template <typename To, typename Ti>
__host__ __device__ __forceinline__ cplx<To> ccast(cplx<Ti> a) { return mk<To>(To(a.re), To(a.im)); }

// read-only cached loads of complex numbers
__device__ __forceinline__ cplx<float> ldg_c(const cplx<float>* p) {
    float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return mk(v.x, v.y);
}
__device__ __forceinline__ cplx<double> ldg_c(const cplx<double>* p) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return mk(v.x, v.y);
}

// smallest positive normal number of T (guards divisions by vanishing norms)
template <typename T>
__host__ __device__ __forceinline__ T tiny_normal();
template <>
__host__ __device__ __forceinline__ float tiny_normal<float>() { return 1.17549435e-38f; }
template <>
__host__ __device__ __forceinline__ double tiny_normal<double>() { return 2.2250738585072014e-308; }

// ---------------------------------------------------------------------------
// internal lattice ordering
//   fine index i = c * Vb + l; c = block (= coarse site), l = site inside the block.
//   Blocks: all red blocks (even block-coordinate sum) first, then black, each
//   group in lexicographic block order.  Inside a block: even sites first, then
//   odd, each group lexicographic.  Directions d = 2 mu + (backward ? 1 : 0).
// ---------------------------------------------------------------------------
// Per-site (AoS) copies of the FP32 links and site terms for the SAP block solver: all
// components of one site sit together, so each is a vector load at a fixed offset from the
// site's base address (the [comp][V] layout needs a separate offset k V per component).
struct LinksAoS {
    const float4* p;  // [V][4][5]: U_mu(x) as 9 complex (18 floats) + 2 padding floats
};
struct CloverAoS {
    const float4* p;  // [V][18]: the 72 packed reals of the site's two hermitian 6x6 blocks
};
// the same per-site copies in FP16 (half-precision V-cycle): FP32 arithmetic on load
struct LinksAoS16 {
    const uint4* p;  // [V][4][3]: U_mu(x) as 9 complex halves (36 bytes) + 12 padding bytes
};
struct CloverAoS16 {
    const uint4* p;  // [V][9]: the 72 packed reals as halves
};

struct Geom {
    int V;       // fine sites
    int Vb;      // sites per block
    int NB;      // blocks = coarse sites
    int vb_shift;  // log2(Vb) when Vb is a power of two, else -1
    int blk44;     // 1 when the blocks are 4^4 (the specialised SAP kernel applies)
    const int* lnbr;  // [8][Vb]: local index of the neighbour | (crosses block) << 16
    const int* bnbr;  // [8][NB]: neighbouring block
    const int* blex;  // [NB]: internal index of the block of lexicographic index q (traversal order)
};

__device__ __forceinline__ int block_of(const Geom& g, int i) {
    return g.vb_shift >= 0 ? (i >> g.vb_shift) : (i / g.Vb);
}

__device__ __forceinline__ int fine_nbr(const Geom& g, int i, int d) {
    int c = block_of(g, i);
    int l = i - c * g.Vb;
    int e = __ldg(g.lnbr + d * g.Vb + l);
    int c2 = (e >> 16) ? __ldg(g.bnbr + d * g.NB + c) : c;
    return c2 * g.Vb + (e & 0xffff);
}

// ---------------------------------------------------------------------------
// launch bookkeeping
// ---------------------------------------------------------------------------
extern std::atomic<unsigned long long> g_launches;  // several host threads may drive handles at once
void set_error(const std::string& msg);

#define DD_LAUNCHED() (::ddamg::g_launches++)

#define DD_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t _e = (call);                                                          \
        if (_e != cudaSuccess) {                                                          \
            ::ddamg::set_error(std::string(#call) + ": " + cudaGetErrorString(_e));       \
            return DDAMG_ERR_CUDA;                                                        \
        }                                                                                 \
    } while (0)

#define DD_CHECK_LAUNCH()                                                                 \
    do {                                                                                  \
        DD_LAUNCHED();                                                                    \
        cudaError_t _e = cudaGetLastError();                                              \
        if (_e != cudaSuccess) {                                                          \
            ::ddamg::set_error(std::string("kernel launch: ") + cudaGetErrorString(_e));  \
            return DDAMG_ERR_CUDA;                                                        \
        }                                                                                 \
    } while (0)

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace ddamg
