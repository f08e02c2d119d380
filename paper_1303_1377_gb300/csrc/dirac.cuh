// Device helpers of the Wilson-clover operator (Sec. 2.2) shared by the fine
// kernels and the coarse-stencil assembly.
#pragma once
#include <cuda_fp16.h>

#include "common.cuh"

namespace ddamg {

// ---------------------------------------------------------------------------
// spin structure of the hops.  In the chiral basis gamma_mu = [[0, B],[B^H, 0]]
// with a monomial 2x2 block B_mu (one entry per row, a power of i), so
//   (I -+ gamma_mu) psi = [h ; -+ B^H h],  h = psi_up -+ B psi_low.
// SpinB<MU>::c0,p0 : row 0 of B reads column c0 with factor i^p0; likewise row 1,
// and the same for B^H (h-prefixed).
// ---------------------------------------------------------------------------
template <int MU> struct SpinB;
template <> struct SpinB<0> { enum { c0 = 1, p0 = 1, c1 = 0, p1 = 1, hc0 = 1, hp0 = 3, hc1 = 0, hp1 = 3 }; };
template <> struct SpinB<1> { enum { c0 = 1, p0 = 2, c1 = 0, p1 = 0, hc0 = 1, hp0 = 0, hc1 = 0, hp1 = 2 }; };
template <> struct SpinB<2> { enum { c0 = 0, p0 = 1, c1 = 1, p1 = 3, hc0 = 0, hp0 = 3, hc1 = 1, hp1 = 1 }; };
template <> struct SpinB<3> { enum { c0 = 0, p0 = 0, c1 = 1, p1 = 0, hc0 = 0, hp0 = 0, hc1 = 1, hp1 = 0 }; };

// runtime form of SpinB (same entries), for rolled loops over the eight directions:
// [mu][0..7] = c0, p0, c1, p1, hc0, hp0, hc1, hp1
__constant__ unsigned char c_spinb[4][8] = {{1, 1, 0, 1, 1, 3, 0, 3}, {1, 2, 0, 0, 1, 0, 0, 2}, {0, 1, 1, 3, 0, 3, 1, 1},
                                             {0, 0, 1, 0, 0, 0, 1, 0}};

template <typename T>
__device__ __forceinline__ cplx<T> ipow_rt(cplx<T> a, int p) {
    cplx<T> b = (p & 1) ? mk(-a.im, a.re) : a;
    return (p & 2) ? mk(-b.re, -b.im) : b;
}

template <typename T>
struct Spinor {
    cplx<T> v[12];
};

template <typename T, typename Ts>
__device__ __forceinline__ void load_spinor(Spinor<T>& s, const cplx<Ts>* __restrict__ f, int V, int i) {
#pragma unroll
    for (int k = 0; k < 12; ++k) s.v[k] = ccast<T>(f[(size_t)k * V + i]);
}

template <typename T>
__device__ __forceinline__ void load_link(cplx<T> (&W)[9], const cplx<T>* __restrict__ U, int V, int mu, int i) {
#pragma unroll
    for (int q = 0; q < 9; ++q) W[q] = ldg_c(U + (size_t)(mu * 9 + q) * V + i);
}

__device__ __forceinline__ void load_link(cplx<float> (&W)[9], const LinksAoS& U, int /*V*/, int mu, int i) {
    const float4* q = U.p + ((size_t)i * 4 + mu) * 5;
    const float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3), e = __ldg(q + 4);
    W[0] = mk(a.x, a.y), W[1] = mk(a.z, a.w), W[2] = mk(b.x, b.y), W[3] = mk(b.z, b.w), W[4] = mk(c.x, c.y);
    W[5] = mk(c.z, c.w), W[6] = mk(d.x, d.y), W[7] = mk(d.z, d.w), W[8] = mk(e.x, e.y);
}
__device__ __forceinline__ float2 h2f(unsigned u) { return __half22float2(*reinterpret_cast<const __half2*>(&u)); }
__device__ __forceinline__ void load_link(cplx<float> (&W)[9], const LinksAoS16& U, int /*V*/, int mu, int i) {
    const uint4* q = U.p + ((size_t)i * 4 + mu) * 3;
    const uint4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
    const unsigned w[9] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float2 f = h2f(w[k]);
        W[k] = mk(f.x, f.y);
    }
}
// acc += hop of psi_n (the neighbour spinor) through link W in direction MU,
// FWD: (I - gamma_mu) (x) W with W = U_mu(x);  !FWD: (I + gamma_mu) (x) W^H with W = U_mu(x - mu).
// acc collects  [g ; -s B^H g],  g = W h (or W^H h), s = +1 forward / -1 backward.
template <int MU, bool FWD, typename T>
__device__ __forceinline__ void hop_acc(Spinor<T>& acc, const Spinor<T>& pn, const cplx<T> (&W)[9]) {
    using B = SpinB<MU>;
    cplx<T> h[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cplx<T> b0 = ipow<B::p0>(pn.v[(2 + B::c0) * 3 + c]);
        cplx<T> b1 = ipow<B::p1>(pn.v[(2 + B::c1) * 3 + c]);
        if (FWD) {
            h[0][c] = pn.v[0 * 3 + c] - b0;
            h[1][c] = pn.v[1 * 3 + c] - b1;
        } else {
            h[0][c] = pn.v[0 * 3 + c] + b0;
            h[1][c] = pn.v[1 * 3 + c] + b1;
        }
    }
    cplx<T> g[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cplx<T> t = czero<T>();
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (FWD) cmac(t, W[a * 3 + b], h[s][b]);
                else cmac_conj(t, W[b * 3 + a], h[s][b]);
            }
            g[s][a] = t;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc.v[0 * 3 + c] = acc.v[0 * 3 + c] + g[0][c];
        acc.v[1 * 3 + c] = acc.v[1 * 3 + c] + g[1][c];
        cplx<T> l0 = ipow<B::hp0>(g[B::hc0][c]);
        cplx<T> l1 = ipow<B::hp1>(g[B::hc1][c]);
        if (FWD) {  // -s = -1
            acc.v[2 * 3 + c] = acc.v[2 * 3 + c] - l0;
            acc.v[3 * 3 + c] = acc.v[3 * 3 + c] - l1;
        } else {
            acc.v[2 * 3 + c] = acc.v[2 * 3 + c] + l0;
            acc.v[3 * 3 + c] = acc.v[3 * 3 + c] + l1;
        }
    }
}

// hop_acc with the direction mu and the orientation given at run time
template <typename T>
__device__ __forceinline__ void hop_acc_rt(Spinor<T>& acc, const Spinor<T>& pn, const cplx<T> (&W)[9], int mu, bool fwd) {
    const int c0 = c_spinb[mu][0], p0 = c_spinb[mu][1], c1 = c_spinb[mu][2], p1 = c_spinb[mu][3];
    const int hc0 = c_spinb[mu][4], hp0 = c_spinb[mu][5], hc1 = c_spinb[mu][6], hp1 = c_spinb[mu][7];
    const T sg = fwd ? T(-1) : T(1);
    cplx<T> h[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cplx<T> l2 = pn.v[2 * 3 + c], l3 = pn.v[3 * 3 + c];
        cplx<T> b0 = ipow_rt(c0 ? l3 : l2, p0);
        cplx<T> b1 = ipow_rt(c1 ? l3 : l2, p1);
        h[0][c] = pn.v[0 * 3 + c] + sg * b0;
        h[1][c] = pn.v[1 * 3 + c] + sg * b1;
    }
    cplx<T> g[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cplx<T> t = czero<T>();
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                cplx<T> wf = W[a * 3 + b], wb = conj(W[b * 3 + a]);
                cmac(t, fwd ? wf : wb, h[s][b]);
            }
            g[s][a] = t;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc.v[0 * 3 + c] = acc.v[0 * 3 + c] + g[0][c];
        acc.v[1 * 3 + c] = acc.v[1 * 3 + c] + g[1][c];
        cplx<T> l0 = ipow_rt(hc0 ? g[1][c] : g[0][c], hp0);
        cplx<T> l1 = ipow_rt(hc1 ? g[1][c] : g[0][c], hp1);
        acc.v[2 * 3 + c] = acc.v[2 * 3 + c] + sg * l0;
        acc.v[3 * 3 + c] = acc.v[3 * 3 + c] + sg * l1;
    }
}

// y = A x for a site term stored as two packed hermitian 6x6 blocks
template <typename T>
__device__ __forceinline__ void herm_apply(const T* __restrict__ cl, int V, int i, const Spinor<T>& x, Spinor<T>& y) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const T* base = cl + (size_t)(h * 36) * V + i;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            T d = __ldg(base + (size_t)a * V);
            y.v[h * 6 + a] = d * x.v[h * 6 + a];
        }
        int q = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
#pragma unroll
            for (int b = a + 1; b < 6; ++b) {
                cplx<T> m = mk(__ldg(base + (size_t)(6 + 2 * q) * V), __ldg(base + (size_t)(7 + 2 * q) * V));
                cmac(y.v[h * 6 + a], m, x.v[h * 6 + b]);
                cmac_conj(y.v[h * 6 + b], m, x.v[h * 6 + a]);
                ++q;
            }
        }
    }
}

// the same product with the site term read from its FP16 per-site copy (9 x 16 bytes per site):
// block h's 36 halves start at half 36 h, inside the aligned 16-byte words 4h .. 4h + 4
__device__ __forceinline__ void herm_apply(const CloverAoS16& cl, int /*V*/, int i, const Spinor<float>& x, Spinor<float>& y) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint4* q = cl.p + (size_t)i * 9 + 4 * h;
        unsigned w[20];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const uint4 v = __ldg(q + k);
            w[4 * k] = v.x, w[4 * k + 1] = v.y, w[4 * k + 2] = v.z, w[4 * k + 3] = v.w;
        }
        const int o = 2 * h;  // block h's first half is word o (each word holds two halves)
        auto cf = [&](int j) -> float {
            const float2 f = h2f(w[o + j / 2]);
            return (j & 1) ? f.y : f.x;
        };
#pragma unroll
        for (int a2 = 0; a2 < 6; ++a2) y.v[h * 6 + a2] = cf(a2) * x.v[h * 6 + a2];
        int m = 0;
#pragma unroll
        for (int a2 = 0; a2 < 6; ++a2) {
#pragma unroll
            for (int b2 = a2 + 1; b2 < 6; ++b2) {
                const cplx<float> e = mk(cf(6 + 2 * m), cf(7 + 2 * m));
                cmac(y.v[h * 6 + a2], e, x.v[h * 6 + b2]);
                cmac_conj(y.v[h * 6 + b2], e, x.v[h * 6 + a2]);
                ++m;
            }
        }
    }
}
// the same product with the site term read from its per-site copy (9 float4 per block)
__device__ __forceinline__ void herm_apply(const CloverAoS& cl, int /*V*/, int i, const Spinor<float>& x, Spinor<float>& y) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float4* q = cl.p + (size_t)i * 18 + h * 9;
        float c[36];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float4 v = __ldg(q + k);
            c[4 * k] = v.x, c[4 * k + 1] = v.y, c[4 * k + 2] = v.z, c[4 * k + 3] = v.w;
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) y.v[h * 6 + a] = c[a] * x.v[h * 6 + a];
        int m = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
#pragma unroll
            for (int b = a + 1; b < 6; ++b) {
                const cplx<float> e = mk(c[6 + 2 * m], c[7 + 2 * m]);
                cmac(y.v[h * 6 + a], e, x.v[h * 6 + b]);
                cmac_conj(y.v[h * 6 + b], e, x.v[h * 6 + a]);
                ++m;
            }
        }
    }
}

}  // namespace ddamg
