// Fine-grid kernels: clover-improved Wilson Dslash (Sec. 2.2), clover term and
// its even-site inverses, and the fused red-black SAP block solver (Sec. 2.3,
// local odd-even MR of Sec. 6).
//
// Field layouts (internal site order, see common.cuh):
//   spinor  cplx<T>[nrhs][12][V]  component k = spin*3 + colour (SoA: coalesced per component)
//   links   cplx<T>[4][9][V]      U_mu(x)[a][b] at ((mu*9 + a*3 + b) * V + x)
//   clover  T[72][V]              two hermitian 6x6 chiral blocks (spins {0,1}, {2,3}),
//                                 each 6 real diagonal entries + 15 complex upper entries
#include <cuda_fp16.h>

#include "kernels.h"
#include "dirac.cuh"
#include "dw.cuh"

namespace ddamg {

// gamma_mu gamma_nu for the six planes mu < nu in the chiral basis of Sec. 2.2,
// restricted to its two 2x2 chiral blocks: [plane][half][s][t] (re, im)
__constant__ double c_gg[6][2][2][2][2];

// ---------------------------------------------------------------------------
// 4^4 blocks.  Local order of a block (common.cuh): parity p (even first), then rank = lex >> 1
// among the sites of that parity, lex = ((y0 * 4 + y1) * 4 + y2) * 4 + y3.  Neighbours follow from
// the in-block lexicographic index and the (warp-uniform) neighbouring blocks, with no table load
// per site.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lex44_of_local(int l) {
    const int p = l >> 7, k = l & 127, row = k >> 1;  // row = y0 * 16 + y1 * 4 + y2
    const int q = __popc(row & 0x15) & 1;             // parity of y0 + y1 + y2
    return 4 * row + ((p ^ q) & 1) + 2 * (k & 1);     // y3 = (p - q) mod 2 + 2 (k mod 2)
}
// global index of the neighbour of local site (lex L, parity p) of block c in direction MU,
// forward or backward; bn = the neighbouring block in that direction
template <int MU, bool FWD>
__device__ __forceinline__ int nbr44(int L, int p, int c, int bn) {
    constexpr int SH = 2 * (3 - MU), S = 1 << SH;
    const int y = (L >> SH) & 3;
    const bool cross = FWD ? y == 3 : y == 0;
    const int L2 = FWD ? (cross ? L - 3 * S : L + S) : (cross ? L + 3 * S : L - S);
    return (cross ? bn : c) * 256 + (((p ^ 1) << 7) | (L2 >> 1));
}

template <int MU, typename T, typename Ts, typename UT>
__device__ __forceinline__ void hop_pair_nb(const UT& U, const cplx<Ts>* __restrict__ in, int V, int i, int f, int bk, Spinor<T>& acc) {
    cplx<T> W[9];
    Spinor<T> pn;
    load_link(W, U, V, MU, i);
    load_spinor(pn, in, V, f);
    hop_acc<MU, true>(acc, pn, W);
    load_link(W, U, V, MU, bk);
    load_spinor(pn, in, V, bk);
    hop_acc<MU, false>(acc, pn, W);
}

// out = D in (RESID: out = b - D in) on 4^4 blocks.  CTA = 32 sites of one block x ry right-hand
// sides (one warp per right-hand side, sharing the links and site terms through L1).  The CTAs walk
// the blocks in lexicographic block order, red and black interleaved, so that a block and its
// neighbours in three of the four directions are read close together in time and the neighbours'
// spinors are still in L2.
template <typename T, typename Ts, bool RESID>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 384 : 128, sizeof(T) == 4 ? 2 : 1)
    dslash44_kernel(Geom g, FineOp<T> op, const int* __restrict__ blex, const cplx<Ts>* __restrict__ in, const cplx<T>* __restrict__ b,
                    cplx<T>* __restrict__ out, int nrhs) {
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    const int q = blockIdx.x >> 3;
    const int l = (blockIdx.x & 7) * 32 + threadIdx.x;
    if (r >= nrhs) return;
    const int c = __ldg(blex + q);
    const int i = c * 256 + l;
    const int L = lex44_of_local(l), p = l >> 7;
    int bn[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) bn[d] = __ldg(g.bnbr + d * g.NB + c);
    const size_t off = (size_t)r * 12 * g.V;
    const cplx<Ts>* inr = in + off;
    Spinor<T> acc;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc.v[k] = czero<T>();
    hop_pair_nb<0>(op.U, inr, g.V, i, nbr44<0, true>(L, p, c, bn[0]), nbr44<0, false>(L, p, c, bn[1]), acc);
    hop_pair_nb<1>(op.U, inr, g.V, i, nbr44<1, true>(L, p, c, bn[2]), nbr44<1, false>(L, p, c, bn[3]), acc);
    hop_pair_nb<2>(op.U, inr, g.V, i, nbr44<2, true>(L, p, c, bn[4]), nbr44<2, false>(L, p, c, bn[5]), acc);
    hop_pair_nb<3>(op.U, inr, g.V, i, nbr44<3, true>(L, p, c, bn[6]), nbr44<3, false>(L, p, c, bn[7]), acc);
    Spinor<T> x, y;
    load_spinor(x, inr, g.V, i);
    herm_apply(op.clov, g.V, i, x, y);
    cplx<T>* o = out + off;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        cplx<T> d = y.v[k] - T(0.5) * acc.v[k];
        if (RESID) d = b[off + (size_t)k * g.V + i] - d;
        o[(size_t)k * g.V + i] = d;
    }
}

template <int MU, typename T, typename Ts, typename UT>
__device__ __forceinline__ void hop_pair(const Geom& g, const UT& U, const cplx<Ts>* __restrict__ in, int i, Spinor<T>& acc) {
    cplx<T> W[9];
    Spinor<T> pn;
    int f = fine_nbr(g, i, 2 * MU);
    load_link(W, U, g.V, MU, i);
    load_spinor(pn, in, g.V, f);
    hop_acc<MU, true>(acc, pn, W);
    int bk = fine_nbr(g, i, 2 * MU + 1);
    load_link(W, U, g.V, MU, bk);
    load_spinor(pn, in, g.V, bk);
    hop_acc<MU, false>(acc, pn, W);
}

// out = D in  (RESID: out = b - D in).  in may be of a different precision Ts.
// Thread (x, y) of a CTA: site tile * 32 + x, right-hand side blockIdx.y * blockDim.y + y, so the
// warps of one CTA cover the same 32 sites for several right-hand sides and share the links and
// site terms through L1; each warp's spinor loads stay 32 consecutive sites of one field.
template <typename T, typename Ts, bool RESID>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 384 : 128, sizeof(T) == 4 ? 2 : 1) dslash_kernel(Geom g, FineOp<T> op, const cplx<Ts>* __restrict__ in,
                                                     const cplx<T>* __restrict__ b, cplx<T>* __restrict__ out, int nrhs) {
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    const int i = blockIdx.x * 32 + threadIdx.x;
    if (i >= g.V || r >= nrhs) return;
    const size_t off = (size_t)r * 12 * g.V;
    const cplx<Ts>* inr = in + off;
    Spinor<T> acc;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc.v[k] = czero<T>();
    hop_pair<0>(g, op.U, inr, i, acc);
    hop_pair<1>(g, op.U, inr, i, acc);
    hop_pair<2>(g, op.U, inr, i, acc);
    hop_pair<3>(g, op.U, inr, i, acc);
    Spinor<T> x, y;
    load_spinor(x, inr, g.V, i);
    herm_apply(op.clov, g.V, i, x, y);
    cplx<T>* o = out + off;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        cplx<T> d = y.v[k] - T(0.5) * acc.v[k];
        if (RESID) d = b[off + (size_t)k * g.V + i] - d;
        o[(size_t)k * g.V + i] = d;
    }
}

template <typename T, typename Ts>
int launch_dslash(const Geom& g, const FineOp<T>& op, const cplx<Ts>* in, const cplx<T>* b, cplx<T>* out, int nrhs,
                  cudaStream_t st) {
    const int ry = std::min(nrhs, sizeof(T) == 4 ? 12 : 4);  // right-hand sides per CTA
    if (g.blk44 && g.blex) {
        const dim3 grid((unsigned)g.NB * 8, (unsigned)ceil_div(nrhs, ry)), block(32, ry);
        if (b)
            dslash44_kernel<T, Ts, true><<<grid, block, 0, st>>>(g, op, g.blex, in, b, out, nrhs);
        else
            dslash44_kernel<T, Ts, false><<<grid, block, 0, st>>>(g, op, g.blex, in, b, out, nrhs);
        DD_CHECK_LAUNCH();
        return 0;
    }
    const dim3 grid((unsigned)ceil_div(g.V, 32), (unsigned)ceil_div(nrhs, ry)), block(32, ry);
    if (b)
        dslash_kernel<T, Ts, true><<<grid, block, 0, st>>>(g, op, in, b, out, nrhs);
    else
        dslash_kernel<T, Ts, false><<<grid, block, 0, st>>>(g, op, in, b, out, nrhs);
    DD_CHECK_LAUNCH();
    return 0;
}

template int launch_dslash<double, double>(const Geom&, const FineOp<double>&, const cplx<double>*, const cplx<double>*,
                                           cplx<double>*, int, cudaStream_t);
template int launch_dslash<double, float>(const Geom&, const FineOp<double>&, const cplx<float>*, const cplx<double>*,
                                          cplx<double>*, int, cudaStream_t);
template int launch_dslash<float, float>(const Geom&, const FineOp<float>&, const cplx<float>*, const cplx<float>*,
                                         cplx<float>*, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Red-black SAP: one launch per colour.  A CTA owns one block of that colour and
// one right-hand side: it forms r = b - D z on its block (neighbouring blocks are
// of the other colour and are not written in this launch), solves D_i e = r_i by
// odd-even MR (mr_steps steps, zero initial guess) and adds e to z.
// Thread t < Vb/2 owns the even site t and the odd site Vb/2 + t of the block.
// ---------------------------------------------------------------------------

// sum over in-block neighbours of the hops of D applied to a block-local field
// held in shared memory (sm[k * H + local index]), at local site l (global i).
template <int MU, typename T, typename UT>
__device__ __forceinline__ void block_hop_pair(const Geom& g, const UT& U, const cplx<T>* sm, int H, int base_local, int l, int i,
                                               int blk, Spinor<T>& acc) {
    cplx<T> W[9];
    Spinor<T> pn;
    int e = __ldg(g.lnbr + (2 * MU) * g.Vb + l);
    if (!(e >> 16)) {
        int ln = (e & 0xffff) - base_local;
#pragma unroll
        for (int k = 0; k < 12; ++k) pn.v[k] = sm[k * H + ln];
        load_link(W, U, g.V, MU, i);
        hop_acc<MU, true>(acc, pn, W);
    }
    e = __ldg(g.lnbr + (2 * MU + 1) * g.Vb + l);
    if (!(e >> 16)) {
        int lnb = e & 0xffff;
        int ln = lnb - base_local;
#pragma unroll
        for (int k = 0; k < 12; ++k) pn.v[k] = sm[k * H + ln];
        load_link(W, U, g.V, MU, blk * g.Vb + lnb);
        hop_acc<MU, false>(acc, pn, W);
    }
}

template <typename T, typename UT>
__device__ __forceinline__ void block_hops(const Geom& g, const UT& U, const cplx<T>* sm, int H, int base_local, int l, int i, int blk,
                                           Spinor<T>& acc) {
#pragma unroll
    for (int k = 0; k < 12; ++k) acc.v[k] = czero<T>();
    block_hop_pair<0>(g, U, sm, H, base_local, l, i, blk, acc);
    block_hop_pair<1>(g, U, sm, H, base_local, l, i, blk, acc);
    block_hop_pair<2>(g, U, sm, H, base_local, l, i, blk, acc);
    block_hop_pair<3>(g, U, sm, H, base_local, l, i, blk, acc);
}

// full D at one site with z read from global memory (residual)
template <typename T, typename OpT>
__device__ __forceinline__ void site_D(const Geom& g, const OpT& op, const cplx<T>* __restrict__ z, int i, Spinor<T>& out) {
    Spinor<T> acc;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc.v[k] = czero<T>();
    hop_pair<0>(g, op.U, z, i, acc);
    hop_pair<1>(g, op.U, z, i, acc);
    hop_pair<2>(g, op.U, z, i, acc);
    hop_pair<3>(g, op.U, z, i, acc);
    Spinor<T> x;
    load_spinor(x, z, g.V, i);
    herm_apply(op.clov, g.V, i, x, out);
#pragma unroll
    for (int k = 0; k < 12; ++k) out.v[k] = out.v[k] - T(0.5) * acc.v[k];
}

template <typename T>
__device__ __forceinline__ void block_reduce3(T& a, T& b, T& c, T* red) {
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
        red[3 * w] = a;
        red[3 * w + 1] = b;
        red[3 * w + 2] = c;
    }
    __syncthreads();
    a = b = c = T(0);
    for (int q = 0; q < nw; ++q) {
        a += red[3 * q];
        b += red[3 * q + 1];
        c += red[3 * q + 2];
    }
}

// reduction over the HT threads of one slot (slots are whole warps)
template <typename T>
__device__ __forceinline__ void block_reduce3_slot(T& a, T& b, T& c, T* red, int HT) {
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    const int w = (threadIdx.x % HT) >> 5, lane = threadIdx.x & 31, nw = HT >> 5;
    __syncthreads();
    if (lane == 0) {
        red[3 * w] = a;
        red[3 * w + 1] = b;
        red[3 * w + 2] = c;
    }
    __syncthreads();
    a = b = c = T(0);
    for (int q = 0; q < nw; ++q) {
        a += red[3 * q];
        b += red[3 * q + 1];
        c += red[3 * q + 2];
    }
}

// R right-hand-side slots per CTA (R * HT threads, HT = Vb/2 rounded up to a warp):
// the slots share the block's links and site terms through L1.
template <typename T, int R>
__global__ void __launch_bounds__(128 * R, 1) sap_colour_kernel(Geom g, FineOp<T> op, const cplx<T>* __restrict__ bsrc,
                                                                cplx<T>* __restrict__ z, int colour, int nrhs, int mr_steps) {
    extern __shared__ unsigned char smem_raw[];
    const int H = g.Vb / 2;
    const int HT = blockDim.x / R;
    const int slot = threadIdx.x / HT;
    const int t = threadIdx.x % HT;
    cplx<T>* SE = reinterpret_cast<cplx<T>*>(smem_raw) + (size_t)slot * 36 * H;  // [12][H] even-site work vector
    cplx<T>* SO = SE + 12 * H;                                                   // [12][H] odd-site work vector (rho, then x_o)
    cplx<T>* SR = SO + 12 * H;                                                   // [12][H] r_e
    T* red = reinterpret_cast<T*>(reinterpret_cast<cplx<T>*>(smem_raw) + (size_t)R * 36 * H) + (size_t)slot * 3 * (HT / 32);

    const int nslots = (nrhs + R - 1) / R;
    const int r = (blockIdx.x % nslots) * R + slot;
    const int blk = colour * (g.NB / 2) + blockIdx.x / nslots;
    const bool act = t < H && r < nrhs;
    const int le = t, lo = H + t;
    const int ie = blk * g.Vb + le, io = blk * g.Vb + lo;
    const size_t off = (size_t)(r < nrhs ? r : 0) * 12 * g.V;
    const cplx<T>* b = bsrc + off;
    cplx<T>* zr = z + off;

    Spinor<T> ro, xo, tmp, tmp2;
    // 1. residual r = b - D z on both sites; even part: SE <- A_ee^{-1} r_e, SR <- r_e
    if (act) {
        site_D(g, op, zr, ie, tmp);
#pragma unroll
        for (int k = 0; k < 12; ++k) tmp.v[k] = b[(size_t)k * g.V + ie] - tmp.v[k];
#pragma unroll
        for (int k = 0; k < 12; ++k) SR[k * H + t] = tmp.v[k];
        herm_apply(op.clovinv, g.V, ie, tmp, tmp2);
#pragma unroll
        for (int k = 0; k < 12; ++k) SE[k * H + t] = tmp2.v[k];
        site_D(g, op, zr, io, tmp);
#pragma unroll
        for (int k = 0; k < 12; ++k) ro.v[k] = b[(size_t)k * g.V + io] - tmp.v[k];
    }
    __syncthreads();
    // 2. reduced right-hand side rho = r_o - D_oe A_ee^{-1} r_e ; x_o = 0
    if (act) {
        block_hops(g, op.U, SE, H, 0, lo, io, blk, tmp);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            ro.v[k] = ro.v[k] - T(-0.5) * tmp.v[k];  // block hops of D carry the -1/2
            SO[k * H + t] = ro.v[k];
            xo.v[k] = czero<T>();
        }
    }
    __syncthreads();
    // 3. MR steps on S = A_oo - D_oe A_ee^{-1} D_eo
    for (int it = 0; it < mr_steps; ++it) {
        if (act) {  // even: SE <- A_ee^{-1} D_eo rho
            block_hops(g, op.U, SO, H, H, le, ie, blk, tmp);
#pragma unroll
            for (int k = 0; k < 12; ++k) tmp.v[k] = T(-0.5) * tmp.v[k];
            herm_apply(op.clovinv, g.V, ie, tmp, tmp2);
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int k = 0; k < 12; ++k) SE[k * H + t] = tmp2.v[k];
        }
        __syncthreads();
        T num_re = 0, num_im = 0, den = 0;
        if (act) {  // odd: t = A_oo rho - D_oe SE
            herm_apply(op.clov, g.V, io, ro, tmp2);
            block_hops(g, op.U, SE, H, 0, lo, io, blk, tmp);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                tmp.v[k] = tmp2.v[k] + T(0.5) * tmp.v[k];
                num_re += tmp.v[k].re * ro.v[k].re + tmp.v[k].im * ro.v[k].im;
                num_im += tmp.v[k].re * ro.v[k].im - tmp.v[k].im * ro.v[k].re;
                den += norm2(tmp.v[k]);
            }
        }
        block_reduce3_slot(num_re, num_im, den, red, HT);
        cplx<T> alpha = czero<T>();
        if (den > tiny_normal<T>()) alpha = mk(num_re / den, num_im / den);
        if (act) {
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                cmac(xo.v[k], alpha, ro.v[k]);
                ro.v[k] = ro.v[k] - alpha * tmp.v[k];
                SO[k * H + t] = ro.v[k];
            }
        }
        __syncthreads();
    }
    // 4. back-substitution x_e = A_ee^{-1} (r_e - D_eo x_o) and update z
    if (act) {
#pragma unroll
        for (int k = 0; k < 12; ++k) SO[k * H + t] = xo.v[k];
    }
    __syncthreads();
    if (act) {
        block_hops(g, op.U, SO, H, H, le, ie, blk, tmp);
#pragma unroll
        for (int k = 0; k < 12; ++k) tmp.v[k] = SR[k * H + t] + T(0.5) * tmp.v[k];
        herm_apply(op.clovinv, g.V, ie, tmp, tmp2);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            zr[(size_t)k * g.V + ie] = zr[(size_t)k * g.V + ie] + tmp2.v[k];
            zr[(size_t)k * g.V + io] = zr[(size_t)k * g.V + io] + xo.v[k];
        }
    }
}

// ---------------------------------------------------------------------------
// SAP block solve with all per-site MR state in shared memory (r_e, rho, x_o and
// the even work vector): only temporaries live in registers, so the kernel runs
// at 128 registers and four CTAs per SM.  One CTA = one block of the colour and
// one right-hand side; thread t owns the even site t and the odd site H + t.
// ---------------------------------------------------------------------------
// R right-hand sides ride in adjacent lanes (lane = R * site-pair + slot), so the
// link and site-term loads of the R lanes of one site are a single transaction.
// HC: the half-block size as a compile-time constant (0: taken from g at run time), which turns
// every shared-memory offset k * H into an immediate.
template <typename T, int R, typename OpT, int HC = 0>
__global__ void __launch_bounds__(128 * R, (R == 1 ? 4 : 1)) sap_colour_lean_kernel(Geom g, OpT op, const cplx<T>* __restrict__ bsrc,
                                                                                     cplx<T>* __restrict__ z, int colour, int nrhs,
                                                                                     int mr_steps) {
    extern __shared__ unsigned char smem_raw[];
    const int H = HC ? HC : g.Vb / 2;
    const int slot = threadIdx.x % R;
    const int t = threadIdx.x / R;
    const int slot_stride = 36 * H + 4;  // complex numbers per slot (+4: bank offset between slots)
    cplx<T>* SE = reinterpret_cast<cplx<T>*>(smem_raw) + (size_t)slot * slot_stride;  // [12][H] even work vector
    cplx<T>* SO = SE + 12 * H;                                                         // [12][H] rho
    cplx<T>* SX = SO + 12 * H;                                                         // [12][H] x_o (first: r_o)
    T* red = reinterpret_cast<T*>(reinterpret_cast<cplx<T>*>(smem_raw) + (size_t)R * slot_stride);  // [nwarps][R][3]
    const int ngroups = (nrhs + R - 1) / R;
    const int r = (blockIdx.x % ngroups) * R + slot;
    const int blk = colour * (g.NB / 2) + blockIdx.x / ngroups;
    const bool act = t < H && r < nrhs;
    const int le = t, lo = H + t;
    const int ie = blk * g.Vb + le, io = blk * g.Vb + lo;
    const size_t off = (size_t)(r < nrhs ? r : 0) * 12 * g.V;
    const cplx<T>* b = bsrc + off;
    cplx<T>* zr = z + off;
    {
        Spinor<T> tmp, tmp2;
        if (act) {
            site_D(g, op, zr, ie, tmp);
#pragma unroll
            for (int k = 0; k < 12; ++k) tmp.v[k] = b[(size_t)k * g.V + ie] - tmp.v[k];
            herm_apply(op.clovinv, g.V, ie, tmp, tmp2);
#pragma unroll
            for (int k = 0; k < 12; ++k) SE[k * H + t] = tmp2.v[k];
            site_D(g, op, zr, io, tmp);
#pragma unroll
            for (int k = 0; k < 12; ++k) SX[k * H + t] = b[(size_t)k * g.V + io] - tmp.v[k];
        }
    }
    __syncthreads();  // every read of z in this block is done: z may be updated from here on
    if (act) {  // z_e += A_ee^{-1} r_e (the even part of the correction that does not depend on x_o);
                // rho = r_o - D_oe A_ee^{-1} r_e ; x_o = 0
#pragma unroll
        for (int k = 0; k < 12; ++k) zr[(size_t)k * g.V + ie] = zr[(size_t)k * g.V + ie] + SE[k * H + t];
        Spinor<T> hs;
        block_hops(g, op.U, SE, H, 0, lo, io, blk, hs);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            SO[k * H + t] = SX[k * H + t] + T(0.5) * hs.v[k];
            SX[k * H + t] = czero<T>();
        }
    }
    __syncthreads();
    for (int it = 0; it < mr_steps; ++it) {
        if (act) {  // even: SE = A_ee^{-1} D_eo rho  (reads only SO, writes only SE)
            Spinor<T> hs, tmp2;
            block_hops(g, op.U, SO, H, H, le, ie, blk, hs);
#pragma unroll
            for (int k = 0; k < 12; ++k) hs.v[k] = T(-0.5) * hs.v[k];
            herm_apply(op.clovinv, g.V, ie, hs, tmp2);
#pragma unroll
            for (int k = 0; k < 12; ++k) SE[k * H + t] = tmp2.v[k];
        }
        __syncthreads();
        T num_re = 0, num_im = 0, den = 0;
        Spinor<T> sr;
        if (act) {  // odd: S rho = A_oo rho + 1/2 hops(SE)
            Spinor<T> rho, hs;
#pragma unroll
            for (int k = 0; k < 12; ++k) rho.v[k] = SO[k * H + t];
            herm_apply(op.clov, g.V, io, rho, sr);
            block_hops(g, op.U, SE, H, 0, lo, io, blk, hs);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                sr.v[k] = sr.v[k] + T(0.5) * hs.v[k];
                num_re += sr.v[k].re * rho.v[k].re + sr.v[k].im * rho.v[k].im;
                num_im += sr.v[k].re * rho.v[k].im - sr.v[k].im * rho.v[k].re;
                den += norm2(sr.v[k]);
            }
        }
        // reduction over the site pairs of each slot: lanes of equal slot first, then warps
#pragma unroll
        for (int o = R; o < 32; o <<= 1) {
            num_re += __shfl_xor_sync(0xffffffffu, num_re, o);
            num_im += __shfl_xor_sync(0xffffffffu, num_im, o);
            den += __shfl_xor_sync(0xffffffffu, den, o);
        }
        const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        __syncthreads();
        if ((threadIdx.x & 31) < R) {
            red[(w * R + slot) * 3] = num_re;
            red[(w * R + slot) * 3 + 1] = num_im;
            red[(w * R + slot) * 3 + 2] = den;
        }
        __syncthreads();
        num_re = num_im = den = T(0);
        for (int q = 0; q < nw; ++q) {
            num_re += red[(q * R + slot) * 3];
            num_im += red[(q * R + slot) * 3 + 1];
            den += red[(q * R + slot) * 3 + 2];
        }
        cplx<T> alpha = czero<T>();
        if (den > tiny_normal<T>()) alpha = mk(num_re / den, num_im / den);
        if (act) {
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                cplx<T> rv = SO[k * H + t];
                cplx<T> xv = SX[k * H + t];
                cmac(xv, alpha, rv);
                SX[k * H + t] = xv;
                SO[k * H + t] = rv - alpha * sr.v[k];
            }
        }
        __syncthreads();
    }
    if (act) {  // x_e = A_ee^{-1} (r_e - D_eo x_o); z += x
        Spinor<T> hs, tmp2;
        block_hops(g, op.U, SX, H, H, le, ie, blk, hs);
#pragma unroll
        for (int k = 0; k < 12; ++k) hs.v[k] = T(0.5) * hs.v[k];  // x_e = A_ee^{-1} r_e (added above) + A_ee^{-1} (1/2 hops x_o)
        herm_apply(op.clovinv, g.V, ie, hs, tmp2);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            zr[(size_t)k * g.V + ie] = zr[(size_t)k * g.V + ie] + tmp2.v[k];
            zr[(size_t)k * g.V + io] = zr[(size_t)k * g.V + io] + SX[k * H + t];
        }
    }
}

// ---------------------------------------------------------------------------
// SAP block solve specialised to 4^4 blocks (H = 128 sites per parity) with four right-hand sides
// in adjacent lanes.  Same algorithm and shared-memory state as sap_colour_lean_kernel; what the
// fixed block shape buys:
//  - in-block neighbours are computed from the site's lexicographic index inside the block, so a
//    hop's shared-memory read and link load wait on no table load;
//  - the MR step size is summed by one warp from the per-warp partials and broadcast through
//    shared memory, instead of every thread summing all partials.
// ---------------------------------------------------------------------------
// in-block hops in direction MU of a site with in-block lexicographic index L; sm holds the field
// on the neighbours' parity, indexed by rank; nb0 = global index of local site 0 of that parity.
template <int MU, typename T, typename UT>
__device__ __forceinline__ void hop_pair44(const UT& U, const cplx<T>* sm, int L, int nb0, int i, Spinor<T>& acc) {
    constexpr int SH = 2 * (3 - MU), S = 1 << SH;
    const int c = (L >> SH) & 3;
    cplx<T> W[9];
    Spinor<T> pn;
    if (c < 3) {
        const int n = (L + S) >> 1;
#pragma unroll
        for (int k = 0; k < 12; ++k) pn.v[k] = sm[k * 128 + n];
        load_link(W, U, 0, MU, i);
        hop_acc<MU, true>(acc, pn, W);
    }
    if (c > 0) {
        const int n = (L - S) >> 1;
#pragma unroll
        for (int k = 0; k < 12; ++k) pn.v[k] = sm[k * 128 + n];
        load_link(W, U, 0, MU, nb0 + n);
        hop_acc<MU, false>(acc, pn, W);
    }
}
template <typename T, typename UT>
__device__ __forceinline__ void hops44(const UT& U, const cplx<T>* sm, int L, int nb0, int i, Spinor<T>& acc) {
#pragma unroll
    for (int k = 0; k < 12; ++k) acc.v[k] = czero<T>();
    hop_pair44<0>(U, sm, L, nb0, i, acc);
    hop_pair44<1>(U, sm, L, nb0, i, acc);
    hop_pair44<2>(U, sm, L, nb0, i, acc);
    hop_pair44<3>(U, sm, L, nb0, i, acc);
}

// full D at local site (lex L, parity p) of block c with z read from global memory (residual)
template <typename T, typename OpT>
__device__ __forceinline__ void site_D44(const Geom& g, const OpT& op, const cplx<T>* __restrict__ z, int c, int L, int p, int i,
                                         const int (&bn)[8], Spinor<T>& out) {
    Spinor<T> acc;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc.v[k] = czero<T>();
    hop_pair_nb<0>(op.U, z, g.V, i, nbr44<0, true>(L, p, c, bn[0]), nbr44<0, false>(L, p, c, bn[1]), acc);
    hop_pair_nb<1>(op.U, z, g.V, i, nbr44<1, true>(L, p, c, bn[2]), nbr44<1, false>(L, p, c, bn[3]), acc);
    hop_pair_nb<2>(op.U, z, g.V, i, nbr44<2, true>(L, p, c, bn[4]), nbr44<2, false>(L, p, c, bn[5]), acc);
    hop_pair_nb<3>(op.U, z, g.V, i, nbr44<3, true>(L, p, c, bn[6]), nbr44<3, false>(L, p, c, bn[7]), acc);
    Spinor<T> x;
    load_spinor(x, z, g.V, i);
    herm_apply(op.clov, g.V, i, x, out);
#pragma unroll
    for (int k = 0; k < 12; ++k) out.v[k] = out.v[k] - T(0.5) * acc.v[k];
}

template <typename OpT>
__global__ void __launch_bounds__(512, 1) sap44_kernel(Geom g, OpT op, const cplx<float>* __restrict__ bsrc, cplx<float>* __restrict__ z,
                                                       int colour, int nrhs, int mr_steps) {
    using T = float;
    constexpr int R = 4, H = 128, NW = 16;
    extern __shared__ unsigned char smem_raw[];
    const int slot = threadIdx.x % R;
    const int t = threadIdx.x / R;
    const int slot_stride = 36 * H + 4;  // complex numbers per slot (+4: bank offset between slots)
    cplx<T>* SE = reinterpret_cast<cplx<T>*>(smem_raw) + (size_t)slot * slot_stride;  // [12][H] even work vector
    cplx<T>* SO = SE + 12 * H;                                                         // [12][H] rho
    cplx<T>* SX = SO + 12 * H;                                                         // [12][H] x_o (first: r_o)
    float4* red = reinterpret_cast<float4*>(reinterpret_cast<cplx<T>*>(smem_raw) + (size_t)R * slot_stride);  // [NW][R]
    cplx<T>* salpha = reinterpret_cast<cplx<T>*>(red + NW * R);                                               // [R]
    const int ngroups = (nrhs + R - 1) / R;
    const int r = (blockIdx.x % ngroups) * R + slot;
    const int blk = colour * (g.NB / 2) + blockIdx.x / ngroups;
    const bool act = r < nrhs;
    const int ie = blk * g.Vb + t, io = blk * g.Vb + H + t;
    const int Le = lex44_of_local(t), Lo = lex44_of_local(H + t);
    const int nb_even = blk * g.Vb, nb_odd = blk * g.Vb + H;  // global index of local site 0 of each parity
    const size_t off = (size_t)(act ? r : 0) * 12 * g.V;
    const cplx<T>* b = bsrc + off;
    cplx<T>* zr = z + off;
    {
        int bn[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) bn[d] = __ldg(g.bnbr + d * g.NB + blk);
        Spinor<T> tmp, tmp2;
        if (act) {
            site_D44(g, op, zr, blk, Le, 0, ie, bn, tmp);
#pragma unroll
            for (int k = 0; k < 12; ++k) tmp.v[k] = b[(size_t)k * g.V + ie] - tmp.v[k];
            herm_apply(op.clovinv, g.V, ie, tmp, tmp2);
#pragma unroll
            for (int k = 0; k < 12; ++k) SE[k * H + t] = tmp2.v[k];
            site_D44(g, op, zr, blk, Lo, 1, io, bn, tmp);
#pragma unroll
            for (int k = 0; k < 12; ++k) SX[k * H + t] = b[(size_t)k * g.V + io] - tmp.v[k];
        }
    }
    __syncthreads();  // every read of z in this block is done: z may be updated from here on
    if (act) {  // z_e += A_ee^{-1} r_e; rho = r_o - D_oe A_ee^{-1} r_e; x_o = 0
#pragma unroll
        for (int k = 0; k < 12; ++k) zr[(size_t)k * g.V + ie] = zr[(size_t)k * g.V + ie] + SE[k * H + t];
        Spinor<T> hs;
        hops44(op.U, SE, Lo, nb_even, io, hs);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            SO[k * H + t] = SX[k * H + t] + T(0.5) * hs.v[k];
            SX[k * H + t] = czero<T>();
        }
    }
    __syncthreads();
    for (int it = 0; it < mr_steps; ++it) {
        if (act) {  // even: SE = A_ee^{-1} D_eo rho
            Spinor<T> hs, tmp2;
            hops44(op.U, SO, Le, nb_odd, ie, hs);
#pragma unroll
            for (int k = 0; k < 12; ++k) hs.v[k] = T(-0.5) * hs.v[k];
            herm_apply(op.clovinv, g.V, ie, hs, tmp2);
#pragma unroll
            for (int k = 0; k < 12; ++k) SE[k * H + t] = tmp2.v[k];
        }
        __syncthreads();
        T num_re = 0, num_im = 0, den = 0;
        Spinor<T> sr;
        if (act) {  // odd: S rho = A_oo rho + 1/2 hops(SE)
            Spinor<T> rho, hs;
#pragma unroll
            for (int k = 0; k < 12; ++k) rho.v[k] = SO[k * H + t];
            herm_apply(op.clov, g.V, io, rho, sr);
            hops44(op.U, SE, Lo, nb_even, io, hs);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                sr.v[k] = sr.v[k] + T(0.5) * hs.v[k];
                num_re += sr.v[k].re * rho.v[k].re + sr.v[k].im * rho.v[k].im;
                num_im += sr.v[k].re * rho.v[k].im - sr.v[k].im * rho.v[k].re;
                den += norm2(sr.v[k]);
            }
        }
        // per-warp partial sums of each slot (lanes of equal slot), then warp 0 sums the warps
#pragma unroll
        for (int o = R; o < 32; o <<= 1) {
            num_re += __shfl_xor_sync(0xffffffffu, num_re, o);
            num_im += __shfl_xor_sync(0xffffffffu, num_im, o);
            den += __shfl_xor_sync(0xffffffffu, den, o);
        }
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane < R) red[w * R + slot] = make_float4(num_re, num_im, den, 0.f);
        __syncthreads();
        if (w == 0) {  // lane = 4 q + slot (slot = lane % R): warps q and q + 8
            const float4 a = red[lane], c = red[32 + lane];
            float nr = a.x + c.x, ni = a.y + c.y, dd = a.z + c.z;
#pragma unroll
            for (int o = R; o < 32; o <<= 1) {
                nr += __shfl_xor_sync(0xffffffffu, nr, o);
                ni += __shfl_xor_sync(0xffffffffu, ni, o);
                dd += __shfl_xor_sync(0xffffffffu, dd, o);
            }
            if (lane < R) salpha[lane] = dd > tiny_normal<T>() ? mk(nr / dd, ni / dd) : czero<T>();
        }
        __syncthreads();
        if (act) {
            const cplx<T> alpha = salpha[slot];
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                cplx<T> rv = SO[k * H + t];
                cplx<T> xv = SX[k * H + t];
                cmac(xv, alpha, rv);
                SX[k * H + t] = xv;
                SO[k * H + t] = rv - alpha * sr.v[k];
            }
        }
        __syncthreads();
    }
    if (act) {  // x_e = A_ee^{-1} (r_e - D_eo x_o); z += x
        Spinor<T> hs, tmp2;
        hops44(op.U, SX, Le, nb_odd, ie, hs);
#pragma unroll
        for (int k = 0; k < 12; ++k) hs.v[k] = T(0.5) * hs.v[k];  // x_e = A_ee^{-1} r_e (added above) + A_ee^{-1} (1/2 hops x_o)
        herm_apply(op.clovinv, g.V, ie, hs, tmp2);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            zr[(size_t)k * g.V + ie] = zr[(size_t)k * g.V + ie] + tmp2.v[k];
            zr[(size_t)k * g.V + io] = zr[(size_t)k * g.V + io] + SX[k * H + t];
        }
    }
}

template <typename OpT>
static int launch_sap44(const Geom& g, const OpT& op, const cplx<float>* b, cplx<float>* z, int colour, int nrhs, int mr_steps,
                        cudaStream_t st) {
    constexpr int R = 4, H = 128, NW = 16;
    const size_t smem = (size_t)R * (36 * H + 4) * sizeof(cplx<float>) + (size_t)NW * R * sizeof(float4) + R * sizeof(cplx<float>);
    // set once per kernel instance (a function-local static initialiser is thread safe)
    static const bool attr = [] {
        cudaFuncSetAttribute(sap44_kernel<OpT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        return true;
    }();
    (void)attr;
    const long long nblk = (long long)(g.NB / 2) * ((nrhs + R - 1) / R);
    sap44_kernel<OpT><<<(unsigned)nblk, R * H, smem, st>>>(g, op, b, z, colour, nrhs, mr_steps);
    DD_CHECK_LAUNCH();
    return 0;
}

template <typename T, int R>
static int launch_sap_r(const Geom& g, const FineOp<T>& op, const cplx<T>* b, cplx<T>* z, int colour, int nrhs, int mr_steps,
                        cudaStream_t st) {
    const int H = g.Vb / 2;
    const int nt = ((H + 31) / 32) * 32;
    size_t smem = (size_t)R * 36 * H * sizeof(cplx<T>) + (size_t)R * 3 * 32 * sizeof(T);
    // set once per kernel instance (a function-local static initialiser is thread safe)
    static const bool attr_set = [] {
        cudaFuncSetAttribute(sap_colour_kernel<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        return true;
    }();
    (void)attr_set;
    long long nblk = (long long)(g.NB / 2) * ((nrhs + R - 1) / R);
    sap_colour_kernel<T, R><<<(unsigned)nblk, R * nt, smem, st>>>(g, op, b, z, colour, nrhs, mr_steps);
    DD_CHECK_LAUNCH();
    return 0;
}

template <typename T, int R, typename OpT, int HC = 0>
static int launch_sap_lean(const Geom& g, const OpT& op, const cplx<T>* b, cplx<T>* z, int colour, int nrhs, int mr_steps,
                           cudaStream_t st) {
    const int H = g.Vb / 2;
    size_t smem = (size_t)R * (36 * H + 4) * sizeof(cplx<T>) + (size_t)(R * H / 32 + 1) * R * 3 * sizeof(T) + 64;
    // set once per kernel instance (a function-local static initialiser is thread safe)
    static const bool attr = [] {
        cudaFuncSetAttribute(sap_colour_lean_kernel<T, R, OpT, HC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        return true;
    }();
    (void)attr;
    long long nblk = (long long)(g.NB / 2) * ((nrhs + R - 1) / R);
    sap_colour_lean_kernel<T, R, OpT, HC><<<(unsigned)nblk, R * H, smem, st>>>(g, op, b, z, colour, nrhs, mr_steps);
    DD_CHECK_LAUNCH();
    return 0;
}

template <typename T>
int launch_sap_colour(const Geom& g, const FineOp<T>& op, const cplx<T>* b, cplx<T>* z, int colour, int nrhs, int mr_steps,
                      cudaStream_t st) {
    const int H = g.Vb / 2;
    if constexpr (sizeof(T) == 4) {
        // four right-hand sides per site in adjacent lanes (needs 4 H to be a whole number of warps)
        if (nrhs >= 4 && (4 * H) % 32 == 0 && 4 * H <= 512) return launch_sap_lean<T, 4>(g, op, b, z, colour, nrhs, mr_steps, st);
        if (H % 32 == 0) return launch_sap_lean<T, 1>(g, op, b, z, colour, nrhs, mr_steps, st);
    }
    if (sizeof(T) == 4 && H <= 128 && nrhs >= 2) return launch_sap_r<T, 2>(g, op, b, z, colour, nrhs, mr_steps, st);
    return launch_sap_r<T, 1>(g, op, b, z, colour, nrhs, mr_steps, st);
}
bool sap_aos_supported(const Geom& g, int nrhs) {
    const int H = g.Vb / 2;
    return (nrhs >= 4 && (4 * H) % 32 == 0 && 4 * H <= 512) || H % 32 == 0;
}
int launch_sap_colour_aos(const Geom& g, const FineOpAoS& op, const cplx<float>* b, cplx<float>* z, int colour, int nrhs, int mr_steps,
                          cudaStream_t st) {
    const int H = g.Vb / 2;
    if (nrhs >= 4 && H == 128 && g.blk44) return launch_sap44(g, op, b, z, colour, nrhs, mr_steps, st);  // 4^4 blocks
    if (nrhs >= 4 && H == 128) return launch_sap_lean<float, 4, FineOpAoS, 128>(g, op, b, z, colour, nrhs, mr_steps, st);
    if (nrhs >= 4 && (4 * H) % 32 == 0 && 4 * H <= 512) return launch_sap_lean<float, 4>(g, op, b, z, colour, nrhs, mr_steps, st);
    if (H % 32 == 0) return launch_sap_lean<float, 1>(g, op, b, z, colour, nrhs, mr_steps, st);
    return -1;
}

int launch_sap_colour_aos16(const Geom& g, const FineOpAoS16& op, const cplx<float>* b, cplx<float>* z, int colour, int nrhs,
                            int mr_steps, cudaStream_t st) {
    const int H = g.Vb / 2;
    if (nrhs >= 4 && H == 128 && g.blk44) return launch_sap44(g, op, b, z, colour, nrhs, mr_steps, st);  // 4^4 blocks
    if (nrhs >= 4 && H == 128) return launch_sap_lean<float, 4, FineOpAoS16, 128>(g, op, b, z, colour, nrhs, mr_steps, st);
    if (nrhs >= 4 && (4 * H) % 32 == 0 && 4 * H <= 512) return launch_sap_lean<float, 4>(g, op, b, z, colour, nrhs, mr_steps, st);
    if (H % 32 == 0) return launch_sap_lean<float, 1>(g, op, b, z, colour, nrhs, mr_steps, st);
    return -1;
}

__device__ __forceinline__ unsigned pack_h2(float a, float b) {
    __half2 v = __floats2half2_rn(a, b);
    return *reinterpret_cast<unsigned*>(&v);
}
__global__ void links_to_aos16_kernel(const cplx<float>* __restrict__ U, uint4* __restrict__ out, int V) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;  // q = site * 4 + mu
    if (q >= 4 * V) return;
    const int i = q / 4, mu = q % 4;
    unsigned w[12];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const cplx<float> u = U[(size_t)(mu * 9 + c) * V + i];
        w[c] = pack_h2(u.re, u.im);
    }
    w[9] = w[10] = w[11] = 0u;
#pragma unroll
    for (int k = 0; k < 3; ++k) out[(size_t)q * 3 + k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
}
int links_to_aos16(const cplx<float>* U, uint4* out, int V, cudaStream_t st) {
    links_to_aos16_kernel<<<ceil_div(4LL * V, 256), 256, 0, st>>>(U, out, V);
    DD_CHECK_LAUNCH();
    return 0;
}
__global__ void clover_to_aos16_kernel(const float* __restrict__ cl, uint4* __restrict__ out, int V) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // q = site * 9 + k
    if (q >= (size_t)9 * V) return;
    const int i = (int)(q / 9), k = (int)(q % 9);
    unsigned w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) w[e] = pack_h2(cl[(size_t)(8 * k + 2 * e) * V + i], cl[(size_t)(8 * k + 2 * e + 1) * V + i]);
    out[q] = make_uint4(w[0], w[1], w[2], w[3]);
}
int clover_to_aos16(const float* cl, uint4* out, int V, cudaStream_t st) {
    clover_to_aos16_kernel<<<ceil_div(9LL * V, 256), 256, 0, st>>>(cl, out, V);
    DD_CHECK_LAUNCH();
    return 0;
}

__global__ void links_to_aos_kernel(const cplx<float>* __restrict__ U, float4* __restrict__ out, int V) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;  // q = site * 4 + mu
    if (q >= 4 * V) return;
    const int i = q / 4, mu = q % 4;
    float f[20];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const cplx<float> u = U[(size_t)(mu * 9 + c) * V + i];
        f[2 * c] = u.re, f[2 * c + 1] = u.im;
    }
    f[18] = f[19] = 0.f;
#pragma unroll
    for (int k = 0; k < 5; ++k) out[(size_t)q * 5 + k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
}
int links_to_aos(const cplx<float>* U, float4* out, int V, cudaStream_t st) {
    links_to_aos_kernel<<<ceil_div(4LL * V, 256), 256, 0, st>>>(U, out, V);
    DD_CHECK_LAUNCH();
    return 0;
}
__global__ void clover_to_aos_kernel(const float* __restrict__ cl, float4* __restrict__ out, int V) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // q = site * 18 + k
    if (q >= (size_t)18 * V) return;
    const int i = (int)(q / 18), k = (int)(q % 18);
    out[q] = make_float4(cl[(size_t)(4 * k) * V + i], cl[(size_t)(4 * k + 1) * V + i], cl[(size_t)(4 * k + 2) * V + i],
                         cl[(size_t)(4 * k + 3) * V + i]);
}
int clover_to_aos(const float* cl, float4* out, int V, cudaStream_t st) {
    clover_to_aos_kernel<<<ceil_div(18LL * V, 256), 256, 0, st>>>(cl, out, V);
    DD_CHECK_LAUNCH();
    return 0;
}

template int launch_sap_colour<double>(const Geom&, const FineOp<double>&, const cplx<double>*, cplx<double>*, int, int, int,
                                       cudaStream_t);
template int launch_sap_colour<float>(const Geom&, const FineOp<float>&, const cplx<float>*, cplx<float>*, int, int, int,
                                      cudaStream_t);

// ---------------------------------------------------------------------------
// Clover term (Sec. 2.2):  A(x) = (m0 + 4) I - c_sw/16 sum_{mu<nu} (gamma_mu gamma_nu) (x) F_mu,nu(x),
// F = Q_mu,nu - Q_mu,nu^H (Q_nu,mu is the same four leaves traversed backwards, i.e. Q_mu,nu^H),
// Q_mu,nu = sum of the four plaquette leaves at x.  Computed in FP64, stored
// packed; the inverse of each 6x6 block by Gauss-Jordan with partial pivoting.
// ---------------------------------------------------------------------------
struct M3 {
    cplx<double> m[9];
};
__device__ __forceinline__ M3 ld3(const cplx<double>* __restrict__ U, int V, int mu, int i) {
    M3 r;
#pragma unroll
    for (int q = 0; q < 9; ++q) r.m[q] = U[(size_t)(mu * 9 + q) * V + i];
    return r;
}
__device__ __forceinline__ M3 mul3(const M3& a, const M3& b) {
    M3 r;
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int y = 0; y < 3; ++y) {
            cplx<double> t = czero<double>();
#pragma unroll
            for (int k = 0; k < 3; ++k) cmac(t, a.m[x * 3 + k], b.m[k * 3 + y]);
            r.m[x * 3 + y] = t;
        }
    return r;
}
__device__ __forceinline__ M3 dag3(const M3& a) {
    M3 r;
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int y = 0; y < 3; ++y) r.m[x * 3 + y] = conj(a.m[y * 3 + x]);
    return r;
}

__global__ void clover_kernel(Geom g, const cplx<double>* __restrict__ U, double m0, double csw, double* __restrict__ clov,
                              double* __restrict__ clovinv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    cplx<double> A[2][6][6];
    for (int h = 0; h < 2; ++h)
        for (int p = 0; p < 6; ++p)
            for (int q = 0; q < 6; ++q) A[h][p][q] = mk(p == q ? m0 + 4.0 : 0.0, 0.0);
    int plane = 0;
    for (int mu = 0; mu < 4; ++mu) {
        for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
            const int fm = 2 * mu, bm = 2 * mu + 1, fn = 2 * nu, bn = 2 * nu + 1;
            int xpm = fine_nbr(g, i, fm), xpn = fine_nbr(g, i, fn);
            int xmm = fine_nbr(g, i, bm), xmn = fine_nbr(g, i, bn);
            int xmmpn = fine_nbr(g, xmm, fn);   // x - mu + nu
            int xmmmn = fine_nbr(g, xmm, bn);   // x - mu - nu
            int xmnpm = fine_nbr(g, xmn, fm);   // x - nu + mu
            M3 l1 = mul3(mul3(ld3(U, g.V, mu, i), ld3(U, g.V, nu, xpm)), mul3(dag3(ld3(U, g.V, mu, xpn)), dag3(ld3(U, g.V, nu, i))));
            M3 l2 = mul3(mul3(ld3(U, g.V, nu, i), dag3(ld3(U, g.V, mu, xmmpn))), mul3(dag3(ld3(U, g.V, nu, xmm)), ld3(U, g.V, mu, xmm)));
            M3 l3 = mul3(mul3(dag3(ld3(U, g.V, mu, xmm)), dag3(ld3(U, g.V, nu, xmmmn))), mul3(ld3(U, g.V, mu, xmmmn), ld3(U, g.V, nu, xmn)));
            M3 l4 = mul3(mul3(dag3(ld3(U, g.V, nu, xmn)), ld3(U, g.V, mu, xmn)), mul3(ld3(U, g.V, nu, xmnpm), dag3(ld3(U, g.V, mu, i))));
            cplx<double> F[9];
            for (int q = 0; q < 9; ++q) F[q] = l1.m[q] + l2.m[q] + l3.m[q] + l4.m[q];
            cplx<double> Fd[9];
            for (int a = 0; a < 3; ++a)
                for (int b2 = 0; b2 < 3; ++b2) Fd[a * 3 + b2] = F[a * 3 + b2] - conj(F[b2 * 3 + a]);
            for (int h = 0; h < 2; ++h)
                for (int s = 0; s < 2; ++s)
                    for (int t2 = 0; t2 < 2; ++t2) {
                        cplx<double> gst = mk(c_gg[plane][h][s][t2][0], c_gg[plane][h][s][t2][1]);
                        if (gst.re == 0.0 && gst.im == 0.0) continue;
                        for (int a = 0; a < 3; ++a)
                            for (int b2 = 0; b2 < 3; ++b2) {
                                cplx<double> v = gst * Fd[a * 3 + b2];
                                A[h][s * 3 + a][t2 * 3 + b2] = A[h][s * 3 + a][t2 * 3 + b2] - (csw / 16.0) * v;
                            }
                    }
        }
    }
    for (int h = 0; h < 2; ++h) {
        // pack A
        for (int a = 0; a < 6; ++a) clov[(size_t)(h * 36 + a) * g.V + i] = A[h][a][a].re;
        int q = 0;
        for (int a = 0; a < 6; ++a)
            for (int b2 = a + 1; b2 < 6; ++b2, ++q) {
                clov[(size_t)(h * 36 + 6 + 2 * q) * g.V + i] = A[h][a][b2].re;
                clov[(size_t)(h * 36 + 7 + 2 * q) * g.V + i] = A[h][a][b2].im;
            }
        // Gauss-Jordan inverse with partial pivoting
        cplx<double> M[6][6], Inv[6][6];
        for (int a = 0; a < 6; ++a)
            for (int b2 = 0; b2 < 6; ++b2) {
                M[a][b2] = A[h][a][b2];
                Inv[a][b2] = mk(a == b2 ? 1.0 : 0.0, 0.0);
            }
        for (int c = 0; c < 6; ++c) {
            int piv = c;
            double best = norm2(M[c][c]);
            for (int rr = c + 1; rr < 6; ++rr)
                if (norm2(M[rr][c]) > best) {
                    best = norm2(M[rr][c]);
                    piv = rr;
                }
            if (piv != c)
                for (int k = 0; k < 6; ++k) {
                    cplx<double> t = M[c][k];
                    M[c][k] = M[piv][k];
                    M[piv][k] = t;
                    t = Inv[c][k];
                    Inv[c][k] = Inv[piv][k];
                    Inv[piv][k] = t;
                }
            double dn = norm2(M[c][c]);
            cplx<double> invp = mk(M[c][c].re / dn, -M[c][c].im / dn);
            for (int k = 0; k < 6; ++k) {
                M[c][k] = M[c][k] * invp;
                Inv[c][k] = Inv[c][k] * invp;
            }
            for (int rr = 0; rr < 6; ++rr) {
                if (rr == c) continue;
                cplx<double> f = M[rr][c];
                for (int k = 0; k < 6; ++k) {
                    M[rr][k] = M[rr][k] - f * M[c][k];
                    Inv[rr][k] = Inv[rr][k] - f * Inv[c][k];
                }
            }
        }
        for (int a = 0; a < 6; ++a) clovinv[(size_t)(h * 36 + a) * g.V + i] = Inv[a][a].re;
        q = 0;
        for (int a = 0; a < 6; ++a)
            for (int b2 = a + 1; b2 < 6; ++b2, ++q) {
                clovinv[(size_t)(h * 36 + 6 + 2 * q) * g.V + i] = Inv[a][b2].re;
                clovinv[(size_t)(h * 36 + 7 + 2 * q) * g.V + i] = Inv[a][b2].im;
            }
    }
}

int upload_gamma_products(const double* gg) {
    DD_CUDA(cudaMemcpyToSymbol(c_gg, gg, sizeof(double) * 6 * 2 * 2 * 2 * 2));
    return 0;
}

int launch_clover(const Geom& g, const cplx<double>* U, double m0, double csw, double* clov, double* clovinv, cudaStream_t st) {
    clover_kernel<<<ceil_div(g.V, 64), 64, 0, st>>>(g, U, m0, csw, clov, clovinv);
    DD_CHECK_LAUNCH();
    return 0;
}


// ---------------------------------------------------------------------------
// D z for an FP32 field z with an FP64-accurate result, evaluated in double-word
// FP32 arithmetic (pairs hi + lo of floats; error-free transformations TwoSum
// (Knuth) and TwoProduct via FMA, as in Joldes, Muller, Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic",
// ACM TOMS 2017).  Used for w = D z_k inside FGMRES, where z_k is the V-cycle
// output and hence exactly an FP32 vector.  On GB300 an FP64 instruction costs
// about sixty FP32 instructions, and the double-word form needs about twelve per
// real multiply-add, with relative accuracy ~1e-14.
// Links and site terms are stored as double-word pairs (same bytes as FP64).
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ cdw ld_cdw(const float4* p) {
    float4 v = __ldg(p);
    return {{v.x, v.y}, {v.z, v.w}};
}

__device__ __forceinline__ cdw cdw_ipow_rt(const cdw& a, int p) {
    cdw b = (p & 1) ? cdw{dw_neg(a.im), a.re} : a;
    return (p & 2) ? cdw{dw_neg(b.re), dw_neg(b.im)} : b;
}

// one hop of D (direction mu, orientation fwd, given at run time) in double-word arithmetic
__device__ __noinline__ void dw_hop_rt(cdw (&acc)[12], const cplx<float>* __restrict__ in, int V, int nb, const float4* __restrict__ U,
                                       int link_site, int mu, bool fwd) {
    const int c0 = c_spinb[mu][0], p0 = c_spinb[mu][1], c1 = c_spinb[mu][2], p1 = c_spinb[mu][3];
    const int hc0 = c_spinb[mu][4], hp0 = c_spinb[mu][5], hc1 = c_spinb[mu][6], hp1 = c_spinb[mu][7];
    cdw h[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cplx<float> u0 = in[(size_t)(0 * 3 + c) * V + nb], u1 = in[(size_t)(1 * 3 + c) * V + nb];
        cplx<float> l2 = in[(size_t)(2 * 3 + c) * V + nb], l3 = in[(size_t)(3 * 3 + c) * V + nb];
        cdw b0 = cdw_ipow_rt(c0 ? cdw{{l3.re, 0.f}, {l3.im, 0.f}} : cdw{{l2.re, 0.f}, {l2.im, 0.f}}, p0);
        cdw b1 = cdw_ipow_rt(c1 ? cdw{{l3.re, 0.f}, {l3.im, 0.f}} : cdw{{l2.re, 0.f}, {l2.im, 0.f}}, p1);
        cdw a0 = {{u0.re, 0.f}, {u0.im, 0.f}}, a1 = {{u1.re, 0.f}, {u1.im, 0.f}};
        h[0][c] = fwd ? cdw_sub(a0, b0) : cdw_add(a0, b0);
        h[1][c] = fwd ? cdw_sub(a1, b1) : cdw_add(a1, b1);
    }
    cdw W[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) W[q] = ld_cdw(U + (size_t)(mu * 9 + q) * V + link_site);
    cdw gv[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cdw t = cdw_zero();
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (fwd) cdw_mac(t, W[a * 3 + b], h[s][b]);
                else cdw_mac_conj(t, W[b * 3 + a], h[s][b]);
            }
            t.re = dw_norm(t.re);
            t.im = dw_norm(t.im);
            gv[s][a] = t;
            acc[s * 3 + a] = cdw_add(acc[s * 3 + a], t);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cdw l0 = cdw_ipow_rt(hc0 ? gv[1][c] : gv[0][c], hp0);
        cdw l1 = cdw_ipow_rt(hc1 ? gv[1][c] : gv[0][c], hp1);
        acc[2 * 3 + c] = fwd ? cdw_sub(acc[2 * 3 + c], l0) : cdw_add(acc[2 * 3 + c], l0);
        acc[3 * 3 + c] = fwd ? cdw_sub(acc[3 * 3 + c], l1) : cdw_add(acc[3 * 3 + c], l1);
    }
}

}  // namespace

// thread (x, y): site blockIdx.x * 32 + x, right-hand side blockIdx.y * blockDim.y + y (the warps of
// a CTA share the double-word links and site terms of 32 sites through L1)
template <bool OUT_DW>
__global__ void __launch_bounds__(128) dslash_dw_kernel(Geom g, const float4* __restrict__ U, const float2* __restrict__ clov,
                                                        const cplx<float>* __restrict__ in, void* __restrict__ outp, int nrhs) {
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    const int i = blockIdx.x * 32 + threadIdx.x;
    if (i >= g.V || r >= nrhs) return;
    const size_t off = (size_t)r * 12 * g.V;
    const cplx<float>* inr = in + off;
    cdw acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = cdw_zero();
#pragma unroll 1
    for (int d = 0; d < 8; ++d) {
        const int nb = fine_nbr(g, i, d);
        const bool fwd = (d & 1) == 0;
        dw_hop_rt(acc, inr, g.V, nb, U, fwd ? i : nb, d >> 1, fwd);
    }
    // site term: y = A x with two packed hermitian 6x6 blocks (double-word entries), x FP32
    cdw y[12];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float x[12];
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            cplx<float> v = inr[(size_t)(h * 6 + a) * g.V + i];
            x[2 * a] = v.re;
            x[2 * a + 1] = v.im;
        }
        const float2* base = clov + (size_t)(h * 36) * g.V + i;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            float2 dv = __ldg(base + (size_t)a * g.V);
            dw d = {dv.x, dv.y};
            cdw t = cdw_zero();
            dw_macf(t.re, d, x[2 * a]);
            dw_macf(t.im, d, x[2 * a + 1]);
            y[h * 6 + a] = t;
        }
        int q = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
#pragma unroll
            for (int b = a + 1; b < 6; ++b) {
                float2 mr = __ldg(base + (size_t)(6 + 2 * q) * g.V), mi = __ldg(base + (size_t)(7 + 2 * q) * g.V);
                dw m_re = {mr.x, mr.y}, m_im = {mi.x, mi.y};
                // y[a] += m x[b];  y[b] += conj(m) x[a]
                dw_macf(y[h * 6 + a].re, m_re, x[2 * b]);
                dw_macf(y[h * 6 + a].re, dw_neg(m_im), x[2 * b + 1]);
                dw_macf(y[h * 6 + a].im, m_re, x[2 * b + 1]);
                dw_macf(y[h * 6 + a].im, m_im, x[2 * b]);
                dw_macf(y[h * 6 + b].re, m_re, x[2 * a]);
                dw_macf(y[h * 6 + b].re, m_im, x[2 * a + 1]);
                dw_macf(y[h * 6 + b].im, m_re, x[2 * a + 1]);
                dw_macf(y[h * 6 + b].im, dw_neg(m_im), x[2 * a]);
                ++q;
            }
        }
    }
    if (OUT_DW) {
        float4* o = reinterpret_cast<float4*>(outp) + off;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            dw re = dw_norm(dw_add(y[k].re, {-0.5f * acc[k].re.h, -0.5f * acc[k].re.l}));
            dw im = dw_norm(dw_add(y[k].im, {-0.5f * acc[k].im.h, -0.5f * acc[k].im.l}));
            o[(size_t)k * g.V + i] = make_float4(re.h, re.l, im.h, im.l);
        }
    } else {
        cplx<double>* o = reinterpret_cast<cplx<double>*>(outp) + off;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double re = (double)y[k].re.h + (double)y[k].re.l - 0.5 * ((double)acc[k].re.h + (double)acc[k].re.l);
            double im = (double)y[k].im.h + (double)y[k].im.l - 0.5 * ((double)acc[k].im.h + (double)acc[k].im.l);
            o[(size_t)k * g.V + i] = mk(re, im);
        }
    }
}

int launch_dslash_dw(const Geom& g, const float4* U, const float2* clov, const cplx<float>* in, void* out, bool out_dw, int nrhs,
                     cudaStream_t st) {
    const int ry = std::min(nrhs, 4);
    const dim3 grid((unsigned)ceil_div(g.V, 32), (unsigned)ceil_div(nrhs, ry)), block(32, ry);
    if (out_dw) dslash_dw_kernel<true><<<grid, block, 0, st>>>(g, U, clov, in, out, nrhs);
    else dslash_dw_kernel<false><<<grid, block, 0, st>>>(g, U, clov, in, out, nrhs);
    DD_CHECK_LAUNCH();
    return 0;
}

// FP64 array -> double-word pairs (hi = nearest float, lo = nearest float of the remainder)
__global__ void to_dw_kernel(const double* __restrict__ in, float2* __restrict__ out, size_t n) {
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        double x = in[q];
        float h = (float)x;
        out[q] = make_float2(h, (float)(x - (double)h));
    }
}
int launch_to_dw(const double* in, float2* out, size_t n, cudaStream_t st) {
    int blocks = ceil_div((long long)n, 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    to_dw_kernel<<<blocks, 256, 0, st>>>(in, out, n);
    DD_CHECK_LAUNCH();
    return 0;
}

}  // namespace ddamg
