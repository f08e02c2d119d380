// Level-1 operations of the recursion to a third level (Sec. 3 applied to the coarse system;
// Sec. 6.4): red-black SAP over blocks of level-1 sites with odd-even MR block solves (Sec. 2.3 and
// Sec. 6 on D_1 = P^H D P), Gamma5-compatible aggregation of level-1 test vectors with ordered
// local orthonormalisation (Sec. 3.1-3.2), restriction, prolongation and the Galerkin operator
// D_2 = P_1^H D_1 P_1 as a nine-block stencil.
//
// Every operation is a functor computing one output element per index, __host__ __device__, and
// the orchestration is written once against an executor: on the GPU the executor launches a
// grid-stride kernel over the index range, on the host it is a plain loop.  Reductions (the MR
// step sizes, the Gram-Schmidt of one aggregate) are one index per block or aggregate with a
// serial inner loop.
//
// Layouts (internal orders of ml_geom.h):
//   level-1 field   cplx[nrhs][NB][nc]
//   D_1 blocks      B1[NB][9][nc (column)][nc (row)], direction 0 = self, 1 + 2 mu + backward
//   even inverses   Dinv1[NB/2][nc][nc] (inverse of the self block of the even sites, which come first)
//   P_1             P1[NB2][2][Vb1 * nc/2][N1]: aggregate (block, half h), row k = local * nc/2 + a
//                   for component h * nc/2 + a of the block's local site, column j = test vector
//   level-2 vector  cplx[nrhs][NB2][2 N1], component h * N1 + j
//   D_2 blocks      B2[NB2][9][2 N1][2 N1], the layout of B1
#pragma once

#include "common.cuh"

namespace ddamg {

template <typename T>
struct MLView {
    int NB, nc, half;  // level-1 sites, components per site, nc / 2
    int NB2, Vb1, Vb1e, N1;
    const int* nbr1;           // [8][NB]
    const int* sites;          // [NB2][Vb1]
    const int* blk_of;         // [NB]
    const int* loc_of;         // [NB]
    const unsigned char* same;  // [8][NB]
    const cplx<T>* B1;
    const cplx<T>* Dinv1;
    const cplx<T>* P1;
    // half-precision handles: FP16 copies of B1 and Dinv1 (one __half2 (re, im) per entry, same
    // order), read by the fused SAP colour step only; null otherwise
    const void* B1h = nullptr;
    const void* Dinv1h = nullptr;
};

template <typename T>
__host__ __device__ inline T ml_den_floor();
template <>
__host__ __device__ inline double ml_den_floor<double>() { return 1e-280; }
template <>
__host__ __device__ inline float ml_den_floor<float>() { return 1e-36f; }

// row `row` of a column-major nc x nc block times the vector xv[0..nc)
template <typename T>
__host__ __device__ inline cplx<T> ml_rowdot(const cplx<T>* blk, int nc, int row, const cplx<T>* xv) {
    cplx<T> acc = czero<T>();
    for (int col = 0; col < nc; ++col) cmac(acc, blk[(size_t)col * nc + row], xv[col]);
    return acc;
}

template <typename T>
__host__ __device__ inline const cplx<T>* ml_block(const MLView<T>& v, int c, int d) {
    return v.B1 + ((size_t)c * 9 + d) * v.nc * v.nc;
}

// site selection: all sites, or the even / odd sites of the blocks of one colour
enum { ML_ALL = 0, ML_EVEN = 1, ML_ODD = 2 };
template <typename T>
__host__ __device__ inline bool ml_selected(const MLView<T>& v, int c, int parity_sel, int colour) {
    if (colour >= 0 && (v.blk_of[c] < v.NB2 / 2 ? 0 : 1) != colour) return false;
    if (parity_sel == ML_EVEN) return c < v.NB / 2;
    if (parity_sel == ML_ODD) return c >= v.NB / 2;
    return true;
}

// right-hand sides are processed in chunks of ML_RC per thread, so that each matrix entry is read
// once per chunk (the operator, not the vectors, dominates the traffic)
constexpr int ML_RC = 12;  // the twelve point sources of a batch in one pass

// acc[k] += row `row` of the column-major block times the site vector of right-hand side r0 + k
template <typename T>
__host__ __device__ inline void ml_rowdot_rhs(cplx<T> (&acc)[ML_RC], const cplx<T>* blk, int nc, int row, const cplx<T>* x0, size_t fs,
                                              int nk) {
    for (int col = 0; col < nc; ++col) {
        const cplx<T> b = blk[(size_t)col * nc + row];
        for (int k = 0; k < nk; ++k) cmac(acc[k], b, x0[(size_t)k * fs + col]);
    }
}

// y = b - D_1 x (b may be null: y = D_1 x), every site; one index per (site, row)
template <typename T>
struct MLFullApply {
    MLView<T> v;
    const cplx<T>* x;
    const cplx<T>* b;
    cplx<T>* y;
    int nrhs;
    __host__ __device__ void operator()(long long i) const {
        const size_t fs = (size_t)v.NB * v.nc;
        const int c = (int)(i / v.nc), row = (int)(i % v.nc);
        for (int r0 = 0; r0 < nrhs; r0 += ML_RC) {
            const int nk = nrhs - r0 < ML_RC ? nrhs - r0 : ML_RC;
            cplx<T> acc[ML_RC];
            for (int k = 0; k < ML_RC; ++k) acc[k] = czero<T>();
            const cplx<T>* xr = x + (size_t)r0 * fs;
            ml_rowdot_rhs(acc, ml_block(v, c, 0), v.nc, row, xr + (size_t)c * v.nc, fs, nk);
            for (int d = 0; d < 8; ++d) {
                const int n = v.nbr1[(size_t)d * v.NB + c];
                ml_rowdot_rhs(acc, ml_block(v, c, 1 + d), v.nc, row, xr + (size_t)n * v.nc, fs, nk);
            }
            for (int k = 0; k < nk; ++k) {
                const size_t o = (size_t)(r0 + k) * fs + i;
                y[o] = b ? b[o] - acc[k] : acc[k];
            }
        }
    }
};

// on the selected sites: dst = add + B_self self_src + sign * (in-block hops of hop_src);
// elsewhere dst = 0 (zero_others) or unchanged.  Any of add, self_src, hop_src may be null.
// One index per (site, row).
template <typename T>
struct MLHopsCombine {
    MLView<T> v;
    cplx<T>* dst;
    const cplx<T>* add;
    const cplx<T>* self_src;
    const cplx<T>* hop_src;
    T sign;
    int parity_sel, colour;
    bool zero_others;
    int nrhs;
    __host__ __device__ void operator()(long long i) const {
        const size_t fs = (size_t)v.NB * v.nc;
        const int c = (int)(i / v.nc), row = (int)(i % v.nc);
        if (!ml_selected(v, c, parity_sel, colour)) {
            if (zero_others)
                for (int r = 0; r < nrhs; ++r) dst[(size_t)r * fs + i] = czero<T>();
            return;
        }
        for (int r0 = 0; r0 < nrhs; r0 += ML_RC) {
            const int nk = nrhs - r0 < ML_RC ? nrhs - r0 : ML_RC;
            cplx<T> sacc[ML_RC], hacc[ML_RC];
            for (int k = 0; k < ML_RC; ++k) sacc[k] = hacc[k] = czero<T>();
            if (self_src) ml_rowdot_rhs(sacc, ml_block(v, c, 0), v.nc, row, self_src + (size_t)r0 * fs + (size_t)c * v.nc, fs, nk);
            if (hop_src)
                for (int d = 0; d < 8; ++d) {
                    if (!v.same[(size_t)d * v.NB + c]) continue;
                    const int n = v.nbr1[(size_t)d * v.NB + c];
                    ml_rowdot_rhs(hacc, ml_block(v, c, 1 + d), v.nc, row, hop_src + (size_t)r0 * fs + (size_t)n * v.nc, fs, nk);
                }
            for (int k = 0; k < nk; ++k) {
                const size_t o = (size_t)(r0 + k) * fs + i;
                cplx<T> acc = add ? add[o] : czero<T>();
                acc = acc + sacc[k];
                dst[o] = acc + sign * hacc[k];
            }
        }
    }
};

// on the selected even sites: dst = Dinv_1 src; elsewhere 0 (zero_others) or unchanged.
// One index per (site, row).
template <typename T>
struct MLDinvApply {
    MLView<T> v;
    const cplx<T>* src;
    cplx<T>* dst;
    int colour;
    bool zero_others;
    int nrhs;
    __host__ __device__ void operator()(long long i) const {
        const size_t fs = (size_t)v.NB * v.nc;
        const int c = (int)(i / v.nc), row = (int)(i % v.nc);
        if (!ml_selected(v, c, ML_EVEN, colour)) {
            if (zero_others)
                for (int r = 0; r < nrhs; ++r) dst[(size_t)r * fs + i] = czero<T>();
            return;
        }
        for (int r0 = 0; r0 < nrhs; r0 += ML_RC) {
            const int nk = nrhs - r0 < ML_RC ? nrhs - r0 : ML_RC;
            cplx<T> acc[ML_RC];
            for (int k = 0; k < ML_RC; ++k) acc[k] = czero<T>();
            ml_rowdot_rhs(acc, v.Dinv1 + (size_t)c * v.nc * v.nc, v.nc, row, src + (size_t)r0 * fs + (size_t)c * v.nc, fs, nk);
            for (int k = 0; k < nk; ++k) dst[(size_t)(r0 + k) * fs + i] = acc[k];
        }
    }
};

// MR step size of every (right-hand side, block) of one colour over the block's odd sites:
// alpha = <s, rho> / <s, s> with <a, b> = a^H b; 0 where <s, s> vanishes
template <typename T>
struct MLBlockAlpha {
    MLView<T> v;
    const cplx<T>* s;
    const cplx<T>* rho;
    cplx<T>* alpha;  // [nrhs][NB2]
    int colour;
    __host__ __device__ void operator()(long long i) const {
        const int r = (int)(i / v.NB2), c2 = (int)(i % v.NB2);
        if ((c2 < v.NB2 / 2 ? 0 : 1) != colour) {
            alpha[i] = czero<T>();
            return;
        }
        const size_t fs = (size_t)v.NB * v.nc;
        cplx<T> num = czero<T>();
        T den = T(0);
        for (int l = v.Vb1e; l < v.Vb1; ++l) {
            const size_t base = r * fs + (size_t)v.sites[(size_t)c2 * v.Vb1 + l] * v.nc;
            for (int a = 0; a < v.nc; ++a) {
                cmac_conj(num, s[base + a], rho[base + a]);
                den += norm2(s[base + a]);
            }
        }
        alpha[i] = den > ml_den_floor<T>() ? mk(num.re / den, num.im / den) : czero<T>();
    }
};

// x += alpha rho, rho -= alpha s on the odd sites of the blocks of one colour
template <typename T>
struct MLMRUpdate {
    MLView<T> v;
    const cplx<T>* alpha;
    const cplx<T>* s;
    cplx<T>* rho;
    cplx<T>* x;
    int colour;
    __host__ __device__ void operator()(long long i) const {
        const size_t fs = (size_t)v.NB * v.nc;
        const int r = (int)(i / fs), c = (int)((i / v.nc) % v.NB);
        if (!ml_selected(v, c, ML_ODD, colour)) return;
        const cplx<T> a = alpha[(size_t)r * v.NB2 + v.blk_of[c]];
        cmac(x[i], a, rho[i]);
        rho[i] = rho[i] - a * s[i];
    }
};

// z += x on the sites of the blocks of one colour
template <typename T>
struct MLAddColour {
    MLView<T> v;
    const cplx<T>* x;
    cplx<T>* z;
    int colour;
    __host__ __device__ void operator()(long long i) const {
        const int c = (int)((i / v.nc) % v.NB);
        if (ml_selected(v, c, ML_ALL, colour)) z[i] = z[i] + x[i];
    }
};

template <typename T>
struct MLZero {
    cplx<T>* p;
    __host__ __device__ void operator()(long long i) const { p[i] = czero<T>(); }
};

// ordered modified Gram-Schmidt of the test vectors vec[N1][NB][nc] on aggregate (block c2,
// half h) into P1; fail = 1 where a vector's remainder drops below 1e-12 of its own norm there
template <typename T>
struct MLGramSchmidt {
    MLView<T> v;
    const cplx<T>* vec;
    cplx<T>* P;
    int* fail;
    __host__ __device__ void operator()(long long i) const {
        const int c2 = (int)(i / 2), h = (int)(i % 2);
        const int K = v.Vb1 * v.half, N1 = v.N1;
        cplx<T>* Q = P + ((size_t)c2 * 2 + h) * K * N1;
        for (int j = 0; j < N1; ++j) {
            T ref = T(0);
            for (int k = 0; k < K; ++k) {
                const int site = v.sites[(size_t)c2 * v.Vb1 + k / v.half];
                const cplx<T> e = vec[((size_t)j * v.NB + site) * v.nc + h * v.half + k % v.half];
                Q[(size_t)k * N1 + j] = e;
                ref += norm2(e);
            }
            for (int p = 0; p < j; ++p) {
                cplx<T> hij = czero<T>();
                for (int k = 0; k < K; ++k) cmac_conj(hij, Q[(size_t)k * N1 + p], Q[(size_t)k * N1 + j]);
                for (int k = 0; k < K; ++k) Q[(size_t)k * N1 + j] = Q[(size_t)k * N1 + j] - hij * Q[(size_t)k * N1 + p];
            }
            T nrm = T(0);
            for (int k = 0; k < K; ++k) nrm += norm2(Q[(size_t)k * N1 + j]);
            nrm = sqrt(nrm);
            if (!(nrm > T(1e-12) * sqrt(ref))) {
                *fail = 1;
                nrm = T(1);
            }
            const T inv = T(1) / nrm;
            for (int k = 0; k < K; ++k) Q[(size_t)k * N1 + j] = inv * Q[(size_t)k * N1 + j];
        }
    }
};

// e = P_1^H x: e[r][c2][h N1 + j] = sum_k conj(P1[c2][h][k][j]) x[r][site(c2, k)][component(h, k)]
template <typename T>
struct MLRestrict {
    MLView<T> v;
    const cplx<T>* x;
    cplx<T>* e;
    __host__ __device__ void operator()(long long i) const {
        const int nc2 = 2 * v.N1;
        const int r = (int)(i / ((size_t)v.NB2 * nc2)), c2 = (int)((i / nc2) % v.NB2), q = (int)(i % nc2);
        const int h = q / v.N1, j = q % v.N1, K = v.Vb1 * v.half;
        const cplx<T>* Q = v.P1 + ((size_t)c2 * 2 + h) * K * v.N1;
        const cplx<T>* xr = x + (size_t)r * v.NB * v.nc;
        cplx<T> acc = czero<T>();
        for (int k = 0; k < K; ++k) {
            const int site = v.sites[(size_t)c2 * v.Vb1 + k / v.half];
            cmac_conj(acc, Q[(size_t)k * v.N1 + j], xr[(size_t)site * v.nc + h * v.half + k % v.half]);
        }
        e[i] = acc;
    }
};

// y = P_1 e (every level-1 element)
template <typename T>
struct MLProlong {
    MLView<T> v;
    const cplx<T>* e;
    cplx<T>* y;
    __host__ __device__ void operator()(long long i) const {
        const size_t fs = (size_t)v.NB * v.nc;
        const int r = (int)(i / fs), c = (int)((i / v.nc) % v.NB), a = (int)(i % v.nc);
        const int c2 = v.blk_of[c], h = a / v.half, k = v.loc_of[c] * v.half + a % v.half, K = v.Vb1 * v.half;
        const cplx<T>* Q = v.P1 + (((size_t)c2 * 2 + h) * K + k) * v.N1;
        const cplx<T>* er = e + ((size_t)r * v.NB2 + c2) * 2 * v.N1 + h * v.N1;
        cplx<T> acc = czero<T>();
        for (int j = 0; j < v.N1; ++j) cmac(acc, Q[j], er[j]);
        y[i] = acc;
    }
};

// the couplings in direction `dir` that leave the block: dst = B_{1+dir} x[nbr] where the
// neighbour lies in another block, 0 elsewhere.  One index per (site, row).
template <typename T>
struct MLCrossHop {
    MLView<T> v;
    const cplx<T>* x;
    cplx<T>* dst;
    int dir;
    int nrhs;
    __host__ __device__ void operator()(long long i) const {
        const size_t fs = (size_t)v.NB * v.nc;
        const int c = (int)(i / v.nc), row = (int)(i % v.nc);
        if (v.same[(size_t)dir * v.NB + c]) {
            for (int r = 0; r < nrhs; ++r) dst[(size_t)r * fs + i] = czero<T>();
            return;
        }
        const int n = v.nbr1[(size_t)dir * v.NB + c];
        for (int r0 = 0; r0 < nrhs; r0 += ML_RC) {
            const int nk = nrhs - r0 < ML_RC ? nrhs - r0 : ML_RC;
            cplx<T> acc[ML_RC];
            for (int k = 0; k < ML_RC; ++k) acc[k] = czero<T>();
            ml_rowdot_rhs(acc, ml_block(v, c, 1 + dir), v.nc, row, x + (size_t)r0 * fs + (size_t)n * v.nc, fs, nk);
            for (int k = 0; k < nk; ++k) dst[(size_t)(r0 + k) * fs + i] = acc[k];
        }
    }
};

// unit coarse vectors: E[col][c2][q] = (q == col), one right-hand side per column
template <typename T>
struct MLUnitColumns {
    int NB2, nc2;
    cplx<T>* E;
    __host__ __device__ void operator()(long long i) const {
        const int col = (int)(i / ((size_t)NB2 * nc2)), q = (int)(i % nc2);
        E[i] = q == col ? mk(T(1), T(0)) : czero<T>();
    }
};

// B2[c2][d][col][row] = e[col][c2][row]
template <typename T>
struct MLScatterB2 {
    int NB2, nc2, d;
    const cplx<T>* e;
    cplx<T>* B2;
    __host__ __device__ void operator()(long long i) const {
        const int col = (int)(i / ((size_t)NB2 * nc2)), c2 = (int)((i / nc2) % NB2), row = (int)(i % nc2);
        B2[(((size_t)c2 * 9 + d) * nc2 + col) * nc2 + row] = e[i];
    }
};

// squared norm of each of the fields x[i] of length fs (one index per field)
template <typename T>
struct MLNorm2 {
    const cplx<T>* x;
    size_t fs;
    T* out;
    __host__ __device__ void operator()(long long i) const {
        T acc = T(0);
        for (size_t k = 0; k < fs; ++k) acc += norm2(x[(size_t)i * fs + k]);
        out[i] = acc;
    }
};

// x[r] /= sqrt(n2[r]) for every field r of length fs
template <typename T>
struct MLNormalize {
    cplx<T>* x;
    size_t fs;
    const T* n2;
    __host__ __device__ void operator()(long long i) const {
        const T s = T(1) / sqrt(n2[(size_t)i / fs]);
        x[i] = s * x[i];
    }
};

// y = a + b (b may alias y)
template <typename T>
struct MLAdd {
    const cplx<T>* a;
    const cplx<T>* b;
    cplx<T>* y;
    __host__ __device__ void operator()(long long i) const { y[i] = a[i] + b[i]; }
};

template <typename T>
struct MLCopy {
    const cplx<T>* a;
    cplx<T>* y;
    __host__ __device__ void operator()(long long i) const { y[i] = a[i]; }
};

// ---------------------------------------------------------------------------
// executors
// ---------------------------------------------------------------------------
struct MLHostExec {
    template <class F>
    int run(long long n, const F& f) const {
        for (long long i = 0; i < n; ++i) f(i);
        return 0;
    }
    // no fused colour step on the host: ml_sap runs the functor sequence
    template <typename T>
    int sap_colour(const MLView<T>&, const cplx<T>*, cplx<T>*, int, int, int) const {
        return 1;
    }
};

// one SAP colour step of ml_sap as a single kernel (ml_sap.cu): FP32, blocks with as many even as
// odd sites, at most 384 (block-half sites x components) threads and the six half-block MR vectors
// of 12 right-hand sides within shared memory
bool ml_sap_fused_supported(const MLView<float>& v);
int launch_ml_sap_fused(const MLView<float>& v, const cplx<float>* b, cplx<float>* z, int nrhs, int colour, int mr_steps,
                        cudaStream_t st);

// ---------------------------------------------------------------------------
// orchestration
// ---------------------------------------------------------------------------
template <typename T>
struct MLSapWork {
    cplx<T> *r, *te, *rho, *u, *w, *s, *x;  // level-1 fields of nrhs right-hand sides
    cplx<T>* alpha;                          // [nrhs][NB2]
};

// nu red-black SAP iterations on D_1 z = b, updating z in place (Sec. 2.3): per colour,
// r = b - D_1 z; on the blocks of that colour the odd-site Schur complement
// S = A_oo - A_oe A_ee^{-1} A_eo is solved by mr_steps MR steps from zero, the even sites are
// back-substituted, and z += the block solution.
template <class X, typename T>
int ml_sap(const X& ex, const MLView<T>& v, const cplx<T>* b, cplx<T>* z, int nrhs, int nu, int mr_steps, const MLSapWork<T>& w) {
    const long long nf = (long long)nrhs * v.NB * v.nc, ns = (long long)v.NB * v.nc;
    for (int it = 0; it < nu; ++it)
        for (int col = 0; col < 2; ++col) {
            int rc = ex.sap_colour(v, b, z, nrhs, col, mr_steps);  // 0: done by the executor's fused step
            if (rc < 0) return rc;
            if (rc == 0) continue;
            if ((rc = ex.run(ns, MLFullApply<T>{v, z, b, w.r, nrhs}))) return rc;
            // t_e = A_ee^{-1} r_e; rho = r_o - A_oe t_e; x = 0
            if ((rc = ex.run(ns, MLDinvApply<T>{v, w.r, w.te, col, true, nrhs}))) return rc;
            if ((rc = ex.run(ns, MLHopsCombine<T>{v, w.rho, w.r, nullptr, w.te, T(-1), ML_ODD, col, true, nrhs}))) return rc;
            if ((rc = ex.run(nf, MLZero<T>{w.x}))) return rc;
            for (int k = 0; k < mr_steps; ++k) {
                // s = S rho = A_oo rho - A_oe A_ee^{-1} A_eo rho
                if ((rc = ex.run(ns, MLHopsCombine<T>{v, w.u, nullptr, nullptr, w.rho, T(1), ML_EVEN, col, true, nrhs}))) return rc;
                if ((rc = ex.run(ns, MLDinvApply<T>{v, w.u, w.w, col, true, nrhs}))) return rc;
                if ((rc = ex.run(ns, MLHopsCombine<T>{v, w.s, nullptr, w.rho, w.w, T(-1), ML_ODD, col, true, nrhs}))) return rc;
                if ((rc = ex.run((long long)nrhs * v.NB2, MLBlockAlpha<T>{v, w.s, w.rho, w.alpha, col}))) return rc;
                if ((rc = ex.run(nf, MLMRUpdate<T>{v, w.alpha, w.s, w.rho, w.x, col}))) return rc;
            }
            // x_e = A_ee^{-1} (r_e - A_eo x_o); z += x on the blocks of this colour
            if ((rc = ex.run(ns, MLHopsCombine<T>{v, w.u, w.r, nullptr, w.x, T(-1), ML_EVEN, col, true, nrhs}))) return rc;
            if ((rc = ex.run(ns, MLDinvApply<T>{v, w.u, w.x, col, false, nrhs}))) return rc;
            if ((rc = ex.run(nf, MLAddColour<T>{v, w.x, z, col}))) return rc;
        }
    return 0;
}

// level-1 V-cycle (Sec. 4.2 on D_1): x = P_1 D_2^{-1} P_1^H r with the level-2 solve supplied by
// coarse(eb, ex, nrhs), then nu SAP iterations on D_1 x = r from that x (which adds
// M_SAP^(nu) (r - D_1 x), the SAP iteration being affine).  eb, ex: level-2 work vectors.
template <class X, typename T, class Coarse>
int ml_vcycle1_t(const X& ex, const MLView<T>& v, const cplx<T>* r, cplx<T>* x, int nrhs, int nu, int mr_steps, const MLSapWork<T>& w,
                 cplx<T>* eb, cplx<T>* exx, Coarse&& coarse) {
    int rc;
    if ((rc = ex.run((long long)nrhs * v.NB2 * 2 * v.N1, MLRestrict<T>{v, r, eb}))) return rc;
    if ((rc = coarse(eb, exx, nrhs))) return rc;
    if ((rc = ex.run((long long)nrhs * v.NB * v.nc, MLProlong<T>{v, exx, x}))) return rc;
    return ml_sap(ex, v, r, x, nrhs, nu, mr_steps, w);
}

// The setup of level 1 (Algorithm 1 phase 1, then n_inv rounds of Algorithm 2 -- or Algorithm 1's
// update when idsetup -- on D_1), all N_1 vectors as one batch: P_1 and D_2 are frozen within a
// round, so the updates are independent.  vec[N1][NB][nc] holds the initial vectors and returns
// the final ones; rebuild(vec) forms P_1, D_2 and its inverses from vec (it is called at the start
// of every round and once after the last); vcycle(r, x, nrhs) is the level-1 V-cycle; t, u are work
// fields of N1 level-1 vectors, n2 a work array of N1 reals.
template <class X, typename T, class Rebuild, class VCycle>
int ml_setup1_t(const X& ex, const MLView<T>& v, cplx<T>* vec, int n_inv, bool idsetup, int mr_steps, const MLSapWork<T>& w, cplx<T>* t,
                cplx<T>* u, T* n2, Rebuild&& rebuild, VCycle&& vcycle) {
    const int N1 = v.N1;
    const size_t fs = (size_t)v.NB * v.nc;
    const long long nf = (long long)N1 * fs;
    int rc;
    // phase 1: v_j <- M_SAP^(eta) v_j for eta = 1, 2, 3 (SAP from zero, v_j the right-hand side)
    for (int eta = 1; eta <= 3; ++eta) {
        if ((rc = ex.run(nf, MLZero<T>{t}))) return rc;
        if ((rc = ml_sap(ex, v, vec, t, N1, eta, mr_steps, w))) return rc;
        if ((rc = ex.run(nf, MLCopy<T>{t, vec}))) return rc;
    }
    for (int it = 0; it < n_inv; ++it) {
        if ((rc = rebuild(vec))) return rc;
        if (idsetup) {
            if ((rc = vcycle(vec, u, N1))) return rc;  // v <- C v
            if ((rc = ex.run(nf, MLCopy<T>{u, vec}))) return rc;
        } else {
            if ((rc = ex.run((long long)v.NB * v.nc, MLFullApply<T>{v, vec, vec, t, N1}))) return rc;  // t = v - D_1 v
            if ((rc = vcycle(t, u, N1))) return rc;                             // u = C t
            if ((rc = ex.run(nf, MLAdd<T>{vec, u, vec}))) return rc;           // v <- v + C (v - D_1 v)
        }
        if ((rc = ex.run(N1, MLNorm2<T>{vec, fs, n2}))) return rc;
        if ((rc = ex.run(nf, MLNormalize<T>{vec, fs, n2}))) return rc;
    }
    return rebuild(vec);
}

// D_2 = P_1^H D_1 P_1 (Sec. 3.2): the block of direction 0 collects the self blocks and the
// couplings inside each block, direction 1 + dir the couplings in dir that leave it.  E, W, Y are
// work arrays of 2 N1 level-2 vectors (E, e) and 2 N1 level-1 fields (W, Y).
template <class X, typename T>
int ml_galerkin(const X& ex, const MLView<T>& v, cplx<T>* B2, cplx<T>* E, cplx<T>* W, cplx<T>* Y, cplx<T>* e) {
    const int nc2 = 2 * v.N1;
    const long long n2 = (long long)nc2 * v.NB2 * nc2, n1 = (long long)nc2 * v.NB * v.nc, ns = (long long)v.NB * v.nc;
    int rc;
    if ((rc = ex.run(n2, MLUnitColumns<T>{v.NB2, nc2, E}))) return rc;
    if ((rc = ex.run(n1, MLProlong<T>{v, E, W}))) return rc;
    if ((rc = ex.run(ns, MLHopsCombine<T>{v, Y, nullptr, W, W, T(1), ML_ALL, -1, true, nc2}))) return rc;
    if ((rc = ex.run(n2, MLRestrict<T>{v, Y, e}))) return rc;
    if ((rc = ex.run(n2, MLScatterB2<T>{v.NB2, nc2, 0, e, B2}))) return rc;
    for (int dir = 0; dir < 8; ++dir) {
        if ((rc = ex.run(ns, MLCrossHop<T>{v, W, Y, dir, nc2}))) return rc;
        if ((rc = ex.run(n2, MLRestrict<T>{v, Y, e}))) return rc;
        if ((rc = ex.run(n2, MLScatterB2<T>{v.NB2, nc2, 1 + dir, e, B2}))) return rc;
    }
    return 0;
}

}  // namespace ddamg
