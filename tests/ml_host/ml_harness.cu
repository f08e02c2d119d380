// Test harness: runs the level-1 operations of the CUDA library (the functors and orchestration of
// ml_ops.cuh, the blocking of ml_geom.h) on the host through the loop executor, so that their index
// arithmetic and algebra can be compared with the oracle without a GPU.  Built by the tests as a
// host-only shared library; the product never loads it.  Arrays are complex128 as (re, im) pairs in
// the internal orders described in ml_ops.cuh; B1/Dinv1/B2 column-major.
#include <cstring>
#include <utility>
#include <vector>

#include "ml_geom.h"
#include "ml_ops.cuh"

using namespace ddamg;
using C = cplx<double>;

namespace {
struct HostLevel {
    MLHostGeom g;
    MLView<double> v{};
    int ok = -1;
    HostLevel(const int* L1, const int* b1, int nc, int N1, const double* B1, const double* Dinv1, const double* P1) {
        ok = ml_build_geom(L1, b1, g);
        if (ok) return;
        v.NB = g.NB;
        v.nc = nc;
        v.half = nc / 2;
        v.NB2 = g.NB2;
        v.Vb1 = g.Vb1;
        v.Vb1e = g.Vb1e;
        v.N1 = N1;
        v.nbr1 = g.nbr1.data();
        v.sites = g.sites.data();
        v.blk_of = g.blk_of.data();
        v.loc_of = g.loc_of.data();
        v.same = g.same.data();
        v.B1 = reinterpret_cast<const C*>(B1);
        v.Dinv1 = reinterpret_cast<const C*>(Dinv1);
        v.P1 = reinterpret_cast<const C*>(P1);
    }
};
}  // namespace

extern "C" {

int mlh_geom_sizes(const int* L1, const int* b1, int* out /* NB, NB2, Vb1, Vb1e */) {
    MLHostGeom g;
    if (ml_build_geom(L1, b1, g)) return -1;
    out[0] = g.NB;
    out[1] = g.NB2;
    out[2] = g.Vb1;
    out[3] = g.Vb1e;
    return 0;
}

int mlh_geom_fill(const int* L1, const int* b1, int* lex1, int* nbr1, int* sites, int* blk_of, int* loc_of, unsigned char* same,
                  int* nbr2, int* lex2) {
    MLHostGeom g;
    if (ml_build_geom(L1, b1, g)) return -1;
    std::memcpy(lex1, g.lex1.data(), g.lex1.size() * sizeof(int));
    std::memcpy(nbr1, g.nbr1.data(), g.nbr1.size() * sizeof(int));
    std::memcpy(sites, g.sites.data(), g.sites.size() * sizeof(int));
    std::memcpy(blk_of, g.blk_of.data(), g.blk_of.size() * sizeof(int));
    std::memcpy(loc_of, g.loc_of.data(), g.loc_of.size() * sizeof(int));
    std::memcpy(same, g.same.data(), g.same.size());
    std::memcpy(nbr2, g.nbr2.data(), g.nbr2.size() * sizeof(int));
    std::memcpy(lex2, g.lex2.data(), g.lex2.size() * sizeof(int));
    return 0;
}

// z <- nu SAP iterations on D_1 z = b from the given z
int mlh_sap(const int* L1, const int* b1, int nc, const double* B1, const double* Dinv1, const double* b, double* z, int nrhs, int nu,
            int mr_steps) {
    HostLevel L(L1, b1, nc, 1, B1, Dinv1, nullptr);
    if (L.ok) return -1;
    const size_t nf = (size_t)nrhs * L.g.NB * nc;
    std::vector<C> r(nf), te(nf), rho(nf), u(nf), w(nf), s(nf), x(nf), alpha((size_t)nrhs * L.g.NB2);
    MLSapWork<double> wk{r.data(), te.data(), rho.data(), u.data(), w.data(), s.data(), x.data(), alpha.data()};
    return ml_sap(MLHostExec{}, L.v, reinterpret_cast<const C*>(b), reinterpret_cast<C*>(z), nrhs, nu, mr_steps, wk);
}

// the same SAP in FP32 (the precision of the solves on SINGLE and HALF handles): inputs and the
// result are complex128, rounded to complex64 on entry
int mlh_sap_f32(const int* L1, const int* b1, int nc, const double* B1, const double* Dinv1, const double* b, double* z, int nrhs,
                int nu, int mr_steps) {
    MLHostGeom g;
    if (ml_build_geom(L1, b1, g)) return -1;
    auto to_f = [](const double* p, size_t n) {
        std::vector<cplx<float>> out(n);
        for (size_t i = 0; i < n; ++i) out[i] = mk((float)p[2 * i], (float)p[2 * i + 1]);
        return out;
    };
    const size_t nf = (size_t)nrhs * g.NB * nc;
    std::vector<cplx<float>> Bf = to_f(B1, (size_t)g.NB * 9 * nc * nc), Df = to_f(Dinv1, (size_t)(g.NB / 2) * nc * nc), bf = to_f(b, nf),
                             zf = to_f(z, nf);
    MLView<float> v{};
    v.NB = g.NB;
    v.nc = nc;
    v.half = nc / 2;
    v.NB2 = g.NB2;
    v.Vb1 = g.Vb1;
    v.Vb1e = g.Vb1e;
    v.N1 = 1;
    v.nbr1 = g.nbr1.data();
    v.sites = g.sites.data();
    v.blk_of = g.blk_of.data();
    v.loc_of = g.loc_of.data();
    v.same = g.same.data();
    v.B1 = Bf.data();
    v.Dinv1 = Df.data();
    std::vector<cplx<float>> r(nf), te(nf), rho(nf), u(nf), w(nf), s(nf), x(nf), alpha((size_t)nrhs * g.NB2);
    MLSapWork<float> wk{r.data(), te.data(), rho.data(), u.data(), w.data(), s.data(), x.data(), alpha.data()};
    const int rc = ml_sap(MLHostExec{}, v, bf.data(), zf.data(), nrhs, nu, mr_steps, wk);
    for (size_t i = 0; i < nf; ++i) {
        z[2 * i] = zf[i].re;
        z[2 * i + 1] = zf[i].im;
    }
    return rc;
}

int mlh_gram_schmidt(const int* L1, const int* b1, int nc, int N1, const double* vec, double* P1) {
    HostLevel L(L1, b1, nc, N1, nullptr, nullptr, nullptr);
    if (L.ok) return -1;
    int fail = 0;
    MLHostExec{}.run((long long)L.g.NB2 * 2, MLGramSchmidt<double>{L.v, reinterpret_cast<const C*>(vec), reinterpret_cast<C*>(P1), &fail});
    return fail ? -8 : 0;
}

int mlh_restrict(const int* L1, const int* b1, int nc, int N1, const double* P1, const double* x, double* e, int nrhs) {
    HostLevel L(L1, b1, nc, N1, nullptr, nullptr, P1);
    if (L.ok) return -1;
    return MLHostExec{}.run((long long)nrhs * L.g.NB2 * 2 * N1, MLRestrict<double>{L.v, reinterpret_cast<const C*>(x), reinterpret_cast<C*>(e)});
}

int mlh_prolong(const int* L1, const int* b1, int nc, int N1, const double* P1, const double* e, double* y, int nrhs) {
    HostLevel L(L1, b1, nc, N1, nullptr, nullptr, P1);
    if (L.ok) return -1;
    return MLHostExec{}.run((long long)nrhs * L.g.NB * nc, MLProlong<double>{L.v, reinterpret_cast<const C*>(e), reinterpret_cast<C*>(y)});
}

int mlh_apply(const int* L1, const int* b1, int nc, const double* B1, const double* x, double* y, int nrhs) {
    HostLevel L(L1, b1, nc, 1, B1, nullptr, nullptr);
    if (L.ok) return -1;
    return MLHostExec{}.run((long long)L.g.NB * nc,
                            MLFullApply<double>{L.v, reinterpret_cast<const C*>(x), nullptr, reinterpret_cast<C*>(y), nrhs});
}

int mlh_galerkin(const int* L1, const int* b1, int nc, int N1, const double* B1, const double* P1, double* B2) {
    HostLevel L(L1, b1, nc, N1, B1, nullptr, P1);
    if (L.ok) return -1;
    const int nc2 = 2 * N1;
    std::vector<C> E((size_t)nc2 * L.g.NB2 * nc2), e(E.size()), W((size_t)nc2 * L.g.NB * nc), Y(W.size());
    return ml_galerkin(MLHostExec{}, L.v, reinterpret_cast<C*>(B2), E.data(), W.data(), Y.data(), e.data());
}

// ---- the level-1 V-cycle and setup with an exact level-2 solve (dense inverse of D_2) ----

namespace {
// inverse of a dense n x n complex matrix (row-major) by Gauss-Jordan with partial pivoting
bool dense_inverse(std::vector<C>& A, int n) {
    std::vector<C> I((size_t)n * n, czero<double>());
    for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = mk(1.0, 0.0);
    for (int p = 0; p < n; ++p) {
        int piv = p;
        for (int i = p + 1; i < n; ++i)
            if (norm2(A[(size_t)i * n + p]) > norm2(A[(size_t)piv * n + p])) piv = i;
        if (norm2(A[(size_t)piv * n + p]) == 0.0) return false;
        for (int j = 0; j < n; ++j) {
            std::swap(A[(size_t)p * n + j], A[(size_t)piv * n + j]);
            std::swap(I[(size_t)p * n + j], I[(size_t)piv * n + j]);
        }
        const C d = A[(size_t)p * n + p];
        const double dn = norm2(d);
        const C dinv = mk(d.re / dn, -d.im / dn);
        for (int j = 0; j < n; ++j) {
            A[(size_t)p * n + j] = dinv * A[(size_t)p * n + j];
            I[(size_t)p * n + j] = dinv * I[(size_t)p * n + j];
        }
        for (int i = 0; i < n; ++i) {
            if (i == p) continue;
            const C f = A[(size_t)i * n + p];
            for (int j = 0; j < n; ++j) {
                A[(size_t)i * n + j] = A[(size_t)i * n + j] - f * A[(size_t)p * n + j];
                I[(size_t)i * n + j] = I[(size_t)i * n + j] - f * I[(size_t)p * n + j];
            }
        }
    }
    A.swap(I);
    return true;
}

// the dense matrix of D_2 (internal level-2 order, row-major) from its nine-block stencil
std::vector<C> dense_D2(const MLHostGeom& g, const C* B2, int nc2) {
    const int n = g.NB2 * nc2;
    std::vector<C> M((size_t)n * n, czero<double>());
    for (int c2 = 0; c2 < g.NB2; ++c2)
        for (int d = 0; d < 9; ++d) {
            const int nb = d == 0 ? c2 : g.nbr2[(size_t)(d - 1) * g.NB2 + c2];
            for (int col = 0; col < nc2; ++col)
                for (int row = 0; row < nc2; ++row) {
                    C& m = M[(size_t)(c2 * nc2 + row) * n + nb * nc2 + col];
                    m = m + B2[(((size_t)c2 * 9 + d) * nc2 + col) * nc2 + row];
                }
        }
    return M;
}

struct DenseCoarse {
    const std::vector<C>* inv;
    int n;
    int operator()(const C* eb, C* ex, int nrhs) const {
        for (int r = 0; r < nrhs; ++r)
            for (int i = 0; i < n; ++i) {
                C acc = czero<double>();
                for (int j = 0; j < n; ++j) cmac(acc, (*inv)[(size_t)i * n + j], eb[(size_t)r * n + j]);
                ex[(size_t)r * n + i] = acc;
            }
        return 0;
    }
};

struct SapBufs {
    std::vector<C> r, te, rho, u, w, s, x, alpha;
    SapBufs(size_t nf, size_t na) : r(nf), te(nf), rho(nf), u(nf), w(nf), s(nf), x(nf), alpha(na) {}
    MLSapWork<double> work() { return {r.data(), te.data(), rho.data(), u.data(), w.data(), s.data(), x.data(), alpha.data()}; }
};
}  // namespace

// x = the level-1 V-cycle of r with D_2 solved exactly (D2inv: dense inverse, internal order)
int mlh_vcycle1(const int* L1, const int* b1, int nc, int N1, const double* B1, const double* Dinv1, const double* P1, const double* D2inv,
                const double* r, double* x, int nrhs, int nu, int mr_steps) {
    HostLevel L(L1, b1, nc, N1, B1, Dinv1, P1);
    if (L.ok) return -1;
    const int n2 = L.g.NB2 * 2 * N1;
    std::vector<C> inv(reinterpret_cast<const C*>(D2inv), reinterpret_cast<const C*>(D2inv) + (size_t)n2 * n2);
    SapBufs sb((size_t)nrhs * L.g.NB * nc, (size_t)nrhs * L.g.NB2);
    std::vector<C> eb((size_t)nrhs * n2), ex((size_t)nrhs * n2);
    return ml_vcycle1_t(MLHostExec{}, L.v, reinterpret_cast<const C*>(r), reinterpret_cast<C*>(x), nrhs, nu, mr_steps, sb.work(), eb.data(),
                        ex.data(), DenseCoarse{&inv, n2});
}

// the level-1 V-cycle in FP32 (SINGLE and HALF handles): inputs rounded to complex64, the exact
// level-2 solve applied in FP32 too, the result returned as complex128
int mlh_vcycle1_f32(const int* L1, const int* b1, int nc, int N1, const double* B1, const double* Dinv1, const double* P1, const double* D2inv,
                    const double* r, double* x, int nrhs, int nu, int mr_steps) {
    MLHostGeom g;
    if (ml_build_geom(L1, b1, g)) return -1;
    using F = cplx<float>;
    auto to_f = [](const double* p, size_t n) {
        std::vector<F> out(n);
        for (size_t i = 0; i < n; ++i) out[i] = mk((float)p[2 * i], (float)p[2 * i + 1]);
        return out;
    };
    const int n2 = g.NB2 * 2 * N1;
    const size_t nf = (size_t)nrhs * g.NB * nc;
    std::vector<F> Bf = to_f(B1, (size_t)g.NB * 9 * nc * nc), Df = to_f(Dinv1, (size_t)(g.NB / 2) * nc * nc),
                   Pf = to_f(P1, (size_t)g.NB * nc * N1), If = to_f(D2inv, (size_t)n2 * n2), rf = to_f(r, nf), xf(nf);
    MLView<float> v{};
    v.NB = g.NB;
    v.nc = nc;
    v.half = nc / 2;
    v.NB2 = g.NB2;
    v.Vb1 = g.Vb1;
    v.Vb1e = g.Vb1e;
    v.N1 = N1;
    v.nbr1 = g.nbr1.data();
    v.sites = g.sites.data();
    v.blk_of = g.blk_of.data();
    v.loc_of = g.loc_of.data();
    v.same = g.same.data();
    v.B1 = Bf.data();
    v.Dinv1 = Df.data();
    v.P1 = Pf.data();
    std::vector<F> r1(nf), te(nf), rho(nf), u(nf), w(nf), s(nf), x1(nf), alpha((size_t)nrhs * g.NB2), eb((size_t)nrhs * n2),
        ex((size_t)nrhs * n2);
    MLSapWork<float> wk{r1.data(), te.data(), rho.data(), u.data(), w.data(), s.data(), x1.data(), alpha.data()};
    auto coarse = [&](const F* b2, F* x2, int nr) {
        for (int q = 0; q < nr; ++q)
            for (int i = 0; i < n2; ++i) {
                F acc = czero<float>();
                for (int j = 0; j < n2; ++j) cmac(acc, If[(size_t)i * n2 + j], b2[(size_t)q * n2 + j]);
                x2[(size_t)q * n2 + i] = acc;
            }
        return 0;
    };
    const int rc = ml_vcycle1_t(MLHostExec{}, v, rf.data(), xf.data(), nrhs, nu, mr_steps, wk, eb.data(), ex.data(), coarse);
    for (size_t i = 0; i < nf; ++i) {
        x[2 * i] = xf[i].re;
        x[2 * i + 1] = xf[i].im;
    }
    return rc;
}

// the level-1 setup from the initial vectors vec (returned updated), with exact level-2 solves;
// P1 and B2 receive the final interpolation and D_2
int mlh_setup1(const int* L1, const int* b1, int nc, int N1, const double* B1, const double* Dinv1, double* vec, int n_inv, int idsetup,
               int nu, int mr_steps, double* P1, double* B2) {
    HostLevel L(L1, b1, nc, N1, B1, Dinv1, P1);
    if (L.ok) return -1;
    const int nc2 = 2 * N1, n2 = L.g.NB2 * nc2;
    const size_t fs = (size_t)L.g.NB * nc;
    SapBufs sb((size_t)N1 * fs, (size_t)N1 * L.g.NB2);
    std::vector<C> t((size_t)N1 * fs), u((size_t)N1 * fs), E((size_t)nc2 * L.g.NB2 * nc2), e(E.size()), W((size_t)nc2 * fs), Y(W.size());
    std::vector<C> inv;
    std::vector<double> nrm(N1);
    C* Pm = reinterpret_cast<C*>(P1);
    C* Bm = reinterpret_cast<C*>(B2);
    const MLView<double> v = L.v;
    auto rebuild = [&](const C* vv) -> int {
        int fail = 0;
        MLHostExec{}.run((long long)L.g.NB2 * 2, MLGramSchmidt<double>{v, vv, Pm, &fail});
        if (fail) return -8;
        if (ml_galerkin(MLHostExec{}, v, Bm, E.data(), W.data(), Y.data(), e.data())) return -1;
        inv = dense_D2(L.g, Bm, nc2);
        return dense_inverse(inv, n2) ? 0 : -8;
    };
    std::vector<C> eb((size_t)N1 * n2), ex((size_t)N1 * n2);
    SapBufs sv((size_t)N1 * fs, (size_t)N1 * L.g.NB2);
    auto vcycle = [&](const C* r, C* x, int nr) -> int {
        return ml_vcycle1_t(MLHostExec{}, v, r, x, nr, nu, mr_steps, sv.work(), eb.data(), ex.data(), DenseCoarse{&inv, n2});
    };
    return ml_setup1_t(MLHostExec{}, v, reinterpret_cast<C*>(vec), n_inv, idsetup != 0, mr_steps, sb.work(), t.data(), u.data(), nrm.data(),
                       rebuild, vcycle);
}

}  // extern "C"
