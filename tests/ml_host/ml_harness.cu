// Test harness: runs the level-1 operations of the CUDA library (the functors and orchestration of
// ml_ops.cuh, the blocking of ml_geom.h) on the host through the loop executor, so that their index
// arithmetic and algebra can be compared with the oracle without a GPU.  Built by the tests as a
// host-only shared library; the product never loads it.  Arrays are complex128 as (re, im) pairs in
// the internal orders described in ml_ops.cuh; B1/Dinv1/B2 column-major.
#include <cstring>
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
    return MLHostExec{}.run((long long)nrhs * L.g.NB * nc,
                            MLFullApply<double>{L.v, reinterpret_cast<const C*>(x), nullptr, reinterpret_cast<C*>(y)});
}

int mlh_galerkin(const int* L1, const int* b1, int nc, int N1, const double* B1, const double* P1, double* B2) {
    HostLevel L(L1, b1, nc, N1, B1, nullptr, P1);
    if (L.ok) return -1;
    const int nc2 = 2 * N1;
    std::vector<C> E((size_t)nc2 * L.g.NB2 * nc2), e(E.size()), W((size_t)nc2 * L.g.NB * nc), Y(W.size());
    return ml_galerkin(MLHostExec{}, L.v, reinterpret_cast<C*>(B2), E.data(), W.data(), Y.data(), e.data());
}

}  // extern "C"
