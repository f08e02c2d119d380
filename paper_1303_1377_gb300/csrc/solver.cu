// Host side of libddamg: the handle, the internal lattice ordering, the
// adaptive setup (Algorithms 1-2), the V-cycle (Sec. 4.2), batched restarted
// GMRES for the odd-even coarse system (Sec. 6) and the outer FGMRES (Sec. 5),
// and every extern "C" entry point declared in include/ddamg.h.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <random>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_fp16.h>

#include "blas.h"
#include "kernels.h"

namespace ddamg {

std::atomic<unsigned long long> g_launches{0};
static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }
static int g_fail_allocs = 0;

static int dalloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (g_fail_allocs > 0) {
        --g_fail_allocs;
        set_error("device allocation failed (forced by ddamg_debug_fail_allocs)");
        return DDAMG_ERR_OOM;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        return DDAMG_ERR_OOM;
    }
    return 0;
}
template <typename T>
static int dalloc_n(T** p, size_t n) {
    return dalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}
template <typename T>
static void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

#define DD_TRY(x)                  \
    do {                           \
        int _rc = (x);             \
        if (_rc) return _rc;       \
    } while (0)

// profiling families
// (the two ml_ families are wall time of whole recursion stages, recorded with zero bytes)
enum { PF_DSLASH64 = 0, PF_DSLASH32, PF_SAP, PF_COARSE, PF_RESTRICT, PF_PROLONG, PF_DSLASHDW, PF_ORTHO, PF_UPDATE, PF_ML_VCYCLE,
       PF_ML_COARSE, PF_COUNT };
static const char* kPfNames[PF_COUNT] = {"dslash_fp64", "dslash_fp32",   "sap_block_mr", "coarse_stencil", "restrict",   "prolong",
                                         "dslash_dw",   "krylov_ortho",  "krylov_update", "ml_vcycle1",   "ml_coarse2"};

struct ProfRec {
    int fam;
    cudaEvent_t e0, e1;
    double bytes;
    double flops;
};

// a growable set of device buffers kept by the handle
struct Scratch {
    void* p = nullptr;
    size_t bytes = 0;
    int ensure(size_t b) {
        if (b <= bytes) return 0;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        DD_TRY(dalloc(&p, b));
        bytes = b;
        return 0;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T>
    T* as() const {
        return reinterpret_cast<T*>(p);
    }
};

// Krylov state + small buffers for nrhs right-hand sides, restart length m
struct KrylovBufs {
    int nrhs = 0, m = 0;
    KrylovState s{};
    cplx<double>* hcol = nullptr;   // [(m+2)][nrhs]
    cplx<double>* hcol2 = nullptr;  // second Gram-Schmidt pass
    cplx<double>* scale = nullptr;  // [nrhs]
    cplx<double>* y = nullptr;      // [m][nrhs]
    cplx<double>* nrm = nullptr;    // [nrhs]
    cplx<double>* ones = nullptr;   // [nrhs] = 1
    float4* coefdw = nullptr;       // [(m+2)][nrhs] double-word coefficients
    cplx<double>* nbefore = nullptr;  // [nrhs] ||w||^2 before orthogonalisation
    int* dflag = nullptr;             // device-side "second Gram-Schmidt pass" decision
    unsigned* tickets = nullptr;      // [nrhs] last-CTA counters of the FP32 reductions (kept at zero between launches)
    double* dscr = nullptr;         // multidot scratch
    int* h_active = nullptr;        // pinned copy of active flags
    int* h_active_lag[2] = {nullptr, nullptr};  // lagged convergence check: flags of steps k-1 and k
    cudaEvent_t ev_lag[2] = {nullptr, nullptr};
    int* h_steps = nullptr;
    double* h_resid = nullptr;
    int* h_flags = nullptr;
    // Arnoldi steps captured as CUDA graphs (problems that allow it, KrylovProblem::graph), one per
    // step index k.  The signature lists every pointer and size the captured launches baked in; a step
    // runs eagerly the first time a signature is seen, is captured the second time and replayed after.
    struct StepGraph {
        cudaGraphExec_t exec = nullptr;
        std::array<uintptr_t, 12> sig{};
        bool seen = false;
        size_t nkern = 0;  // kernel launches in the graph (counted again at every replay)
    };
    std::vector<StepGraph> graphs;
    bool graphs_off = false;  // a capture failed: steps of this solver run eagerly from then on
    void drop_graphs() {
        for (auto& g : graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        graphs.clear();
    }
    int alloc(int nr, int mm) {
        if (nr <= nrhs && mm == m) return 0;
        release();
        nrhs = nr;
        m = mm;
        s.nrhs = nr;
        s.m = mm;
        DD_TRY(dalloc_n(&s.H, (size_t)nr * (mm + 1) * mm));
        DD_TRY(dalloc_n(&s.cs, (size_t)nr * mm));
        DD_TRY(dalloc_n(&s.sn, (size_t)nr * mm));
        DD_TRY(dalloc_n(&s.g, (size_t)nr * (mm + 1)));
        DD_TRY(dalloc_n(&s.steps, nr));
        DD_TRY(dalloc_n(&s.resid, nr));
        DD_TRY(dalloc_n(&s.active, nr));
        DD_TRY(dalloc_n(&s.enabled, nr));
        DD_TRY(dalloc_n(&s.flags, nr));
        DD_TRY(dalloc_n(&s.target, nr));
        DD_TRY(dalloc_n(&s.ctarget, nr));
        s.cycle_tol = 0.0;
        DD_TRY(dalloc_n(&hcol, (size_t)(mm + 2) * nr));
        DD_TRY(dalloc_n(&hcol2, (size_t)(mm + 2) * nr));
        DD_TRY(dalloc_n(&scale, nr));
        DD_TRY(dalloc_n(&y, (size_t)mm * nr));
        DD_TRY(dalloc_n(&nrm, nr));
        DD_TRY(dalloc_n(&ones, nr));
        DD_TRY(dalloc_n(&coefdw, (size_t)(mm + 2) * nr));
        DD_TRY(dalloc_n(&nbefore, nr));
        DD_TRY(dalloc_n(&dflag, 1));
        DD_TRY(dalloc_n(&tickets, nr));
        DD_CUDA(cudaMemset(tickets, 0, sizeof(unsigned) * nr));
        {
            std::vector<cplx<double>> one(nr, mk(1.0, 0.0));
            DD_CUDA(cudaMemcpy(ones, one.data(), sizeof(cplx<double>) * nr, cudaMemcpyHostToDevice));
        }
        DD_TRY(dalloc_n(&dscr, multidot_scratch_doubles(1) + multidot_scratch_doubles(nr)));
        DD_CUDA(cudaMallocHost(&h_active, sizeof(int) * nr));
        for (int q = 0; q < 2; ++q) {
            DD_CUDA(cudaMallocHost(&h_active_lag[q], sizeof(int) * nr));
            DD_CUDA(cudaEventCreateWithFlags(&ev_lag[q], cudaEventDisableTiming));
        }
        DD_CUDA(cudaMallocHost(&h_steps, sizeof(int) * nr));
        DD_CUDA(cudaMallocHost(&h_resid, sizeof(double) * nr));
        DD_CUDA(cudaMallocHost(&h_flags, sizeof(int) * nr));
        return 0;
    }
    void release() {
        drop_graphs();
        dfree(s.H);
        dfree(s.cs);
        dfree(s.sn);
        dfree(s.g);
        dfree(s.steps);
        dfree(s.resid);
        dfree(s.active);
        dfree(s.enabled);
        dfree(s.flags);
        dfree(s.target);
        dfree(s.ctarget);
        dfree(hcol);
        dfree(hcol2);
        dfree(scale);
        dfree(y);
        dfree(nrm);
        dfree(ones);
        dfree(coefdw);
        dfree(nbefore);
        dfree(dflag);
        dfree(tickets);
        dfree(dscr);
        if (h_active) cudaFreeHost(h_active);
        for (int q = 0; q < 2; ++q) {
            if (h_active_lag[q]) cudaFreeHost(h_active_lag[q]);
            if (ev_lag[q]) cudaEventDestroy(ev_lag[q]);
            h_active_lag[q] = nullptr;
            ev_lag[q] = nullptr;
        }
        if (h_steps) cudaFreeHost(h_steps);
        if (h_resid) cudaFreeHost(h_resid);
        if (h_flags) cudaFreeHost(h_flags);
        h_active = h_steps = h_flags = nullptr;
        h_resid = nullptr;
        nrhs = m = 0;
    }
};

}  // namespace ddamg

using namespace ddamg;

namespace ddamg {
struct MLState;  // third level of the recursion (multilevel.inc)
}

struct ddamg_handle {
    // geometry
    int L[4], b[4], nbk[4];
    int V, Vb, NB, N, nc;
    int device = 0;  // the CUDA device current at creation: every allocation and stream of the handle is on it
    ddamg_params p;
    double m0, csw;
    cudaStream_t own_stream = nullptr, stream = nullptr;
    std::vector<int> h_lex_of, h_clex_of;
    int *d_blex = nullptr;
    int *d_lnbr = nullptr, *d_bnbr = nullptr, *d_lex_of = nullptr, *d_clex_of = nullptr, *d_sites = nullptr;
    int nsites[9];
    Geom g;
    // operator (FP64 always, FP32 copy for the single/half modes)
    cplx<double>* U64 = nullptr;
    double *clov64 = nullptr, *clovinv64 = nullptr;
    cplx<float>* U32 = nullptr;
    float *clov32 = nullptr, *clovinv32 = nullptr;
    float4 *Uaos = nullptr, *clov_aos = nullptr, *clovinv_aos = nullptr;  // per-site FP32 copies for the SAP
    uint4 *Uaos16 = nullptr, *clov_aos16 = nullptr, *clovinv_aos16 = nullptr;  // half mode: FP16 per-site copies
    float4* Udw = nullptr;    // links as double-word FP32 pairs (FGMRES matvec on FP32 inputs)
    float2* clovdw = nullptr;  // site terms as double-word pairs
    // interpolation
    bool ready = false;
    cplx<double>* V64 = nullptr;  // test vectors [N][12][V]
    cplx<double>* P64 = nullptr;
    cplx<float>* P32 = nullptr;
    double *B64 = nullptr, *Dinv64 = nullptr;
    float *B32 = nullptr, *Dinv32 = nullptr;
    uint4 *Bh = nullptr, *Dh = nullptr;  // half mode: FP16 fragments of D_c and D_ee^{-1}
    cplx<__half>* P16 = nullptr;          // half mode: FP16 interpolation
    CoarseTC tc{};
    int* d_flag = nullptr;
    int* d_tc_err = nullptr;  // half mode: set by a coarse-stencil kernel whose bulk copy did not complete
    // workspaces
    Scratch ws_fine[6], ws_coarse[8], ws_io[3], ws_outer[5];
    Scratch ws_rmax;  // per right-hand-side field maxima of the tensor-core restriction
    KrylovBufs kc, ko;
    // continuous batching: right-hand sides and iterates of the slots (internal order, FP64)
    int n_slots = 0;
    cplx<double>* slot_b = nullptr;
    cplx<double>* slot_x = nullptr;
    std::vector<int> slot_state;
    std::vector<long long> slot_iters;
    std::vector<double> slot_resid;  // coarse GMRES, outer FGMRES
    // stats of the current call
    long long coarse_iters = 0;
    int vcycles = 0;
    double coarse_seconds = 0;
    // profiling
    int prof_mask = 0;  // bit f: record kernel family f
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    // recursion to a third level (ddamg_ml_build); coarse_gen counts rebuilds and shifts of D_c
    ddamg::MLState* ml = nullptr;
    unsigned long long coarse_gen = 0;
    bool ml_route = false;  // set by ddamg_ml_solve: the fine V-cycle takes the recursive coarse solve
    // last setup: update rounds run, and (n_inv_auto_rhs) the probes' estimated iterations per solve
    int setup_rounds = 0;
    std::vector<double> setup_est_iters;

    bool single() const { return p.precision != DDAMG_PREC_DOUBLE; }
    bool half() const { return p.precision == DDAMG_PREC_HALF; }
};

namespace ddamg {

static cudaEvent_t get_event(ddamg_handle* h) {
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

struct Prof {
    ddamg_handle* h;
    ProfRec r;
    bool on;
    Prof(ddamg_handle* hh, int fam, double bytes, double flops = 0.0) : h(hh), on((hh->prof_mask >> fam) & 1) {
        if (on) {
            r.fam = fam;
            r.bytes = bytes;
            r.flops = flops;
            r.e0 = get_event(h);
            r.e1 = get_event(h);
            cudaEventRecord(r.e0, h->stream);
        }
    }
    ~Prof() {
        if (on) {
            cudaEventRecord(r.e1, h->stream);
            h->prof.push_back(r);
        }
    }
};

// ---------------------------------------------------------------------------
// internal ordering (see common.cuh)
// ---------------------------------------------------------------------------
static int build_geometry(ddamg_handle* h) {
    int nbt = 1, vb = 1;
    for (int m = 0; m < 4; ++m) {
        h->nbk[m] = h->L[m] / h->b[m];
        nbt *= h->nbk[m];
        vb *= h->b[m];
    }
    h->NB = nbt;
    h->Vb = vb;
    h->V = nbt * vb;
    // blocks: red (even block-coordinate sum) first, each colour lexicographic
    std::vector<std::array<int, 4>> bcoord(nbt);
    std::vector<int> blex_to_int(nbt);
    {
        int idx = 0;
        for (int colour = 0; colour < 2; ++colour)
            for (int q = 0; q < nbt; ++q) {
                int c3 = q % h->nbk[3], c2 = (q / h->nbk[3]) % h->nbk[2], c1 = (q / (h->nbk[3] * h->nbk[2])) % h->nbk[1],
                    c0 = q / (h->nbk[3] * h->nbk[2] * h->nbk[1]);
                if (((c0 + c1 + c2 + c3) & 1) != colour) continue;
                bcoord[idx] = {c0, c1, c2, c3};
                blex_to_int[q] = idx;
                ++idx;
            }
    }
    h->h_clex_of.resize(nbt);
    for (int q = 0; q < nbt; ++q) h->h_clex_of[blex_to_int[q]] = q;
    // local sites: even first, each lexicographic
    std::vector<std::array<int, 4>> lcoord(vb);
    std::vector<int> llex_to_int(vb);
    {
        int idx = 0;
        for (int par = 0; par < 2; ++par)
            for (int q = 0; q < vb; ++q) {
                int y3 = q % h->b[3], y2 = (q / h->b[3]) % h->b[2], y1 = (q / (h->b[3] * h->b[2])) % h->b[1],
                    y0 = q / (h->b[3] * h->b[2] * h->b[1]);
                if (((y0 + y1 + y2 + y3) & 1) != par) continue;
                lcoord[idx] = {y0, y1, y2, y3};
                llex_to_int[q] = idx;
                ++idx;
            }
    }
    auto llex = [&](const std::array<int, 4>& y) { return ((y[0] * h->b[1] + y[1]) * h->b[2] + y[2]) * h->b[3] + y[3]; };
    auto blex = [&](const std::array<int, 4>& c) { return ((c[0] * h->nbk[1] + c[1]) * h->nbk[2] + c[2]) * h->nbk[3] + c[3]; };
    std::vector<int> lnbr(8 * vb), bnbr(8 * nbt);
    std::vector<int> sites(9 * vb, 0);
    for (int d = 0; d < 9; ++d) h->nsites[d] = 0;
    for (int l = 0; l < vb; ++l) sites[h->nsites[0]++] = l;
    for (int d = 0; d < 8; ++d) {
        int mu = d >> 1, s = (d & 1) ? -1 : 1;
        for (int l = 0; l < vb; ++l) {
            std::array<int, 4> y = lcoord[l];
            y[mu] += s;
            int cross = 0;
            if (y[mu] < 0 || y[mu] >= h->b[mu]) {
                cross = 1;
                y[mu] = (y[mu] + h->b[mu]) % h->b[mu];
            }
            lnbr[d * vb + l] = llex_to_int[llex(y)] | (cross << 16);
            if (cross) sites[(1 + d) * vb + h->nsites[1 + d]++] = l;
        }
        for (int c = 0; c < nbt; ++c) {
            std::array<int, 4> cc = bcoord[c];
            cc[mu] = (cc[mu] + s + h->nbk[mu]) % h->nbk[mu];
            bnbr[d * nbt + c] = blex_to_int[blex(cc)];
        }
    }
    h->h_lex_of.resize(h->V);
    for (int c = 0; c < nbt; ++c)
        for (int l = 0; l < vb; ++l) {
            int x[4];
            for (int m = 0; m < 4; ++m) x[m] = bcoord[c][m] * h->b[m] + lcoord[l][m];
            h->h_lex_of[(size_t)c * vb + l] = ((x[0] * h->L[1] + x[1]) * h->L[2] + x[2]) * h->L[3] + x[3];
        }
    DD_TRY(dalloc_n(&h->d_lnbr, lnbr.size()));
    DD_TRY(dalloc_n(&h->d_bnbr, bnbr.size()));
    DD_TRY(dalloc_n(&h->d_lex_of, h->h_lex_of.size()));
    DD_TRY(dalloc_n(&h->d_clex_of, h->h_clex_of.size()));
    DD_TRY(dalloc_n(&h->d_sites, sites.size()));
    DD_TRY(dalloc_n(&h->d_blex, blex_to_int.size()));
    DD_CUDA(cudaMemcpy(h->d_blex, blex_to_int.data(), blex_to_int.size() * 4, cudaMemcpyHostToDevice));
    DD_CUDA(cudaMemcpy(h->d_lnbr, lnbr.data(), lnbr.size() * 4, cudaMemcpyHostToDevice));
    DD_CUDA(cudaMemcpy(h->d_bnbr, bnbr.data(), bnbr.size() * 4, cudaMemcpyHostToDevice));
    DD_CUDA(cudaMemcpy(h->d_lex_of, h->h_lex_of.data(), h->h_lex_of.size() * 4, cudaMemcpyHostToDevice));
    DD_CUDA(cudaMemcpy(h->d_clex_of, h->h_clex_of.data(), h->h_clex_of.size() * 4, cudaMemcpyHostToDevice));
    DD_CUDA(cudaMemcpy(h->d_sites, sites.data(), sites.size() * 4, cudaMemcpyHostToDevice));
    h->g.V = h->V;
    h->g.Vb = vb;
    h->g.NB = nbt;
    h->g.vb_shift = -1;
    h->g.blk44 = h->b[0] == 4 && h->b[1] == 4 && h->b[2] == 4 && h->b[3] == 4;
    for (int s = 0; s < 31; ++s)
        if ((1 << s) == vb) h->g.vb_shift = s;
    h->g.lnbr = h->d_lnbr;
    h->g.bnbr = h->d_bnbr;
    h->g.blex = h->d_blex;
    return 0;
}

// gamma_mu gamma_nu (mu < nu) chiral blocks, from the gamma matrices of Sec. 2.2
static int upload_gammas() {
    static bool done = false;
    if (done) return 0;
    typedef std::array<std::array<std::array<double, 2>, 4>, 4> G4;
    G4 gm[4];
    for (auto& g : gm)
        for (auto& r : g)
            for (auto& e : r) e = {0.0, 0.0};
    // gamma_0: (0,3)=i (1,2)=i (2,1)=-i (3,0)=-i
    gm[0][0][3] = {0, 1}; gm[0][1][2] = {0, 1}; gm[0][2][1] = {0, -1}; gm[0][3][0] = {0, -1};
    // gamma_1: (0,3)=-1 (1,2)=1 (2,1)=1 (3,0)=-1
    gm[1][0][3] = {-1, 0}; gm[1][1][2] = {1, 0}; gm[1][2][1] = {1, 0}; gm[1][3][0] = {-1, 0};
    // gamma_2: (0,2)=i (1,3)=-i (2,0)=-i (3,1)=i
    gm[2][0][2] = {0, 1}; gm[2][1][3] = {0, -1}; gm[2][2][0] = {0, -1}; gm[2][3][1] = {0, 1};
    // gamma_3: (0,2)=1 (1,3)=1 (2,0)=1 (3,1)=1
    gm[3][0][2] = {1, 0}; gm[3][1][3] = {1, 0}; gm[3][2][0] = {1, 0}; gm[3][3][1] = {1, 0};
    double gg[6][2][2][2][2];
    int plane = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
            double prod[4][4][2];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    double re = 0, im = 0;
                    for (int k = 0; k < 4; ++k) {
                        re += gm[mu][i][k][0] * gm[nu][k][j][0] - gm[mu][i][k][1] * gm[nu][k][j][1];
                        im += gm[mu][i][k][0] * gm[nu][k][j][1] + gm[mu][i][k][1] * gm[nu][k][j][0];
                    }
                    prod[i][j][0] = re;
                    prod[i][j][1] = im;
                }
            for (int hh = 0; hh < 2; ++hh)
                for (int s = 0; s < 2; ++s)
                    for (int t = 0; t < 2; ++t) {
                        gg[plane][hh][s][t][0] = prod[2 * hh + s][2 * hh + t][0];
                        gg[plane][hh][s][t][1] = prod[2 * hh + s][2 * hh + t][1];
                    }
        }
    DD_TRY(upload_gamma_products(&gg[0][0][0][0][0]));
    done = true;
    return 0;
}

static bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// device view of caller data: device pointers pass through, host data is staged
static int stage_in(ddamg_handle* h, Scratch& s, const void* src, size_t bytes, const void** dev) {
    if (is_device_ptr(src)) {
        *dev = src;
        return 0;
    }
    DD_TRY(s.ensure(bytes));
    DD_CUDA(cudaMemcpyAsync(s.p, src, bytes, cudaMemcpyHostToDevice, h->stream));
    *dev = s.p;
    return 0;
}
static int stage_out_ptr(Scratch& s, void* dst, size_t bytes, void** dev, bool* host) {
    *host = !is_device_ptr(dst);
    if (!*host) {
        *dev = dst;
        return 0;
    }
    DD_TRY(s.ensure(bytes));
    *dev = s.p;
    return 0;
}
static int finish_out(ddamg_handle* h, void* dst, const void* dev, size_t bytes, bool host) {
    if (host) DD_CUDA(cudaMemcpyAsync(dst, dev, bytes, cudaMemcpyDeviceToHost, h->stream));
    DD_CUDA(cudaStreamSynchronize(h->stream));
    return 0;
}

// ---------------------------------------------------------------------------
// precision views
// ---------------------------------------------------------------------------
template <typename T>
struct Level {
    FineOp<T> op;
    const cplx<T>* P;
    CoarseOp<T> cop;
};
static Level<double> level64(ddamg_handle* h) {
    Level<double> L;
    L.op = {h->U64, h->clov64, h->clovinv64};
    L.P = h->P64;
    L.cop = {h->B64, h->Dinv64, h->d_bnbr, h->NB, h->nc};
    return L;
}
static Level<float> level32(ddamg_handle* h) {
    Level<float> L;
    L.op = {h->U32, h->clov32, h->clovinv32};
    L.P = h->P32;
    L.cop = {h->B32, h->Dinv32, h->d_bnbr, h->NB, h->nc};
    return L;
}
template <typename T>
static Level<T> level(ddamg_handle* h);
template <>
Level<double> level<double>(ddamg_handle* h) {
    return level64(h);
}
template <>
Level<float> level<float>(ddamg_handle* h) {
    return level32(h);
}

static double dslash_bytes(ddamg_handle* h, size_t real, int nrhs, bool resid) {
    double site = 36.0 * 2 * real + 72.0 * real;  // links + clover, once per launch
    double vec = (resid ? 36.0 : 24.0) * 2 * real;  // in + out (+ b) per rhs
    return (double)h->V * (site + vec * nrhs);
}

template <typename T, typename Ts>
static int dslash(ddamg_handle* h, const cplx<Ts>* in, const cplx<T>* b, cplx<T>* out, int nrhs) {
    Level<T> L = level<T>(h);
    Prof pr(h, sizeof(T) == 8 ? PF_DSLASH64 : PF_DSLASH32, dslash_bytes(h, sizeof(T), nrhs, b != nullptr));
    return launch_dslash<T, Ts>(h->g, L.op, in, b, out, nrhs, h->stream);
}

// w = D z for FP32 z with an FP64-accurate result (double-word arithmetic)
static int dslash_dw(ddamg_handle* h, const cplx<float>* z, cplx<double>* w, int nrhs) {
    Prof pr(h, PF_DSLASHDW, (double)h->V * (36.0 * 16 + 72.0 * 8 + nrhs * (12.0 * 8 + 12.0 * 16)));
    return launch_dslash_dw(h->g, h->Udw, h->clovdw, z, w, false, nrhs, h->stream);
}

// z <- SAP iterations (nu) on D z = b from the current z (Sec. 2.3)
// algorithmic flops of one red or black SAP sweep per (even, odd) site pair and right-hand side:
// full D at both sites for the residual, A_ee^{-1} r_e, the reduced right-hand side, mr MR steps
// (S rho: in-block hops twice, A_ee^{-1}, A_oo, dot products and updates), back-substitution.
// One hop = 168 flops (spin projection, two SU(3) x colour-vector products, reconstruction),
// one 2 x (6x6 hermitian) site-term product = 504 flops.
static double sap_pair_flops(const ddamg_handle* h) {
    double hin = 0;  // in-block hops per site
    for (int m = 0; m < 4; ++m) hin += 2.0 * (h->b[m] - 1) / h->b[m];
    const double hop = 168, site = 504;
    return 2 * (8 * hop + site) + site + hin * hop + h->p.mr_steps * (2 * hin * hop + 2 * site + 144) + hin * hop + site;
}

template <typename T>
static int sap(ddamg_handle* h, const cplx<T>* b, cplx<T>* z, int nrhs, int nu) {
    Level<T> L = level<T>(h);
    for (int it = 0; it < nu; ++it)
        for (int colour = 0; colour < 2; ++colour) {
            // operator bytes at their stored size: FP16 links and site terms on the half-mode path
            const bool f16 = std::is_same<T, float>::value && h->half() && h->p.smoother_fp16 && sap_aos_supported(h->g, nrhs);
            const double opb = f16 ? 2.0 : (double)sizeof(T);
            Prof pr(h, PF_SAP, (double)h->V / 2 * (36.0 * 2 * opb + 144.0 * opb + nrhs * 36.0 * 2 * sizeof(T)),
                    (double)h->V / 4 * nrhs * sap_pair_flops(h));
            if constexpr (std::is_same<T, float>::value) {
                if (f16) {
                    // half-precision V-cycle: links and site terms of the smoother stored in FP16
                    const FineOpAoS16 op{LinksAoS16{h->Uaos16}, CloverAoS16{h->clov_aos16}, CloverAoS16{h->clovinv_aos16}};
                    DD_TRY(launch_sap_colour_aos16(h->g, op, b, z, colour, nrhs, h->p.mr_steps, h->stream));
                    continue;
                }
                if (sap_aos_supported(h->g, nrhs)) {
                    const FineOpAoS op{LinksAoS{h->Uaos}, CloverAoS{h->clov_aos}, CloverAoS{h->clovinv_aos}};
                    DD_TRY(launch_sap_colour_aos(h->g, op, b, z, colour, nrhs, h->p.mr_steps, h->stream));
                    continue;
                }
            }
            DD_TRY(launch_sap_colour<T>(h->g, L.op, b, z, colour, nrhs, h->p.mr_steps, h->stream));
        }
    return 0;
}

template <typename T>
static int restrict_(ddamg_handle* h, const cplx<T>* in, cplx<T>* out, int nrhs) {
    Level<T> L = level<T>(h);
    const double pb = h->half() ? 2.0 : sizeof(T);
    Prof pr(h, PF_RESTRICT, (double)h->V * (12.0 * h->N * 2 * pb + 12.0 * nrhs * 2 * sizeof(T)));
    if (std::is_same<T, float>::value && h->half()) {
        if (restrict_tc_supported(h->g, h->N)) {
            DD_TRY(h->ws_rmax.ensure(sizeof(int) * nrhs));
            return launch_restrict_tc(h->g, h->P16, h->N, reinterpret_cast<const cplx<float>*>(in), reinterpret_cast<cplx<float>*>(out),
                                      nrhs, h->ws_rmax.as<int>(), h->stream);
        }
        return launch_restrict<float, __half>(h->g, h->P16, h->N, reinterpret_cast<const cplx<float>*>(in),
                                              reinterpret_cast<cplx<float>*>(out), nrhs, h->stream);
    }
    return launch_restrict<T, T>(h->g, L.P, h->N, in, out, nrhs, h->stream);
}
template <typename T>
static int prolong_(ddamg_handle* h, const cplx<T>* in, cplx<T>* out, int nrhs) {
    Level<T> L = level<T>(h);
    const double pb = h->half() ? 2.0 : sizeof(T);
    Prof pr(h, PF_PROLONG, (double)h->V * (12.0 * h->N * 2 * pb + 12.0 * nrhs * 2 * sizeof(T)));
    if (std::is_same<T, float>::value && h->half()) {
        if (prolong_tc_supported(h->g, h->N))
            return launch_prolong_tc(h->g, h->P16, h->N, reinterpret_cast<const cplx<float>*>(in), reinterpret_cast<cplx<float>*>(out),
                                     nrhs, h->stream);
        return launch_prolong<float, __half>(h->g, h->P16, h->N, reinterpret_cast<const cplx<float>*>(in),
                                             reinterpret_cast<cplx<float>*>(out), nrhs, h->stream);
    }
    return launch_prolong<T, T>(h->g, L.P, h->N, in, out, nrhs, h->stream);
}

// coarse stencil dispatch: FP16 tensor-core storage in half mode, CUDA cores otherwise
template <typename T>
static int c_even(ddamg_handle* h, const cplx<T>* b_e, size_t b_rs, const cplx<T>* x_o, size_t x_rs, T beta, cplx<T>* out_e,
                  size_t o_rs, int nrhs) {
    if (std::is_same<T, float>::value && h->half())
        return tc_coarse_even(h->tc, reinterpret_cast<const cplx<float>*>(b_e), b_rs, reinterpret_cast<const cplx<float>*>(x_o), x_rs,
                              (float)beta, reinterpret_cast<cplx<float>*>(out_e), o_rs, nrhs, h->stream);
    return launch_coarse_even<T, T>(level<T>(h).cop, b_e, b_rs, x_o, x_rs, beta, out_e, o_rs, nrhs, h->stream);
}
template <typename T>
static int c_odd(ddamg_handle* h, const cplx<T>* x_o, size_t x_rs, const cplx<T>* t_e, size_t t_rs, int use_diag, cplx<T>* out_o,
                 size_t o_rs, int nrhs) {
    if (std::is_same<T, float>::value && h->half())
        return tc_coarse_odd(h->tc, reinterpret_cast<const cplx<float>*>(x_o), x_rs, reinterpret_cast<const cplx<float>*>(t_e), t_rs,
                             use_diag, reinterpret_cast<cplx<float>*>(out_o), o_rs, nrhs, h->stream);
    return launch_coarse_odd<T, T>(level<T>(h).cop, x_o, x_rs, t_e, t_rs, use_diag, out_o, o_rs, nrhs, h->stream);
}
template <typename T>
static int c_full(ddamg_handle* h, const cplx<T>* x, cplx<T>* y, int nrhs) {
    if (std::is_same<T, float>::value && h->half())
        return tc_coarse_full(h->tc, reinterpret_cast<const cplx<float>*>(x), reinterpret_cast<cplx<float>*>(y), nrhs, h->stream);
    return launch_coarse_full<T, T>(level<T>(h).cop, x, y, nrhs, h->stream);
}

// ---------------------------------------------------------------------------
// batched restarted (F)GMRES.  Vectors of length n per rhs, rhs stride n.
// TB: right-hand side / iterate (and true residuals), TV: Arnoldi basis,
// TZ: preconditioned vectors.  A: w = A z (TZ -> TV); Ax: residual product (TB -> TB);
// M (optional): z = M v (flexible, Z basis kept).
// ---------------------------------------------------------------------------
template <typename TB, typename TV, typename TZ>
struct KrylovProblem {
    size_t n;
    int nrhs;
    int m;
    std::function<int(const cplx<TZ>*, cplx<TV>*)> A;
    std::function<int(const cplx<TB>*, cplx<TB>*)> Ax;
    std::function<int(const cplx<TB>*, cplx<TV>*)> residual;  // optional: V0 = b - A x straight into the basis type
    std::function<int(const cplx<TV>*, cplx<TZ>*)> M;
    const cplx<TB>* b;
    cplx<TB>* x;
    bool x0_zero;
    double tol;            // relative to ||b_r||
    long long maxiter;     // Arnoldi steps per rhs
    bool fixed;            // run exactly maxiter steps (no tolerance)
    bool reorth;           // second Gram-Schmidt pass: always (generic path), on the DGKS test (lean path)
    bool lean = false;     // FP32 basis: one Gram-Schmidt pass, a second one only on heavy cancellation
    double cycle_tol = 0;  // > 0: a cycle ends once every rhs has reduced its residual by this factor
    int max_cycles = 0;    // > 0: return after this many cycles (x updated, no closing residual)
    bool lag_check = false;  // decide "all converged" from the flags of the previous step, without waiting for
                             // the current one (the GPU keeps a step queued; a step after convergence changes
                             // nothing, since inactive right-hand sides are frozen on the device)
    bool graph = false;         // the Arnoldi step (A and the FP32 one-pass Gram-Schmidt) may be captured and replayed:
                                // A has no host synchronisation, and graph_sig names the buffers it bakes in
    std::array<const void*, 4> graph_sig{};
    unsigned graph_prof_mask = 0;  // profile families that A records (no capture while one of them is timed)
    bool has_deadline = false;  // wall-clock limit: checked at every host synchronisation of the iteration;
    std::chrono::steady_clock::time_point deadline{};  // once passed, x takes the current cycle's update and the solve returns
    cplx<TV>* Vb;          // basis [(m+1)][nrhs][n]
    cplx<TZ>* Zb;          // [m][nrhs][n] when M is set
    cplx<TV>* w;           // [nrhs][n]
    cplx<TB>* wB;          // [nrhs][n] residual scratch (may alias w when TB == TV)
    const int* enabled_host;
};

struct KrylovResult {
    std::vector<long long> iters;
    std::vector<double> resid;  // last residual estimate relative to ||b||
    std::vector<double> bnorm;
    std::vector<int> start_active;  // per rhs at the start of the first cycle (0: converged or not enabled)
    std::vector<int> flags;         // per rhs: bit 1 = non-finite value met
    int restarts = 0;
    bool nonfinite = false;
    bool converged = true;
    bool timed_out = false;  // the wall-clock limit ended the iteration (x holds the last iterate)
};

// basis-space kernels (generic precisions / double-word)
template <typename TV>
static int bdot(KrylovBufs& kb, const cplx<TV>* A, size_t istride, int k, const cplx<TV>* w, size_t n, int nr, cplx<double>* out,
                cudaStream_t st) {
    return multidot<TV, TV>(A, istride, n, k, w, n, n, nr, out, nr, kb.dscr, st);
}
template <typename TV>
static int baxpy(KrylovBufs& kb, cplx<TV>* out, bool accumulate, const cplx<TV>* A, size_t istride, int k, const cplx<double>* coef,
                 size_t n, int nr, double alpha, cudaStream_t st) {
    return lincomb<TV, TV>(out, n, accumulate ? 1.0 : 0.0, A, istride, n, k, coef, nr, n, nr, nullptr, st, alpha);
}
template <>
int baxpy<dwf>(KrylovBufs& kb, cplx<dwf>* out, bool accumulate, const cplx<dwf>* A, size_t istride, int k, const cplx<double>* coef,
               size_t n, int nr, double alpha, cudaStream_t st) {
    return lincomb_dw(out, n, accumulate ? 1 : 0, A, istride, n, k, coef, nr, n, nr, alpha, kb.coefdw, st);
}
template <typename TV, typename TB>
static int bfrom(cplx<TV>* out, const cplx<TB>* in, size_t count, cudaStream_t st) {
    if (sizeof(TV) == sizeof(TB)) {
        DD_CUDA(cudaMemcpyAsync(out, in, sizeof(cplx<TV>) * count, cudaMemcpyDeviceToDevice, st));
        return 0;
    }
    set_error("unsupported basis conversion");
    return DDAMG_ERR_INVALID_ARG;
}
template <>
int bfrom<float, double>(cplx<float>* out, const cplx<double>* in, size_t count, cudaStream_t st) {
    return convert<float, double>(reinterpret_cast<const double*>(in), reinterpret_cast<float*>(out), 2 * count, st);
}
template <>
int bfrom<dwf, double>(cplx<dwf>* out, const cplx<double>* in, size_t count, cudaStream_t st) {
    return convert_d2dw(reinterpret_cast<const double*>(in), out, 2 * count, st);
}

// one-pass Gram-Schmidt kernels of the double-word and FP32 bases (w in the V_{k+1} slot)
template <typename TV>
static int lean_multidot(const cplx<TV>* Vb, size_t bstride, size_t n, int k, const cplx<TV>* w, int nr, cplx<double>* out,
                         KrylovBufs& kb, const int* flag, cudaStream_t st, cplx<double>* copy_last = nullptr) {
    if constexpr (std::is_same<TV, dwf>::value) {
        DD_TRY(multidot_dw(Vb, bstride, n, k, w, n, n, nr, out, nr, kb.dscr, flag, st));
        if (copy_last)
            DD_CUDA(cudaMemcpyAsync(copy_last, out + (size_t)(k - 1) * nr, sizeof(cplx<double>) * nr, cudaMemcpyDeviceToDevice, st));
        return 0;
    } else if constexpr (std::is_same<TV, float>::value) {
        if (multidot_f32(Vb, bstride, n, k, w, n, n, nr, out, nr, kb.dscr, kb.tickets, copy_last, flag, st)) {
            set_error("FP32 basis: odd length or misaligned vector");
            return DDAMG_ERR_INVALID_ARG;
        }
        return 0;
    } else {
        set_error("no one-pass Gram-Schmidt for this basis type");
        return DDAMG_ERR_INVALID_ARG;
    }
}
template <typename TV>
static int lean_axpy_norm(cplx<TV>* w, const cplx<TV>* Vb, size_t bstride, size_t n, int k, const cplx<double>* coef, int nr,
                          KrylovBufs& kb, cplx<double>* norm_out, const int* flag, cudaStream_t st) {
    if constexpr (std::is_same<TV, dwf>::value) {
        return axpy_norm_dw(w, Vb, bstride, n, k, coef, nr, n, nr, -1.0, kb.coefdw, kb.dscr, norm_out, flag, st);
    } else if constexpr (std::is_same<TV, float>::value) {
        if (axpy_norm_f32(w, Vb, bstride, n, k, coef, nr, n, nr, -1.0, kb.dscr, kb.tickets, norm_out, flag, st)) {
            set_error("FP32 basis: odd length or misaligned vector");
            return DDAMG_ERR_INVALID_ARG;
        }
        return 0;
    } else {
        set_error("no one-pass Gram-Schmidt for this basis type");
        return DDAMG_ERR_INVALID_ARG;
    }
}

template <typename TB, typename TV, typename TZ>
static int krylov(ddamg_handle* h, KrylovBufs& kb, KrylovProblem<TB, TV, TZ>& P, KrylovResult& R) {
    cudaStream_t st = h->stream;
    const int nr = P.nrhs;
    const size_t n = P.n;
    DD_TRY(kb.alloc(nr, P.m));
    KrylovState& s = kb.s;
    s.nrhs = nr;
    s.cycle_tol = P.cycle_tol;
    R.iters.assign(nr, 0);
    R.resid.assign(nr, 0.0);
    R.bnorm.assign(nr, 0.0);
    R.flags.assign(nr, 0);
    R.start_active.assign(nr, 0);
    int ncycles = 0;
    // ||b||, targets, enabled
    DD_TRY((multidot<TB, TB>(P.b, 0, n, 1, P.b, n, n, nr, kb.nrm, 1, kb.dscr, st)));
    std::vector<cplx<double>> hb(nr);
    DD_CUDA(cudaMemcpyAsync(hb.data(), kb.nrm, sizeof(cplx<double>) * nr, cudaMemcpyDeviceToHost, st));
    DD_CUDA(cudaStreamSynchronize(st));
    std::vector<double> target(nr);
    std::vector<int> en(nr, 1);
    for (int r = 0; r < nr; ++r) {
        R.bnorm[r] = std::sqrt(hb[r].re);
        target[r] = P.fixed ? -1.0 : P.tol * R.bnorm[r];
        if (P.enabled_host && !P.enabled_host[r]) en[r] = 0;
        if (!(R.bnorm[r] == R.bnorm[r])) R.nonfinite = true;
    }
    DD_CUDA(cudaMemcpyAsync(s.target, target.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, st));
    DD_CUDA(cudaMemcpyAsync(s.enabled, en.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, st));
    DD_CUDA(cudaMemsetAsync(s.flags, 0, sizeof(int) * nr, st));
    const size_t bstride = (size_t)nr * n;  // between basis vectors
    cplx<TV>* V0 = P.Vb;
    // V0 = b - A x (in the iterate's precision), or b for a zero guess
    auto residual_to_V0 = [&]() -> int {
        if (P.residual) return P.residual(P.x, V0);
        DD_TRY(P.Ax(P.x, P.wB));
        DD_TRY((lincomb<TB, TB>(P.wB, n, -1.0, P.b, 0, n, 1, kb.ones, nr, n, nr, nullptr, st)));
        return bfrom<TV, TB>(V0, P.wB, n * nr, st);
    };
    if (P.x0_zero) {
        DD_CUDA(cudaMemsetAsync(P.x, 0, sizeof(cplx<TB>) * nr * n, st));
        DD_TRY((bfrom<TV, TB>(V0, P.b, n * nr, st)));
    } else {
        DD_TRY(residual_to_V0());
    }
    long long total = 0;
    while (true) {
        // start of a cycle
        if constexpr (std::is_same<TV, float>::value) {
            if (P.lean) {
                DD_TRY(lean_multidot(V0, 0, n, 1, V0, nr, kb.nrm, kb, nullptr, st));
            } else {
                DD_TRY(bdot<TV>(kb, V0, 0, 1, V0, n, nr, kb.nrm, st));
            }
        } else {
            DD_TRY(bdot<TV>(kb, V0, 0, 1, V0, n, nr, kb.nrm, st));
        }
        DD_TRY(arnoldi_start(s, kb.nrm, kb.scale, P.fixed ? 1 : 0, st));
        if constexpr (std::is_same<TV, float>::value) {
            if (P.lean) {
                if (scale_f32(V0, kb.scale, n, nr, st)) {
                    set_error("FP32 basis: odd length or misaligned vector");
                    return DDAMG_ERR_INVALID_ARG;
                }
            } else {
                DD_TRY(baxpy<TV>(kb, V0, false, V0, 0, 1, kb.scale, n, nr, 1.0, st));
            }
        } else {
            DD_TRY(baxpy<TV>(kb, V0, false, V0, 0, 1, kb.scale, n, nr, 1.0, st));
        }
        DD_CUDA(cudaMemcpyAsync(kb.h_active, s.active, sizeof(int) * nr, cudaMemcpyDeviceToHost, st));
        DD_CUDA(cudaMemcpyAsync(kb.h_resid, s.resid, sizeof(double) * nr, cudaMemcpyDeviceToHost, st));
        DD_CUDA(cudaMemcpyAsync(kb.h_flags, s.flags, sizeof(int) * nr, cudaMemcpyDeviceToHost, st));
        DD_CUDA(cudaStreamSynchronize(st));
        int nact = 0;
        for (int r = 0; r < nr; ++r) {
            nact += kb.h_active[r];
            if (en[r]) R.resid[r] = R.bnorm[r] > 0 ? kb.h_resid[r] / R.bnorm[r] : 0.0;
            R.flags[r] |= kb.h_flags[r];
        }
        if (ncycles == 0) R.start_active.assign(kb.h_active, kb.h_active + nr);
        if (nact == 0) break;
        if (total >= P.maxiter) {
            R.converged = false;
            break;
        }
        if (P.has_deadline && std::chrono::steady_clock::now() >= P.deadline) {
            R.timed_out = true;
            break;
        }
        int k = 0;
        for (; k < P.m; ++k) {
            cplx<TV>* Vk = P.Vb + (size_t)k * bstride;
            const cplx<TZ>* zk;
            if (P.M) {
                cplx<TZ>* Zk = P.Zb + (size_t)k * bstride;
                DD_TRY(P.M(Vk, Zk));
                zk = Zk;
            } else {
                zk = reinterpret_cast<const cplx<TZ>*>(Vk);
            }
            bool lean_step = false;
            if constexpr (std::is_same<TV, dwf>::value || std::is_same<TV, float>::value)
                lean_step = std::is_same<TV, dwf>::value || P.lean;
            // a captured step: FP32 one-pass Gram-Schmidt without the DGKS pass, no preconditioner, the
            // Gram-Schmidt family not being timed (event records cannot time a graph's insides)
            auto step_body = [&]() -> int {
                if (lean_step) {
                    // w is formed in the V_{k+1} slot; one multi-dot gives <V_i, w> (i <= k) and ||w||^2,
                    // the axpy kernel returns ||w'||^2, and the second classical Gram-Schmidt pass runs
                    // only when the first one cancelled more than 1 - eta of w (eta = 1e-3, decided on the
                    // device).  With the 48-bit double-word basis one pass leaves a non-orthogonality of
                    // about 1e-14 ||w|| / ||w'||, far below what a 1e-10 solve needs; the FP64 true residual
                    // at every restart certifies convergence whatever the basis quality.
                    // (FP32 basis: the same scheme; one pass leaves about 1e-7 ||w|| / ||w'|| of
                    // non-orthogonality, ample for a cycle that reduces the residual by cycle_tol)
                    cplx<TV>* wk = P.Vb + (size_t)(k + 1) * bstride;
                    DD_TRY(P.A(zk, wk));
                    const double vb = (double)sizeof(cplx<TV>) * n * nr;
                    Prof pr(h, PF_ORTHO, vb * (2 * (k + 1) + 6));
                    // the last product is ||w||^2 before orthogonalisation, kept for the DGKS test
                    DD_TRY(lean_multidot(P.Vb, bstride, n, k + 2, wk, nr, kb.hcol, kb, nullptr, st, kb.nbefore));
                    DD_TRY(lean_axpy_norm(wk, P.Vb, bstride, n, k + 1, kb.hcol, nr, kb, kb.hcol + (size_t)(k + 1) * nr, nullptr, st));
                    if (P.reorth) {
                        DD_TRY(dgks(kb.nbefore, kb.hcol + (size_t)(k + 1) * nr, s.active, nr, 1e-3, kb.dflag, st));
                        DD_TRY(lean_multidot(P.Vb, bstride, n, k + 1, wk, nr, kb.hcol2, kb, kb.dflag, st));
                        DD_TRY(lean_axpy_norm(wk, P.Vb, bstride, n, k + 1, kb.hcol2, nr, kb, kb.hcol + (size_t)(k + 1) * nr, kb.dflag, st));
                        DD_TRY(add_columns_flag(kb.hcol, kb.hcol2, (k + 1) * nr, kb.dflag, st));
                    }
                    DD_TRY(arnoldi_update(s, k, kb.hcol, kb.scale, st));
                    if constexpr (std::is_same<TV, float>::value) {
                        if (scale_f32(wk, kb.scale, n, nr, st)) {
                            set_error("FP32 basis: odd length or misaligned vector");
                            return DDAMG_ERR_INVALID_ARG;
                        }
                    } else {
                        DD_TRY(baxpy<TV>(kb, wk, false, wk, 0, 1, kb.scale, n, nr, 1.0, st));
                    }
                } else {
                    DD_TRY(P.A(zk, P.w));
                    // classical Gram-Schmidt (twice when reorth)
                    const double vb = (double)sizeof(cplx<TV>) * n * nr;
                    Prof pr(h, PF_ORTHO, vb * ((k + 1) * (P.reorth ? 4 : 2) + 4));
                    DD_TRY(bdot<TV>(kb, P.Vb, bstride, k + 1, P.w, n, nr, kb.hcol, st));
                    DD_TRY(baxpy<TV>(kb, P.w, true, P.Vb, bstride, k + 1, kb.hcol, n, nr, -1.0, st));
                    if (P.reorth) {
                        DD_TRY(bdot<TV>(kb, P.Vb, bstride, k + 1, P.w, n, nr, kb.hcol2, st));
                        DD_TRY(baxpy<TV>(kb, P.w, true, P.Vb, bstride, k + 1, kb.hcol2, n, nr, -1.0, st));
                        DD_TRY(add_columns(kb.hcol, kb.hcol2, (k + 1) * nr, st));
                    }
                    DD_TRY(bdot<TV>(kb, P.w, 0, 1, P.w, n, nr, kb.hcol + (size_t)(k + 1) * nr, st));
                    DD_TRY(arnoldi_update(s, k, kb.hcol, kb.scale, st));
                    DD_TRY(baxpy<TV>(kb, P.Vb + (size_t)(k + 1) * bstride, false, P.w, 0, 1, kb.scale, n, nr, 1.0, st));
                }
                return 0;
            };
            bool graph_step = false;
            if constexpr (std::is_same<TV, float>::value)  // (the legacy default streams cannot be captured)
                graph_step = lean_step && P.graph && !kb.graphs_off && !P.M && !P.reorth &&
                             !(h->prof_mask & ((1u << PF_ORTHO) | P.graph_prof_mask)) &&
                             st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
            if (graph_step) {
                if ((int)kb.graphs.size() < P.m) kb.graphs.resize(P.m);
                KrylovBufs::StepGraph& sg = kb.graphs[k];
                const std::array<uintptr_t, 12> sig = {(uintptr_t)P.Vb, (uintptr_t)n, (uintptr_t)nr, (uintptr_t)kb.s.H,
                                                       (uintptr_t)kb.hcol, (uintptr_t)kb.dscr, (uintptr_t)kb.tickets,
                                                       (uintptr_t)P.graph_sig[0], (uintptr_t)P.graph_sig[1], (uintptr_t)P.graph_sig[2],
                                                       (uintptr_t)P.graph_sig[3], (uintptr_t)(P.cycle_tol * 1e15)};
                if (sg.exec && sg.sig == sig) {
                    DD_CUDA(cudaGraphLaunch(sg.exec, st));
                    g_launches += sg.nkern;
                } else if (sg.seen && sg.sig == sig) {  // second time: capture, then replay
                    if (sg.exec) cudaGraphExecDestroy(sg.exec);
                    sg.exec = nullptr;
                    DD_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                    const int rc = step_body();  // recorded, not run
                    cudaGraph_t g = nullptr;
                    cudaError_t e = cudaStreamEndCapture(st, &g);
                    if (rc == 0 && e == cudaSuccess) {
                        // (the capture counted the graph's launches once: they run once right below)
                        if (cudaGraphGetNodes(g, nullptr, &sg.nkern) != cudaSuccess) sg.nkern = 0;
                        e = cudaGraphInstantiate(&sg.exec, g, 0);
                        if (e != cudaSuccess) sg.exec = nullptr;
                    }
                    if (g) cudaGraphDestroy(g);
                    if (sg.exec) {
                        DD_CUDA(cudaGraphLaunch(sg.exec, st));
                    } else {  // not capturable after all: run the step eagerly, and do not try this problem again
                        (void)cudaGetLastError();
                        kb.graphs_off = true;
                        DD_TRY(step_body());
                    }
                } else {  // first time with this signature: run eagerly
                    if (sg.exec) cudaGraphExecDestroy(sg.exec);
                    sg.exec = nullptr;
                    sg.sig = sig;
                    sg.seen = true;
                    DD_TRY(step_body());
                }
            } else {
                DD_TRY(step_body());
            }
            ++total;
            if (P.fixed) {
                if (total >= P.maxiter) {
                    ++k;
                    break;
                }
                continue;
            }
            int na = 0;
            if (P.lag_check) {
                // flags after this step go to one pinned slot; the host waits only for those of the
                // previous step, which the GPU has finished while this step is queued behind it
                DD_CUDA(cudaMemcpyAsync(kb.h_active_lag[k & 1], s.active, sizeof(int) * nr, cudaMemcpyDeviceToHost, st));
                DD_CUDA(cudaEventRecord(kb.ev_lag[k & 1], st));
                if (k == 0) {
                    na = 1;  // nothing to look at yet (the cycle started with an active right-hand side)
                } else {
                    DD_CUDA(cudaEventSynchronize(kb.ev_lag[(k - 1) & 1]));
                    for (int r = 0; r < nr; ++r) na += kb.h_active_lag[(k - 1) & 1][r];
                }
            } else {
                DD_CUDA(cudaMemcpyAsync(kb.h_active, s.active, sizeof(int) * nr, cudaMemcpyDeviceToHost, st));
                DD_CUDA(cudaStreamSynchronize(st));
                for (int r = 0; r < nr; ++r) na += kb.h_active[r];
            }
            if (na > 0 && P.has_deadline && std::chrono::steady_clock::now() >= P.deadline) R.timed_out = true;
            if (na == 0 || total >= P.maxiter || R.timed_out) {
                ++k;
                break;
            }
        }
        // x += sum_i y_i Z_i (or V_i)
        DD_TRY(arnoldi_solve(s, kb.y, st));
        {
            Prof pru(h, PF_UPDATE, (double)n * nr * (2 * sizeof(cplx<TB>) + std::min(k, P.m) * sizeof(cplx<TZ>)));
            if (P.M && std::is_same<TB, double>::value && std::is_same<TZ, float>::value)
                DD_TRY(xupdate_dw(reinterpret_cast<cplx<double>*>(P.x), reinterpret_cast<const cplx<float>*>(P.Zb), bstride, n,
                                  std::min(k, P.m), kb.y, nr, kb.coefdw, st));
            else if (P.M)
                DD_TRY((lincomb<TB, TZ>(P.x, n, 1.0, P.Zb, bstride, n, std::min(k, P.m), kb.y, nr, n, nr, nullptr, st)));
            else
                DD_TRY((lincomb<TB, TZ>(P.x, n, 1.0, reinterpret_cast<const cplx<TZ>*>(P.Vb), bstride, n, std::min(k, P.m), kb.y, nr,
                                        n, nr, nullptr, st)));
        }
        DD_CUDA(cudaMemcpyAsync(kb.h_steps, s.steps, sizeof(int) * nr, cudaMemcpyDeviceToHost, st));
        DD_CUDA(cudaMemcpyAsync(kb.h_resid, s.resid, sizeof(double) * nr, cudaMemcpyDeviceToHost, st));
        DD_CUDA(cudaMemcpyAsync(kb.h_flags, s.flags, sizeof(int) * nr, cudaMemcpyDeviceToHost, st));
        DD_CUDA(cudaStreamSynchronize(st));
        for (int r = 0; r < nr; ++r) {
            R.iters[r] += kb.h_steps[r];
            if (kb.h_steps[r] > 0) R.resid[r] = R.bnorm[r] > 0 ? kb.h_resid[r] / R.bnorm[r] : 0.0;
            if (kb.h_flags[r] & 2) R.nonfinite = true;
            R.flags[r] |= kb.h_flags[r];
        }
        if (P.fixed && total >= P.maxiter) break;
        if (R.nonfinite || R.timed_out) break;
        ++ncycles;
        if (P.max_cycles > 0 && ncycles >= P.max_cycles) break;
        // restart: V0 = b - A x
        DD_TRY(residual_to_V0());
        ++R.restarts;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// coarse solve: odd-even reduced GMRES(restart) (Sec. 6) on full coarse vectors
// ---------------------------------------------------------------------------
template <typename T>
static int coarse_solve(ddamg_handle* h, const cplx<T>* bc, cplx<T>* xc, int nrhs, int fixed_iters) {
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = h->stream;
    const int H = h->NB / 2, nc = h->nc;
    const size_t hn = (size_t)H * nc, full = (size_t)h->NB * nc;
    const int m = h->p.coarse_restart;
    DD_TRY(h->ws_coarse[0].ensure(sizeof(cplx<T>) * hn * nrhs));
    DD_TRY(h->ws_coarse[1].ensure(sizeof(cplx<T>) * hn * nrhs));
    DD_TRY(h->ws_coarse[2].ensure(sizeof(cplx<T>) * hn * nrhs));
    DD_TRY(h->ws_coarse[3].ensure(sizeof(cplx<T>) * hn * nrhs));
    DD_TRY(h->ws_coarse[4].ensure(sizeof(cplx<T>) * hn * nrhs * (m + 1)));
    cplx<T>* te = h->ws_coarse[0].as<cplx<T>>();
    cplx<T>* bp = h->ws_coarse[1].as<cplx<T>>();
    cplx<T>* xo = h->ws_coarse[2].as<cplx<T>>();
    cplx<T>* w = h->ws_coarse[3].as<cplx<T>>();
    cplx<T>* basis = h->ws_coarse[4].as<cplx<T>>();
    Level<T> L = level<T>(h);
    const double sbytes = (double)h->NB * 9 * nc * nc * (h->half() && sizeof(T) == 4 ? 4.0 : sizeof(cplx<T>));
    const double vbytes = 2.0 * hn * nrhs * sizeof(cplx<T>);  // one half vector in, one out
    {
        Prof pr(h, PF_COARSE, sbytes / 18 + vbytes);
        DD_TRY(c_even<T>(h, bc, full, nullptr, 0, T(0), te, hn, nrhs));
    }
    {
        Prof pr(h, PF_COARSE, sbytes * 4 / 9 + 1.5 * vbytes);
        DD_TRY(c_odd<T>(h, bc + hn, full, te, hn, 0, bp, hn, nrhs));
    }
    KrylovProblem<T, T, T> P;
    P.n = hn;
    P.nrhs = nrhs;
    P.m = m;
    P.A = [&](const cplx<T>* v, cplx<T>* out) -> int {
        {
            Prof pr(h, PF_COARSE, sbytes / 2 + vbytes);
            DD_TRY(c_even<T>(h, nullptr, 0, v, hn, T(1), te, hn, nrhs));
        }
        Prof pr(h, PF_COARSE, sbytes / 2 + 1.5 * vbytes);
        return c_odd<T>(h, v, hn, te, hn, 1, out, hn, nrhs);
    };
    P.Ax = P.A;
    P.b = bp;
    P.x = xo;
    P.x0_zero = true;
    P.tol = h->p.coarse_tol;
    P.fixed = fixed_iters > 0;
    P.maxiter = fixed_iters > 0 ? fixed_iters : h->p.coarse_maxiter;
    P.reorth = false;
    P.lean = std::is_same<T, float>::value;  // FP32 kernels with the norm fused into the update
    P.lag_check = true;
    P.Vb = basis;
    P.Zb = nullptr;
    P.w = w;
    P.wB = w;
    P.enabled_host = nullptr;
    P.graph = true;  // A is two stencil launches on te and the handle's coarse operator
    P.graph_sig = {te, h->half() ? (const void*)h->Bh : (const void*)L.cop.B, (const void*)(uintptr_t)h->NB, nullptr};
    P.graph_prof_mask = 1u << PF_COARSE;
    KrylovResult R;
    DD_TRY((krylov<T, T, T>(h, h->kc, P, R)));
    long long it = 0;
    for (long long v : R.iters) it = std::max(it, v);
    h->coarse_iters += it;
    // back-substitution x_e = D_ee^{-1} (b_e - D_eo x_o); x_o into the odd half
    {
        Prof pr(h, PF_COARSE, sbytes / 2 + 1.5 * vbytes);
        DD_TRY(c_even<T>(h, bc, full, xo, hn, T(-1), xc, full, nrhs));
    }
    DD_CUDA(cudaMemcpy2DAsync(xc + hn, full * sizeof(cplx<T>), xo, hn * sizeof(cplx<T>), hn * sizeof(cplx<T>), nrhs,
                              cudaMemcpyDeviceToDevice, st));
    h->coarse_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return 0;
}

// x = C^(nu) r (Sec. 4.2): x = P D_c^{-1} P^H r, then nu SAP iterations on D x = r
// starting from that x, which adds M_SAP^(nu) (r - D x) (the SAP update is affine).
template <typename T>
static int vcycle(ddamg_handle* h, const cplx<T>* r, cplx<T>* x, int nrhs, int coarse_fixed) {
    const size_t full = (size_t)h->NB * h->nc;
    DD_TRY(h->ws_coarse[5].ensure(sizeof(cplx<T>) * full * nrhs));
    DD_TRY(h->ws_coarse[6].ensure(sizeof(cplx<T>) * full * nrhs));
    cplx<T>* cb = h->ws_coarse[5].as<cplx<T>>();
    cplx<T>* cx = h->ws_coarse[6].as<cplx<T>>();
    DD_TRY(restrict_<T>(h, r, cb, nrhs));
    DD_TRY(coarse_solve<T>(h, cb, cx, nrhs, coarse_fixed));
    DD_TRY(prolong_<T>(h, cx, x, nrhs));
    DD_TRY(sap<T>(h, r, x, nrhs, h->p.nu));
    h->vcycles += nrhs;
    return 0;
}

// ---------------------------------------------------------------------------
// interpolation: P by local orthonormalisation, D_c by assembly, coarse inverses
// ---------------------------------------------------------------------------
static int finish_coarse(ddamg_handle* h);
static int build_interpolation(ddamg_handle* h) {
    cudaStream_t st = h->stream;
    const int N = h->N, nc = h->nc;
    const size_t fld = (size_t)12 * h->V;
    DD_CUDA(cudaMemcpyAsync(h->P64, h->V64, sizeof(cplx<double>) * fld * N, cudaMemcpyDeviceToDevice, st));
    DD_CUDA(cudaMemsetAsync(h->d_flag, 0, sizeof(int), st));
    DD_TRY(launch_gram_schmidt(h->g, h->P64, N, h->d_flag, st));
    int flag = 0;
    DD_CUDA(cudaMemcpyAsync(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    DD_CUDA(cudaStreamSynchronize(st));
    if (flag) {
        set_error("test vectors are linearly dependent on an aggregate");
        return DDAMG_ERR_RANK;
    }
    // D_c = P^H D P direction by direction, over the 2N columns of P in chunks (setup_group columns,
    // all 2N when not set), so that the scratch of D P holds a chunk of FP64 fine fields
    const int chunk = (h->p.setup_group > 0 && h->p.setup_group < 2 * N) ? h->p.setup_group : 2 * N;
    Scratch tscr;
    DD_TRY(tscr.ensure(sizeof(cplx<double>) * fld * chunk));
    FineOp<double> op64{h->U64, h->clov64, h->clovinv64};
    int rc = 0;
    for (int dir = 0; dir < 9 && !rc; ++dir)
        for (int col0 = 0; col0 < 2 * N && !rc; col0 += chunk) {
            const int ncols = std::min(chunk, 2 * N - col0);
            rc = launch_assemble_T(h->g, op64, h->P64, N, dir, col0, ncols, tscr.as<cplx<double>>(), st);
            if (!rc)
                rc = launch_block_project(h->g, h->P64, N, tscr.as<cplx<double>>(), col0, ncols, h->d_sites + (size_t)dir * h->Vb,
                                          h->nsites[dir], h->B64 + (size_t)dir * nc * nc * 2, (size_t)9 * nc * nc, st);
        }
    DD_CUDA(cudaStreamSynchronize(st));
    tscr.release();
    if (rc) return rc;
    return finish_coarse(h);
}

// even-site inverses of D_c and the V-cycle-precision copies of P, D_c, D_ee^{-1}
static int finish_coarse(ddamg_handle* h) {
    cudaStream_t st = h->stream;
    const int N = h->N, nc = h->nc;
    const size_t fld = (size_t)12 * h->V;
    int flag = 0;
    DD_CUDA(cudaMemsetAsync(h->d_flag, 0, sizeof(int), st));
    DD_TRY(launch_coarse_invert(h->B64, h->Dinv64, h->NB, nc, h->d_flag, st));
    DD_CUDA(cudaMemcpyAsync(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    DD_CUDA(cudaStreamSynchronize(st));
    if (flag) {
        set_error("singular diagonal block of the coarse operator");
        return DDAMG_ERR_RANK;
    }
    if (h->half()) {
        DD_TRY(convert_to_half(reinterpret_cast<const double*>(h->P64), h->P16, 2 * fld * N, st));
        DD_TRY(pack_coarse_tc(h->B64, h->Dinv64, h->Bh, h->Dh, h->NB, nc, st));
    } else if (h->single()) {
        DD_TRY((convert<float, double>(reinterpret_cast<const double*>(h->P64), reinterpret_cast<float*>(h->P32), 2 * fld * N, st)));
        DD_TRY((convert<float, double>(h->B64, h->B32, (size_t)h->NB * 9 * nc * nc * 2, st)));
        DD_TRY((convert<float, double>(h->Dinv64, h->Dinv32, (size_t)(h->NB / 2) * nc * nc * 2, st)));
    }
    DD_CUDA(cudaStreamSynchronize(st));
    ++h->coarse_gen;
    h->ready = true;
    return 0;
}

// D_c(m0 + delta) = D_c(m0) + delta I because P^H P = I (Sec. 3.1): shift the diagonal of B_0
__global__ void shift_coarse_diag_kernel(double* B64, int NB, int nc, double delta) {
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)NB * nc) return;
    int c = (int)(q / nc), i = (int)(q % nc);
    B64[((((size_t)c * 9) * nc + i) * nc + i) * 2] += delta;
}

__global__ void gaussian_fill_kernel(double* out, size_t n, unsigned long long seed) {
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        // splitmix64 of (seed, q) -> two uniforms -> Box-Muller
        unsigned long long z = seed * 0x9E3779B97F4A7C15ull + q * 0xBF58476D1CE4E5B9ull + 0x94D049BB133111EBull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        double u1 = ((z >> 11) + 1.0) * (1.0 / 9007199254740993.0);
        unsigned long long y = z * 0xD6E8FEB86659FD93ull + 0x2545F4914F6CDD1Dull;
        y ^= y >> 32;
        double u2 = (y >> 11) * (1.0 / 9007199254740992.0);
        out[q] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    }
}

// Algorithm 2 (Algorithm 1 with the modified update) on vectors in precision T
static int setup_probe(ddamg_handle* h, double* est_iters, double* sec_per_iter);

template <typename T>
static int run_setup_T(ddamg_handle* h, cplx<T>* v) {
    cudaStream_t st = h->stream;
    const int N = h->N;
    const size_t fld = (size_t)12 * h->V;
    // the vectors are processed in groups of G (each vector's update is independent of the others
    // within a phase-1 step or a setup round), so the work fields hold 2 G fine fields
    const int G = (h->p.setup_group > 0 && h->p.setup_group < N) ? h->p.setup_group : N;
    DD_TRY(h->ws_fine[0].ensure(sizeof(cplx<T>) * fld * G));
    DD_TRY(h->ws_fine[1].ensure(sizeof(cplx<T>) * fld * G));
    cplx<T>* t1 = h->ws_fine[0].as<cplx<T>>();
    cplx<T>* t2 = h->ws_fine[1].as<cplx<T>>();
    // phase 1: v_j <- M_SAP^(eta) v_j, eta = 1, 2, 3
    for (int eta = 1; eta <= 3; ++eta)
        for (int j0 = 0; j0 < N; j0 += G) {
            const int g = std::min(G, N - j0);
            cplx<T>* vg = v + (size_t)j0 * fld;
            DD_CUDA(cudaMemsetAsync(t1, 0, sizeof(cplx<T>) * fld * g, st));
            DD_TRY(sap<T>(h, vg, t1, g, eta));
            DD_CUDA(cudaMemcpyAsync(vg, t1, sizeof(cplx<T>) * fld * g, cudaMemcpyDeviceToDevice, st));
        }
    KrylovBufs& kb = h->ko;
    DD_TRY(kb.alloc(std::max(N, kb.nrhs), std::max(1, h->p.n_kv)));
    auto to64 = [&]() -> int {
        if (sizeof(T) == 8)
            DD_CUDA(cudaMemcpyAsync(h->V64, v, sizeof(cplx<T>) * fld * N, cudaMemcpyDeviceToDevice, st));
        else
            DD_TRY((convert<double, T>(reinterpret_cast<const T*>(v), reinterpret_cast<double*>(h->V64), 2 * fld * N, st)));
        return 0;
    };
    // n_inv_auto_rhs: before every round after the first, a probe estimates the iterations per
    // solve with the current interpolation; stop once the last round saved less solve time over
    // n_inv_auto_rhs solves than it cost (P, D_c then stay those just built from the vectors)
    const int auto_rhs = h->p.n_inv_auto_rhs;
    double prev_est = -1.0, round_sec = 0.0;
    bool stopped = false;
    h->setup_rounds = 0;
    h->setup_est_iters.clear();
    for (int it = 0; it < h->p.n_inv; ++it) {
        const auto t_round = std::chrono::steady_clock::now();
        DD_TRY(to64());
        DD_TRY(build_interpolation(h));
        if (auto_rhs > 0) {
            double est = 0, sec_it = 0;
            const auto t_probe = std::chrono::steady_clock::now();
            DD_TRY(setup_probe(h, &est, &sec_it));
            h->setup_est_iters.push_back(est);
            if (prev_est > 0 && (double)auto_rhs * (prev_est - est) * sec_it < round_sec) {
                stopped = true;
                break;
            }
            prev_est = est;
            round_sec = -std::chrono::duration<double>(std::chrono::steady_clock::now() - t_probe).count();
        }
        for (int j0 = 0; j0 < N; j0 += G) {
            const int g = std::min(G, N - j0);
            cplx<T>* vg = v + (size_t)j0 * fld;
            if (h->p.setup_update == DDAMG_SETUP_IDSETUP) {
                // Algorithm 1: v_j <- C v_j
                DD_TRY(vcycle<T>(h, vg, t2, g, 0));
                DD_CUDA(cudaMemcpyAsync(vg, t2, sizeof(cplx<T>) * fld * g, cudaMemcpyDeviceToDevice, st));
            } else {
                // Algorithm 2: v_j <- v_j + C (v_j - D v_j)
                DD_TRY((dslash<T, T>(h, vg, vg, t1, g)));
                DD_TRY(vcycle<T>(h, t1, t2, g, 0));
                DD_TRY((lincomb<T, T>(vg, fld, 1.0, t2, 0, fld, 1, kb.ones, g, fld, g, nullptr, st)));
            }
        }
        // v_j <- v_j / ||v_j||
        DD_TRY((multidot<T, T>(v, 0, fld, 1, v, fld, fld, N, kb.nrm, 1, kb.dscr, st)));
        std::vector<cplx<double>> nn(N);
        DD_CUDA(cudaMemcpyAsync(nn.data(), kb.nrm, sizeof(cplx<double>) * N, cudaMemcpyDeviceToHost, st));
        DD_CUDA(cudaStreamSynchronize(st));
        for (int j = 0; j < N; ++j) {
            double nv = std::sqrt(nn[j].re);
            if (!(nv > 0) || !(nv == nv)) {
                set_error("setup produced a zero or non-finite test vector");
                return DDAMG_ERR_NONFINITE;
            }
            nn[j] = mk(1.0 / nv, 0.0);
        }
        DD_CUDA(cudaMemcpyAsync(kb.scale, nn.data(), sizeof(cplx<double>) * N, cudaMemcpyHostToDevice, st));
        DD_TRY((lincomb<T, T>(v, fld, 0.0, v, 0, fld, 1, kb.scale, N, fld, N, nullptr, st)));
        DD_CUDA(cudaStreamSynchronize(st));
        ++h->setup_rounds;
        // the round's cost: rebuild and updates (the probe's own time excluded)
        round_sec += std::chrono::duration<double>(std::chrono::steady_clock::now() - t_round).count();
    }
    if (stopped) return 0;
    DD_TRY(to64());
    if (h->p.rebuild_after_last || h->p.n_inv == 0) DD_TRY(build_interpolation(h));
    return 0;
}

// FP64 test vectors and interpolation, freed after the setup of a lean handle
static int ensure_fp64_vectors(ddamg_handle* h) {
    const size_t n = (size_t)12 * h->V * h->N;
    if (!h->V64) DD_TRY(dalloc_n(&h->V64, n));
    if (!h->P64) DD_TRY(dalloc_n(&h->P64, n));
    return 0;
}
static void lean_release(ddamg_handle* h) {
    if (!(h->p.lean && h->single())) return;
    cudaStreamSynchronize(h->stream);  // cudaFree would wait too; an error here surfaces at the next call
    dfree(h->V64);
    dfree(h->P64);
}

static int run_setup(ddamg_handle* h, const double* v0) {
    cudaStream_t st = h->stream;
    const int N = h->N;
    const size_t fld = (size_t)12 * h->V;
    DD_TRY(ensure_fp64_vectors(h));
    // initial vectors into V64 (internal order)
    if (v0) {
        const void* dv;
        DD_TRY(stage_in(h, h->ws_io[0], v0, sizeof(cplx<double>) * fld * N, &dv));
        DD_TRY((to_internal<double, double>(reinterpret_cast<const cplx<double>*>(dv), h->V64, h->d_lex_of, h->V, 12, N, st)));
    } else {
        gaussian_fill_kernel<<<1216, 256, 0, st>>>(reinterpret_cast<double*>(h->V64), 2 * fld * N, h->p.seed);
        DD_CHECK_LAUNCH();
    }
    int rc;
    if (h->single()) {
        DD_TRY(h->ws_fine[2].ensure(sizeof(cplx<float>) * fld * N));
        cplx<float>* v = h->ws_fine[2].as<cplx<float>>();
        DD_TRY((convert<float, double>(reinterpret_cast<const double*>(h->V64), reinterpret_cast<float*>(v), 2 * fld * N, st)));
        rc = run_setup_T<float>(h, v);
    } else {
        DD_TRY(h->ws_fine[2].ensure(sizeof(cplx<double>) * fld * N));
        cplx<double>* v = h->ws_fine[2].as<cplx<double>>();
        DD_CUDA(cudaMemcpyAsync(v, h->V64, sizeof(cplx<double>) * fld * N, cudaMemcpyDeviceToDevice, st));
        rc = run_setup_T<double>(h, v);
    }
    for (int q = 0; q < 3; ++q) h->ws_fine[q].release();
    if (!rc) lean_release(h);
    return rc;
}

// ---------------------------------------------------------------------------
// the outer solve: FGMRES(n_kv) in FP64, one V-cycle as right preconditioner
// ---------------------------------------------------------------------------
// TV = basis type: double-word FP32 pairs when the V-cycle is FP32 (GB300's FP64
// rate is a small fraction of its FP32 rate), FP64 for the all-FP64 path.
template <typename T>
static int ml_vcycle0(ddamg_handle* h, const cplx<T>* r, cplx<T>* x, int nrhs, int inner_fixed);  // multilevel.inc

template <typename TZ, typename TV>
static int solve_T(ddamg_handle* h, const cplx<double>* b, cplx<double>* x, int nrhs, double tol, bool x0_zero, KrylovResult& R,
                   const int* enabled_host = nullptr, int max_cycles = 0,
                   const std::chrono::steady_clock::time_point* deadline = nullptr) {
    cudaStream_t st = h->stream;
    const size_t fld = (size_t)12 * h->V;
    const int m = h->p.n_kv;
    DD_TRY(h->ws_outer[0].ensure(sizeof(cplx<TV>) * fld * nrhs * (m + 1)));
    DD_TRY(h->ws_outer[1].ensure(sizeof(cplx<TZ>) * fld * nrhs * m));
    DD_TRY(h->ws_outer[2].ensure(sizeof(cplx<TV>) * fld * nrhs));
    DD_TRY(h->ws_outer[3].ensure(sizeof(cplx<TZ>) * fld * nrhs));
    const bool sep = sizeof(TV) != sizeof(double) * 2 || !std::is_same<TV, double>::value;
    if (sep) DD_TRY(h->ws_outer[4].ensure(sizeof(cplx<double>) * fld * nrhs));
    cplx<TZ>* rT = h->ws_outer[3].as<cplx<TZ>>();
    KrylovProblem<double, TV, TZ> P;
    P.n = fld;
    P.nrhs = nrhs;
    P.m = m;
    P.A = [&](const cplx<TZ>* z, cplx<TV>* w) -> int {
        if constexpr (std::is_same<TV, dwf>::value) {
            Prof pr(h, PF_DSLASHDW, (double)h->V * (36.0 * 16 + 72.0 * 8 + nrhs * (12.0 * 8 + 12.0 * 16)));
            return launch_dslash_dw(h->g, h->Udw, h->clovdw, reinterpret_cast<const cplx<float>*>(z), w, true, nrhs, h->stream);
        } else if constexpr (std::is_same<TV, float>::value) {
            return dslash<float, float>(h, reinterpret_cast<const cplx<float>*>(z), nullptr, w, nrhs);
        } else {
            return dslash<double, TZ>(h, z, nullptr, reinterpret_cast<cplx<double>*>(w), nrhs);
        }
    };
    P.Ax = [&](const cplx<double>* z, cplx<double>* w) -> int { return dslash<double, double>(h, z, nullptr, w, nrhs); };
    if constexpr (std::is_same<TV, float>::value) {
        // The true residual b - D x of the refinement cycles without FP64 arithmetic in D:
        // x = x_h + x_l (FP32 pair, ~2^-48), D x_h in double-word arithmetic (exact products,
        // FP64-accurate sums), D x_l in FP32 (its rounding is ~2^-24 of a term already ~2^-24
        // smaller); b - (D x_h + D x_l) is formed in FP64 and rounded once into the FP32 basis.
        P.residual = [&](const cplx<double>* xx, cplx<TV>* v0) -> int {
            cplx<float>* xh = h->ws_outer[2].as<cplx<float>>();
            cplx<float>* xl = h->ws_outer[3].as<cplx<float>>();
            cplx<double>* w = h->ws_outer[4].as<cplx<double>>();
            DD_TRY(split_f64(xx, xh, xl, fld * nrhs, st));
            DD_TRY(dslash_dw(h, xh, w, nrhs));
            DD_TRY((dslash<float, float>(h, xl, nullptr, xh, nrhs)));
            return residual_f32(b, w, xh, reinterpret_cast<cplx<float>*>(v0), fld * nrhs, st);
        };
    }
    P.M = [&](const cplx<TV>* v, cplx<TZ>* z) -> int {
        const cplx<TZ>* r;
        if (std::is_same<TV, dwf>::value) {
            DD_TRY(convert_dw2f(reinterpret_cast<const cplx<dwf>*>(v), reinterpret_cast<float*>(rT), 2 * fld * nrhs, st));
            r = rT;
        } else if (std::is_same<TV, TZ>::value) {
            r = reinterpret_cast<const cplx<TZ>*>(v);
        } else {
            DD_TRY((convert<TZ, double>(reinterpret_cast<const double*>(v), reinterpret_cast<TZ*>(rT), 2 * fld * nrhs, st)));
            r = rT;
        }
        return h->ml_route ? ml_vcycle0<TZ>(h, r, z, nrhs, 0) : vcycle<TZ>(h, r, z, nrhs, 0);
    };
    P.b = b;
    P.x = x;
    P.x0_zero = x0_zero;
    P.tol = tol;
    P.fixed = false;
    P.maxiter = h->p.max_outer;
    P.reorth = true;
    P.Vb = h->ws_outer[0].as<cplx<TV>>();
    P.Zb = h->ws_outer[1].as<cplx<TZ>>();
    P.w = h->ws_outer[2].as<cplx<TV>>();
    P.wB = sep ? h->ws_outer[4].as<cplx<double>>() : reinterpret_cast<cplx<double>*>(P.w);
    P.enabled_host = enabled_host;
    P.max_cycles = max_cycles;
    if (deadline) {
        P.has_deadline = true;
        P.deadline = *deadline;
    }
    if (std::is_same<TV, float>::value) {
        // refinement: FP32 cycles, each ended at cycle_tol relative reduction (or n_kv steps),
        // with the FP64 iterate updated and the FP64 true residual formed between cycles
        P.lean = true;
        P.cycle_tol = h->p.cycle_tol;
    }
    return krylov<double, TV, TZ>(h, h->ko, P, R);
}

// half mode: a coarse-stencil kernel whose bulk copy of the site matrix never completed sets a
// device flag (the kernel gives up after a bounded wait instead of hanging); report it as a CUDA error
static int tc_check(ddamg_handle* h) {
    if (!h->d_tc_err) return 0;
    int f = 0;
    DD_CUDA(cudaMemcpyAsync(&f, h->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DD_CUDA(cudaStreamSynchronize(h->stream));
    if (f) {
        set_error("coarse stencil: a bulk copy of the site matrix did not complete within the kernel's wait limit");
        return DDAMG_ERR_CUDA;
    }
    return 0;
}

// four FGMRES iterations of the handle's solver from the zero guess on a fixed Gaussian right-hand side
// (seeded from params.seed): the residual reduction per iteration rho gives the estimated iterations
// to params.tol, log(tol) / log(rho); sec_per_iter is the probe's wall time per iteration
static int setup_probe(ddamg_handle* h, double* est_iters, double* sec_per_iter) {
    constexpr int kProbeIters = 4;
    const size_t fld = (size_t)12 * h->V;
    Scratch bx;
    DD_TRY(bx.ensure(sizeof(cplx<double>) * fld * 2));
    cplx<double>* b = bx.as<cplx<double>>();
    cplx<double>* x = b + fld;
    gaussian_fill_kernel<<<1216, 256, 0, h->stream>>>(reinterpret_cast<double*>(b), 2 * fld, h->p.seed + 977);
    DD_CHECK_LAUNCH();
    const int saved = h->p.max_outer;
    h->p.max_outer = kProbeIters;
    KrylovResult R;
    DD_CUDA(cudaStreamSynchronize(h->stream));
    const auto t0 = std::chrono::steady_clock::now();
    int rc = !h->single() ? solve_T<double, double>(h, b, x, 1, 1e-300, true, R)
             : h->p.outer == DDAMG_OUTER_REFINE ? solve_T<float, float>(h, b, x, 1, 1e-300, true, R)
                                                : solve_T<float, dwf>(h, b, x, 1, 1e-300, true, R);
    DD_CUDA(cudaStreamSynchronize(h->stream));
    const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    h->p.max_outer = saved;
    if (rc) return rc;
    const double its = std::max<double>(1.0, (double)R.iters[0]);
    const double red = R.resid[0] > 0 ? R.resid[0] : 1e-300;
    const double rho = std::min(0.999999, std::pow(red, 1.0 / its));
    *est_iters = std::log(h->p.tol) / std::log(rho);
    *sec_per_iter = sec / its;
    return 0;
}

static int check_ready(ddamg_handle* h) {
    if (!h) {
        set_error("null handle");
        return DDAMG_ERR_INVALID_ARG;
    }
    if (!h->ready) {
        set_error("no interpolation: run ddamg_setup / ddamg_setup_from_vectors first");
        return DDAMG_ERR_NOT_READY;
    }
    return 0;
}

static int create(const ddamg_lattice* lat, const double* U, double m0, double csw, const ddamg_params* prm, ddamg_handle** out) {
    if (!lat || !U || !out) {
        set_error("null argument");
        return DDAMG_ERR_INVALID_ARG;
    }
    *out = nullptr;
    ddamg_params p;
    if (prm) p = *prm;
    else ddamg_default_params(&p);
    for (int m = 0; m < 4; ++m) {
        int L = lat->dims[m], b = p.block[m];
        if (L <= 0 || b <= 0 || (b & 1) || L % b || ((L / b) & 1)) {
            set_error("every extent must be divisible by an even block extent into an even number (>= 2) of blocks");
            return DDAMG_ERR_INVALID_ARG;
        }
    }
    if (p.n_vec < 1 || p.n_vec > 32 || p.nu < 0 || p.mr_steps < 0 || p.n_kv < 1 || p.n_kv > 64 || p.coarse_restart < 1 ||
        p.coarse_restart > 64 ||
        p.precision < DDAMG_PREC_DOUBLE || p.precision > DDAMG_PREC_HALF || p.n_inv < 0 ||
        (p.outer != DDAMG_OUTER_DW && p.outer != DDAMG_OUTER_REFINE) ||
        (p.outer == DDAMG_OUTER_REFINE && !(p.cycle_tol > 0 && p.cycle_tol < 1)) ||
        (p.setup_update != DDAMG_SETUP_DDALPHA && p.setup_update != DDAMG_SETUP_IDSETUP)) {
        set_error("parameter out of range (1 <= n_vec <= 32, 1 <= n_kv <= 64, 1 <= coarse_restart <= 64, nu, mr_steps, n_inv >= 0, "
                  "outer in {0, 1}, 0 < cycle_tol < 1, setup_update in {0, 1})");
        return DDAMG_ERR_INVALID_ARG;
    }
    long long vb = (long long)p.block[0] * p.block[1] * p.block[2] * p.block[3];
    if (vb > 1024) {
        set_error("block volume above 1024 sites");
        return DDAMG_ERR_INVALID_ARG;
    }
    ddamg_handle* h = new ddamg_handle();
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        set_error("cudaGetDevice failed");
        return DDAMG_ERR_CUDA;
    }
    for (int m = 0; m < 4; ++m) {
        h->L[m] = lat->dims[m];
        h->b[m] = p.block[m];
    }
    h->p = p;
    h->m0 = m0;
    h->csw = csw;
    h->N = p.n_vec;
    h->nc = 2 * p.n_vec;
    int rc = 0;
    auto fail = [&](int code) {
        ddamg_destroy(h);
        return code;
    };
    if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaStreamCreate failed");
        delete h;
        return DDAMG_ERR_CUDA;
    }
    h->stream = h->own_stream;
    if ((rc = upload_gammas())) return fail(rc);
    if ((rc = build_geometry(h))) return fail(rc);
    const size_t V = h->V, N = h->N, nc = h->nc;
    if ((rc = dalloc_n(&h->U64, V * 36)) || (rc = dalloc_n(&h->clov64, V * 72)) || (rc = dalloc_n(&h->clovinv64, V * 72)) ||
        (rc = dalloc_n(&h->V64, V * 12 * N)) || (rc = dalloc_n(&h->P64, V * 12 * N)) ||
        (rc = dalloc_n(&h->B64, (size_t)h->NB * 9 * nc * nc * 2)) || (rc = dalloc_n(&h->Dinv64, (size_t)(h->NB / 2) * nc * nc * 2)) ||
        (rc = dalloc_n(&h->d_flag, 1)))
        return fail(rc);
    if (h->single()) {
        if ((rc = dalloc_n(&h->U32, V * 36)) || (rc = dalloc_n(&h->clov32, V * 72)) || (rc = dalloc_n(&h->clovinv32, V * 72)) ||
            (rc = dalloc_n(&h->Udw, V * 36)) || (rc = dalloc_n(&h->clovdw, V * 72)) || (rc = dalloc_n(&h->Uaos, V * 20)) ||
            (rc = dalloc_n(&h->clov_aos, V * 18)) || (rc = dalloc_n(&h->clovinv_aos, V * 18)))
            return fail(rc);
    }
    if (h->half()) {
        int Mt, Kta, Kth, Ktd;
        if (tc_dims((int)nc, &Mt, &Kta, &Kth, &Ktd)) {
            set_error("half precision needs n_vec divisible by 4");
            return fail(DDAMG_ERR_INVALID_ARG);
        }
        if ((rc = dalloc_n(&h->Bh, (size_t)h->NB * Mt * Kta * 32)) || (rc = dalloc_n(&h->Dh, (size_t)(h->NB / 2) * Mt * Ktd * 32)) ||
            (rc = dalloc_n(&h->P16, V * 12 * N)))
            return fail(rc);
        if ((rc = dalloc_n(&h->d_tc_err, 1))) return fail(rc);
        if (cudaMemset(h->d_tc_err, 0, sizeof(int)) != cudaSuccess) return fail(DDAMG_ERR_CUDA);
        h->tc = CoarseTC{h->Bh, h->Dh, h->d_bnbr, h->NB, (int)nc, Mt, Kta, Kth, Ktd, h->d_tc_err};
        if (p.smoother_fp16 &&
            ((rc = dalloc_n(&h->Uaos16, V * 12)) || (rc = dalloc_n(&h->clov_aos16, V * 9)) || (rc = dalloc_n(&h->clovinv_aos16, V * 9))))
            return fail(rc);
    } else if (h->single()) {
        if ((rc = dalloc_n(&h->P32, V * 12 * N)) || (rc = dalloc_n(&h->B32, (size_t)h->NB * 9 * nc * nc * 2)) ||
            (rc = dalloc_n(&h->Dinv32, (size_t)(h->NB / 2) * nc * nc * 2)))
            return fail(rc);
    }
    // gauge field -> internal order, clover term and inverses
    const void* dU;
    if ((rc = stage_in(h, h->ws_io[0], U, sizeof(cplx<double>) * V * 36, &dU))) return fail(rc);
    if ((rc = gauge_to_internal(reinterpret_cast<const cplx<double>*>(dU), h->U64, h->d_lex_of, h->V, h->stream))) return fail(rc);
    if ((rc = launch_clover(h->g, h->U64, m0, csw, h->clov64, h->clovinv64, h->stream))) return fail(rc);
    if (h->single()) {
        if ((rc = convert<float, double>(reinterpret_cast<const double*>(h->U64), reinterpret_cast<float*>(h->U32), V * 72, h->stream)) ||
            (rc = convert<float, double>(h->clov64, h->clov32, V * 72, h->stream)) ||
            (rc = convert<float, double>(h->clovinv64, h->clovinv32, V * 72, h->stream)) ||
            (rc = launch_to_dw(reinterpret_cast<const double*>(h->U64), reinterpret_cast<float2*>(h->Udw), V * 72, h->stream)) ||
            (rc = launch_to_dw(h->clov64, h->clovdw, V * 72, h->stream)) || (rc = links_to_aos(h->U32, h->Uaos, h->V, h->stream)) ||
            (rc = clover_to_aos(h->clov32, h->clov_aos, h->V, h->stream)) ||
            (rc = clover_to_aos(h->clovinv32, h->clovinv_aos, h->V, h->stream)))
            return fail(rc);
        if (h->half() && h->p.smoother_fp16 && ((rc = links_to_aos16(h->U32, h->Uaos16, h->V, h->stream)) ||
                          (rc = clover_to_aos16(h->clov32, h->clov_aos16, h->V, h->stream)) ||
                          (rc = clover_to_aos16(h->clovinv32, h->clovinv_aos16, h->V, h->stream))))
            return fail(rc);
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        set_error(std::string("setup kernels: ") + cudaGetErrorString(cudaGetLastError()));
        return fail(DDAMG_ERR_CUDA);
    }
    h->ws_io[0].release();
    *out = h;
    return 0;
}

template <typename T>
static int fine_in(ddamg_handle* h, const double* in, int nrhs, Scratch& tmp, cplx<T>* dst) {
    const size_t fld = (size_t)12 * h->V;
    const void* dv;
    DD_TRY(stage_in(h, h->ws_io[0], in, sizeof(cplx<double>) * fld * nrhs, &dv));
    (void)tmp;
    return to_internal<T, double>(reinterpret_cast<const cplx<double>*>(dv), dst, h->d_lex_of, h->V, 12, nrhs, h->stream);
}
template <typename T>
static int fine_out(ddamg_handle* h, const cplx<T>* src, double* out, int nrhs) {
    const size_t fld = (size_t)12 * h->V;
    void* dv;
    bool host;
    DD_TRY(stage_out_ptr(h->ws_io[1], out, sizeof(cplx<double>) * fld * nrhs, &dv, &host));
    DD_TRY((from_internal<double, T>(src, reinterpret_cast<cplx<double>*>(dv), h->d_lex_of, h->V, 12, nrhs, h->stream)));
    return finish_out(h, out, dv, sizeof(cplx<double>) * fld * nrhs, host);
}
template <typename T>
static int coarse_in(ddamg_handle* h, const double* in, int nrhs, cplx<T>* dst) {
    const size_t n = (size_t)h->NB * h->nc;
    const void* dv;
    DD_TRY(stage_in(h, h->ws_io[0], in, sizeof(cplx<double>) * n * nrhs, &dv));
    return coarse_perm<T, double>(reinterpret_cast<const cplx<double>*>(dv), dst, h->d_clex_of, h->NB, h->nc, nrhs, 1, h->stream);
}
template <typename T>
static int coarse_out(ddamg_handle* h, const cplx<T>* src, double* out, int nrhs) {
    const size_t n = (size_t)h->NB * h->nc;
    void* dv;
    bool host;
    DD_TRY(stage_out_ptr(h->ws_io[1], out, sizeof(cplx<double>) * n * nrhs, &dv, &host));
    DD_TRY((coarse_perm<double, T>(src, reinterpret_cast<cplx<double>*>(dv), h->d_clex_of, h->NB, h->nc, nrhs, 0, h->stream)));
    return finish_out(h, out, dv, sizeof(cplx<double>) * n * nrhs, host);
}

static void ml_release(ddamg_handle* h);  // multilevel.inc

}  // namespace ddamg

// ===========================================================================
// extern "C" entry points
// ===========================================================================
extern "C" {

void ddamg_default_params(ddamg_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->n_inv = 6;
    p->n_vec = 20;
    for (int m = 0; m < 4; ++m) p->block[m] = 4;
    p->coarse_tol = 5e-2;
    p->coarse_restart = 30;
    p->coarse_maxiter = 1000;
    p->n_kv = 25;
    p->tol = 1e-10;
    p->max_outer = 10000;
    p->nu = 2;
    p->mr_steps = 4;
    p->precision = DDAMG_PREC_SINGLE;
    p->rebuild_after_last = 1;
    p->seed = 1;
    p->time_limit_s = 0;
    p->outer = DDAMG_OUTER_REFINE;
    p->cycle_tol = 1e-5;
    p->setup_update = DDAMG_SETUP_DDALPHA;
    p->smoother_fp16 = 1;
    p->setup_group = 0;
    p->n_inv_auto_rhs = 0;
    p->lean = 0;
}

const char* ddamg_error_string(int s) {
    switch (s) {
        case DDAMG_OK: return "ok";
        case DDAMG_ERR_INVALID_ARG: return "invalid argument";
        case DDAMG_ERR_OOM: return "out of device memory";
        case DDAMG_ERR_CUDA: return "CUDA error";
        case DDAMG_ERR_NOT_CONVERGED: return "not converged";
        case DDAMG_ERR_NONFINITE: return "non-finite value";
        case DDAMG_ERR_TIMEOUT: return "time limit exceeded";
        case DDAMG_ERR_NOT_READY: return "setup missing";
        case DDAMG_ERR_RANK: return "rank-deficient aggregate";
        default: return "unknown status";
    }
}

const char* ddamg_last_error(void) { return g_err.c_str(); }

long long ddamg_launch_count(void) { return (long long)g_launches.load(); }

void ddamg_debug_fail_allocs(int n) { g_fail_allocs = n; }

int ddamg_create(const ddamg_lattice* lat, const double* U, double m0, double c_sw, const ddamg_params* params, ddamg_handle** out) {
    return create(lat, U, m0, c_sw, params, out);
}

int ddamg_run_setup(ddamg_handle* h, const double* v0) {
    if (!h) return DDAMG_ERR_INVALID_ARG;
    return run_setup(h, v0);
}

int ddamg_setup(const ddamg_lattice* lat, const double* U, double m0, double c_sw, const ddamg_params* params, ddamg_handle** out) {
    ddamg_handle* h = nullptr;
    int rc = create(lat, U, m0, c_sw, params, &h);
    if (rc) return rc;
    rc = run_setup(h, nullptr);
    if (rc) {
        ddamg_destroy(h);
        return rc;
    }
    *out = h;
    return 0;
}

int ddamg_setup_from_vectors(ddamg_handle* h, const double* V, int N) {
    if (!h || !V || N != h->N) {
        set_error("ddamg_setup_from_vectors: null argument or N differs from params.n_vec");
        return DDAMG_ERR_INVALID_ARG;
    }
    const size_t fld = (size_t)12 * h->V;
    const void* dv;
    DD_TRY(ensure_fp64_vectors(h));
    DD_TRY(stage_in(h, h->ws_io[0], V, sizeof(cplx<double>) * fld * N, &dv));
    DD_TRY((to_internal<double, double>(reinterpret_cast<const cplx<double>*>(dv), h->V64, h->d_lex_of, h->V, 12, N, h->stream)));
    DD_TRY(build_interpolation(h));
    lean_release(h);
    return 0;
}

int ddamg_setup_report(const ddamg_handle* h, int* rounds, double* est_iterations, int max) {
    if (!h || !rounds) return DDAMG_ERR_INVALID_ARG;
    *rounds = h->setup_rounds;
    const int n = (int)h->setup_est_iters.size();
    for (int k = 0; k < n && k < max && est_iterations; ++k) est_iterations[k] = h->setup_est_iters[k];
    return n;
}

int ddamg_get_vectors(const ddamg_handle* hc, double* V) {
    ddamg_handle* h = const_cast<ddamg_handle*>(hc);
    if (!h || !V) return DDAMG_ERR_INVALID_ARG;
    if (!h->V64) {
        set_error("ddamg_get_vectors: the handle is lean (params.lean): its FP64 test vectors were freed after the setup");
        return DDAMG_ERR_NOT_READY;
    }
    return fine_out<double>(h, h->V64, V, h->N);
}

// zero_guess: z is output only and the initial guess is 0 (the paper's choice): z is neither read
// nor staged in, and no initial residual product is formed.
static int solve_common(ddamg_handle* h, const double* b, double* z, int nrhs, double tol, ddamg_stats* st, bool zero_guess = false) {
    DD_TRY(check_ready(h));
    if (!b || !z || nrhs < 1) {
        set_error("solve: null pointer or n_rhs < 1");
        return DDAMG_ERR_INVALID_ARG;
    }
    auto t0 = std::chrono::steady_clock::now();
    const bool limited = h->p.time_limit_s > 0;
    const auto deadline = t0 + std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                                   std::chrono::duration<double>(limited ? h->p.time_limit_s : 0.0));
    if (tol <= 0) tol = h->p.tol;
    const size_t fld = (size_t)12 * h->V;
    DD_TRY(h->ws_io[2].ensure(sizeof(cplx<double>) * fld * nrhs * 2));
    cplx<double>* bi = h->ws_io[2].as<cplx<double>>();
    cplx<double>* xi = bi + fld * nrhs;
    DD_TRY(fine_in<double>(h, b, nrhs, h->ws_io[0], bi));
    if (!zero_guess) DD_TRY(fine_in<double>(h, z, nrhs, h->ws_io[0], xi));
    h->coarse_iters = 0;
    h->vcycles = 0;
    h->coarse_seconds = 0;
    // a zero initial guess (the paper's choice) needs no initial residual product
    bool x0_zero = zero_guess;
    if (!zero_guess) {
        DD_TRY(h->ko.alloc(std::max(nrhs, h->ko.nrhs), std::max(1, h->p.n_kv)));
        DD_TRY((multidot<double, double>(xi, 0, fld, 1, xi, fld, fld, nrhs, h->ko.nrm, 1, h->ko.dscr, h->stream)));
        std::vector<cplx<double>> zn(nrhs);
        DD_CUDA(cudaMemcpyAsync(zn.data(), h->ko.nrm, sizeof(cplx<double>) * nrhs, cudaMemcpyDeviceToHost, h->stream));
        DD_CUDA(cudaStreamSynchronize(h->stream));
        x0_zero = true;
        for (int r = 0; r < nrhs; ++r)
            if (zn[r].re != 0.0) x0_zero = false;
    }
    KrylovResult R;
    const auto* dl = limited ? &deadline : nullptr;
    int rc = !h->single() ? solve_T<double, double>(h, bi, xi, nrhs, tol, x0_zero, R, nullptr, 0, dl)
             : h->p.outer == DDAMG_OUTER_REFINE ? solve_T<float, float>(h, bi, xi, nrhs, tol, x0_zero, R, nullptr, 0, dl)
                                                : solve_T<float, dwf>(h, bi, xi, nrhs, tol, x0_zero, R, nullptr, 0, dl);
    if (rc) return rc;
    DD_TRY(fine_out<double>(h, xi, z, nrhs));
    DD_TRY(tc_check(h));
    double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int status = 0;
    const int unconverged = R.timed_out ? DDAMG_ERR_TIMEOUT : DDAMG_ERR_NOT_CONVERGED;
    if (R.nonfinite) status = DDAMG_ERR_NONFINITE;
    else {
        for (int r = 0; r < nrhs; ++r)
            if (!(R.resid[r] <= tol)) status = unconverged;
    }
    if (st) {
        for (int r = 0; r < nrhs; ++r) {
            st[r].iterations = (int)R.iters[r];
            st[r].restarts = R.restarts;
            st[r].coarse_iterations = h->coarse_iters;
            st[r].vcycles = h->vcycles;
            st[r].rel_residual = R.resid[r];
            st[r].solve_seconds = secs;
            st[r].coarse_seconds = h->coarse_seconds;
            st[r].status = (R.nonfinite ? DDAMG_ERR_NONFINITE : (R.resid[r] <= tol ? 0 : unconverged));
        }
    }
    if (status == DDAMG_ERR_NOT_CONVERGED) set_error("iteration cap reached before the tolerance");
    if (status == DDAMG_ERR_TIMEOUT)
        set_error("time limit of " + std::to_string(h->p.time_limit_s) + " s reached before the tolerance (z holds the last iterate)");
    if (status == DDAMG_ERR_NONFINITE) set_error("non-finite residual");
    return status;
}

int ddamg_solve(ddamg_handle* h, const double* b, double* z, double tol, ddamg_stats* st) { return solve_common(h, b, z, 1, tol, st); }

int ddamg_solve_batch(ddamg_handle* h, const double* b, double* z, int n_rhs, double tol, ddamg_stats* st) {
    return solve_common(h, b, z, n_rhs, tol, st);
}

int ddamg_solve_batch_zero_guess(ddamg_handle* h, const double* b, double* z, int n_rhs, double tol, ddamg_stats* st) {
    return solve_common(h, b, z, n_rhs, tol, st, true);
}

// ---------------------------------------------------------------------------
// continuous batching: right-hand sides enter and leave a fixed set of slots between
// outer cycles; every cycle is one lock-step pass of the outer solver over the running slots
// ---------------------------------------------------------------------------
static int slot_check(ddamg_handle* h, int slot) {
    if (!h || h->n_slots == 0) {
        set_error("no slots: call ddamg_slots_open first");
        return DDAMG_ERR_INVALID_ARG;
    }
    if (slot < 0 || slot >= h->n_slots) {
        set_error("slot index out of range");
        return DDAMG_ERR_INVALID_ARG;
    }
    return 0;
}

int ddamg_slots_close(ddamg_handle* h) {
    if (!h) return DDAMG_ERR_INVALID_ARG;
    dfree(h->slot_b);
    dfree(h->slot_x);
    h->n_slots = 0;
    h->slot_state.clear();
    h->slot_iters.clear();
    h->slot_resid.clear();
    return 0;
}

int ddamg_slots_open(ddamg_handle* h, int n_slots) {
    DD_TRY(check_ready(h));
    if (n_slots < 1) {
        set_error("slots_open: n_slots < 1");
        return DDAMG_ERR_INVALID_ARG;
    }
    DD_TRY(ddamg_slots_close(h));
    const size_t n = (size_t)12 * h->V * n_slots;
    DD_TRY(dalloc_n(&h->slot_b, n));
    DD_TRY(dalloc_n(&h->slot_x, n));
    DD_CUDA(cudaMemsetAsync(h->slot_b, 0, sizeof(cplx<double>) * n, h->stream));
    DD_CUDA(cudaMemsetAsync(h->slot_x, 0, sizeof(cplx<double>) * n, h->stream));
    DD_CUDA(cudaStreamSynchronize(h->stream));
    h->n_slots = n_slots;
    h->slot_state.assign(n_slots, DDAMG_SLOT_FREE);
    h->slot_iters.assign(n_slots, 0);
    h->slot_resid.assign(n_slots, 0.0);
    return 0;
}

int ddamg_slot_put(ddamg_handle* h, int slot, const double* b) {
    DD_TRY(slot_check(h, slot));
    if (!b) return DDAMG_ERR_INVALID_ARG;
    if (h->slot_state[slot] != DDAMG_SLOT_FREE) {
        set_error("slot_put: the slot is not free (take its result first)");
        return DDAMG_ERR_INVALID_ARG;
    }
    const size_t fld = (size_t)12 * h->V;
    DD_TRY(fine_in<double>(h, b, 1, h->ws_io[0], h->slot_b + fld * slot));
    DD_CUDA(cudaMemsetAsync(h->slot_x + fld * slot, 0, sizeof(cplx<double>) * fld, h->stream));
    DD_CUDA(cudaStreamSynchronize(h->stream));
    h->slot_state[slot] = DDAMG_SLOT_RUNNING;
    h->slot_iters[slot] = 0;
    h->slot_resid[slot] = 1.0;
    return 0;
}

int ddamg_slots_cycle(ddamg_handle* h, int* state, ddamg_stats* st) {
    DD_TRY(check_ready(h));
    if (h->n_slots == 0) return slot_check(h, 0);
    const int S = h->n_slots;
    std::vector<int> en(S);
    int nrun = 0;
    for (int r = 0; r < S; ++r) nrun += (en[r] = h->slot_state[r] == DDAMG_SLOT_RUNNING);
    h->coarse_iters = 0;
    h->vcycles = 0;
    h->coarse_seconds = 0;
    auto t0 = std::chrono::steady_clock::now();
    if (nrun > 0) {
        KrylovResult R;
        const double tol = h->p.tol;
        int rc = !h->single() ? solve_T<double, double>(h, h->slot_b, h->slot_x, S, tol, false, R, en.data(), 1)
                 : h->p.outer == DDAMG_OUTER_REFINE ? solve_T<float, float>(h, h->slot_b, h->slot_x, S, tol, false, R, en.data(), 1)
                                                    : solve_T<float, dwf>(h, h->slot_b, h->slot_x, S, tol, false, R, en.data(), 1);
        if (rc) return rc;
        for (int r = 0; r < S; ++r) {
            if (!en[r]) continue;
            h->slot_resid[r] = R.resid[r];
            if (R.flags[r] & 2) {
                h->slot_state[r] = DDAMG_SLOT_FAILED;
            } else if (!R.start_active[r]) {
                h->slot_state[r] = DDAMG_SLOT_DONE;  // certified by the true residual at the start of this cycle
            } else {
                h->slot_iters[r] += R.iters[r];
                if (h->slot_iters[r] >= h->p.max_outer) h->slot_state[r] = DDAMG_SLOT_FAILED;
            }
        }
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int r = 0; r < S; ++r) {
        if (state) state[r] = h->slot_state[r];
        if (st) {
            st[r].iterations = (int)h->slot_iters[r];
            st[r].restarts = 0;
            st[r].coarse_iterations = h->coarse_iters;
            st[r].vcycles = h->vcycles;
            st[r].rel_residual = h->slot_resid[r];
            st[r].solve_seconds = secs;
            st[r].coarse_seconds = h->coarse_seconds;
            st[r].status = h->slot_state[r] == DDAMG_SLOT_FAILED
                               ? (h->slot_iters[r] >= h->p.max_outer ? DDAMG_ERR_NOT_CONVERGED : DDAMG_ERR_NONFINITE)
                               : DDAMG_OK;
        }
    }
    return 0;
}

int ddamg_slot_take(ddamg_handle* h, int slot, double* z) {
    DD_TRY(slot_check(h, slot));
    if (!z) return DDAMG_ERR_INVALID_ARG;
    if (h->slot_state[slot] != DDAMG_SLOT_DONE && h->slot_state[slot] != DDAMG_SLOT_FAILED) {
        set_error("slot_take: the slot has no finished result");
        return DDAMG_ERR_INVALID_ARG;
    }
    const size_t fld = (size_t)12 * h->V;
    DD_TRY(fine_out<double>(h, h->slot_x + fld * slot, z, 1));
    h->slot_state[slot] = DDAMG_SLOT_FREE;
    return 0;
}

int ddamg_apply_D(ddamg_handle* h, const double* in, double* out, int n_rhs) {
    if (!h || !in || !out || n_rhs < 1) return DDAMG_ERR_INVALID_ARG;
    const size_t fld = (size_t)12 * h->V;
    DD_TRY(h->ws_fine[4].ensure(sizeof(cplx<double>) * fld * n_rhs * 2));
    cplx<double>* a = h->ws_fine[4].as<cplx<double>>();
    cplx<double>* o = a + fld * n_rhs;
    DD_TRY(fine_in<double>(h, in, n_rhs, h->ws_io[0], a));
    DD_TRY((dslash<double, double>(h, a, nullptr, o, n_rhs)));
    return fine_out<double>(h, o, out, n_rhs);
}

int ddamg_apply_D_f32(ddamg_handle* h, const float* in, float* out, int n_rhs) {
    if (!h || !in || !out || n_rhs < 1) return DDAMG_ERR_INVALID_ARG;
    if (!h->single()) {
        set_error("ddamg_apply_D_f32 needs a handle in single or half precision");
        return DDAMG_ERR_INVALID_ARG;
    }
    const size_t fld = (size_t)12 * h->V;
    DD_TRY(h->ws_fine[4].ensure(sizeof(cplx<float>) * fld * n_rhs * 2));
    cplx<float>* a = h->ws_fine[4].as<cplx<float>>();
    cplx<float>* o = a + fld * n_rhs;
    const void* dv;
    DD_TRY(stage_in(h, h->ws_io[0], in, sizeof(cplx<float>) * fld * n_rhs, &dv));
    DD_TRY((to_internal<float, float>(reinterpret_cast<const cplx<float>*>(dv), a, h->d_lex_of, h->V, 12, n_rhs, h->stream)));
    DD_TRY((dslash<float, float>(h, a, nullptr, o, n_rhs)));
    void* dout;
    bool host;
    DD_TRY(stage_out_ptr(h->ws_io[1], out, sizeof(cplx<float>) * fld * n_rhs, &dout, &host));
    DD_TRY((from_internal<float, float>(o, reinterpret_cast<cplx<float>*>(dout), h->d_lex_of, h->V, 12, n_rhs, h->stream)));
    return finish_out(h, out, dout, sizeof(cplx<float>) * fld * n_rhs, host);
}

}  // extern "C"

extern "C" {
int ddamg_apply_D_mixed(ddamg_handle* h, const float* in, double* out, int n_rhs) {
    if (!h || !in || !out || n_rhs < 1) return DDAMG_ERR_INVALID_ARG;
    if (!h->single()) {
        set_error("ddamg_apply_D_mixed needs a handle in single or half precision");
        return DDAMG_ERR_INVALID_ARG;
    }
    const size_t fld = (size_t)12 * h->V;
    DD_TRY(h->ws_fine[4].ensure((sizeof(cplx<float>) + sizeof(cplx<double>)) * fld * n_rhs));
    cplx<float>* a = h->ws_fine[4].as<cplx<float>>();
    cplx<double>* o = reinterpret_cast<cplx<double>*>(a + fld * n_rhs);
    const void* dv;
    DD_TRY(stage_in(h, h->ws_io[0], in, sizeof(cplx<float>) * fld * n_rhs, &dv));
    DD_TRY((to_internal<float, float>(reinterpret_cast<const cplx<float>*>(dv), a, h->d_lex_of, h->V, 12, n_rhs, h->stream)));
    DD_TRY(dslash_dw(h, a, o, n_rhs));
    return fine_out<double>(h, o, out, n_rhs);
}
}  // extern "C"

template <typename T>
static int apply_sap_T(ddamg_handle* h, const double* in, double* out, int n_rhs, int nu) {
    const size_t fld = (size_t)12 * h->V;
    DD_TRY(h->ws_fine[4].ensure(sizeof(cplx<T>) * fld * n_rhs * 2));
    cplx<T>* a = h->ws_fine[4].as<cplx<T>>();
    cplx<T>* o = a + fld * n_rhs;
    DD_TRY(fine_in<T>(h, in, n_rhs, h->ws_io[0], a));
    DD_CUDA(cudaMemsetAsync(o, 0, sizeof(cplx<T>) * fld * n_rhs, h->stream));
    DD_TRY(sap<T>(h, a, o, n_rhs, nu));
    return fine_out<T>(h, o, out, n_rhs);
}

extern "C" {
int ddamg_apply_sap(ddamg_handle* h, const double* in, double* out, int n_rhs, int nu) {
    if (!h || !in || !out || n_rhs < 1 || nu < 0) return DDAMG_ERR_INVALID_ARG;
    return h->single() ? apply_sap_T<float>(h, in, out, n_rhs, nu) : apply_sap_T<double>(h, in, out, n_rhs, nu);
}

}  // extern "C"

template <typename T>
static int restrict_T(ddamg_handle* h, const double* in, double* out, int n_rhs) {
    const size_t fld = (size_t)12 * h->V, cn = (size_t)h->NB * h->nc;
    DD_TRY(h->ws_fine[4].ensure(sizeof(cplx<T>) * (fld + cn) * n_rhs));
    cplx<T>* a = h->ws_fine[4].as<cplx<T>>();
    cplx<T>* o = a + fld * n_rhs;
    DD_TRY(fine_in<T>(h, in, n_rhs, h->ws_io[0], a));
    DD_TRY(restrict_<T>(h, a, o, n_rhs));
    DD_TRY(coarse_out<T>(h, o, out, n_rhs));
    return tc_check(h);
}

extern "C" {
int ddamg_restrict(ddamg_handle* h, const double* in, double* out, int n_rhs) {
    DD_TRY(check_ready(h));
    if (!in || !out || n_rhs < 1) return DDAMG_ERR_INVALID_ARG;
    return h->single() ? restrict_T<float>(h, in, out, n_rhs) : restrict_T<double>(h, in, out, n_rhs);
}

}  // extern "C"

template <typename T>
static int prolong_T(ddamg_handle* h, const double* in, double* out, int n_rhs) {
    const size_t fld = (size_t)12 * h->V, cn = (size_t)h->NB * h->nc;
    DD_TRY(h->ws_fine[4].ensure(sizeof(cplx<T>) * (fld + cn) * n_rhs));
    cplx<T>* a = h->ws_fine[4].as<cplx<T>>();
    cplx<T>* o = a + cn * n_rhs;
    DD_TRY(coarse_in<T>(h, in, n_rhs, a));
    DD_TRY(prolong_<T>(h, a, o, n_rhs));
    return fine_out<T>(h, o, out, n_rhs);
}

extern "C" {
int ddamg_prolong(ddamg_handle* h, const double* in, double* out, int n_rhs) {
    DD_TRY(check_ready(h));
    if (!in || !out || n_rhs < 1) return DDAMG_ERR_INVALID_ARG;
    return h->single() ? prolong_T<float>(h, in, out, n_rhs) : prolong_T<double>(h, in, out, n_rhs);
}

}  // extern "C"

template <typename T>
static int apply_Dc_T(ddamg_handle* h, const double* in, double* out, int n_rhs) {
    const size_t cn = (size_t)h->NB * h->nc;
    DD_TRY(h->ws_fine[4].ensure(sizeof(cplx<T>) * cn * n_rhs * 2));
    cplx<T>* a = h->ws_fine[4].as<cplx<T>>();
    cplx<T>* o = a + cn * n_rhs;
    DD_TRY(coarse_in<T>(h, in, n_rhs, a));
    {
        Prof pr(h, PF_COARSE, (double)h->NB * 9 * h->nc * h->nc * sizeof(cplx<T>));
        DD_TRY(c_full<T>(h, a, o, n_rhs));
    }
    DD_TRY(coarse_out<T>(h, o, out, n_rhs));
    return tc_check(h);
}

namespace ddamg {
// D_c applied to caller-owned device vectors, with the two internal-layout staging
// buffers carved out of caller-provided device scratch: this path allocates nothing.
template <typename T>
static int apply_Dc_scratch_T(ddamg_handle* h, const double* in, double* out, int n_rhs, void* scratch, size_t scratch_bytes) {
    const size_t cn = (size_t)h->NB * h->nc;
    const size_t per_rhs = 2 * cn * sizeof(cplx<T>);
    if (per_rhs * (size_t)n_rhs > scratch_bytes) {
        set_error("ddamg_apply_Dc_noalloc: n_rhs " + std::to_string(n_rhs) + " needs " + std::to_string(per_rhs * n_rhs) +
                  " bytes of scratch, the fixed scratch holds " + std::to_string(scratch_bytes) + " (at most " +
                  std::to_string(scratch_bytes / per_rhs) + " right-hand sides for this handle)");
        return DDAMG_ERR_INVALID_ARG;
    }
    cplx<T>* a = reinterpret_cast<cplx<T>*>(scratch);
    cplx<T>* o = a + cn * n_rhs;
    DD_TRY((coarse_perm<T, double>(reinterpret_cast<const cplx<double>*>(in), a, h->d_clex_of, h->NB, h->nc, n_rhs, 1, h->stream)));
    DD_TRY(c_full<T>(h, a, o, n_rhs));
    return coarse_perm<double, T>(o, reinterpret_cast<cplx<double>*>(out), h->d_clex_of, h->NB, h->nc, n_rhs, 0, h->stream);
}

int handle_device(const ddamg_handle* h) { return h ? h->device : -1; }

int apply_Dc_into_scratch(ddamg_handle* h, const double* in, double* out, int n_rhs, void* scratch, size_t scratch_bytes) {
    DD_TRY(check_ready(h));
    if (!in || !out || n_rhs < 1 || !scratch) {
        set_error("ddamg_apply_Dc_noalloc: null pointer or n_rhs < 1");
        return DDAMG_ERR_INVALID_ARG;
    }
    if (!is_device_ptr(in) || !is_device_ptr(out)) {
        set_error("ddamg_apply_Dc_noalloc: in and out must be device memory (host data would need staging buffers)");
        return DDAMG_ERR_INVALID_ARG;
    }
    return h->single() ? apply_Dc_scratch_T<float>(h, in, out, n_rhs, scratch, scratch_bytes)
                       : apply_Dc_scratch_T<double>(h, in, out, n_rhs, scratch, scratch_bytes);
}
}  // namespace ddamg

extern "C" {
int ddamg_apply_Dc(ddamg_handle* h, const double* in, double* out, int n_rhs) {
    DD_TRY(check_ready(h));
    if (!in || !out || n_rhs < 1) return DDAMG_ERR_INVALID_ARG;
    return h->single() ? apply_Dc_T<float>(h, in, out, n_rhs) : apply_Dc_T<double>(h, in, out, n_rhs);
}

int ddamg_get_coarse_stencil(const ddamg_handle* hc, double* out) {
    ddamg_handle* h = const_cast<ddamg_handle*>(hc);
    DD_TRY(check_ready(h));
    if (!out) return DDAMG_ERR_INVALID_ARG;
    const int nc = h->nc;
    const size_t per = (size_t)9 * nc * nc * 2;
    std::vector<double> tmp(per * h->NB);
    DD_CUDA(cudaMemcpyAsync(tmp.data(), h->B64, sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost, h->stream));
    DD_CUDA(cudaStreamSynchronize(h->stream));
    std::vector<double> res(per * h->NB);
    for (int c = 0; c < h->NB; ++c) {
        int cl = h->h_clex_of[c];
        for (int d = 0; d < 9; ++d)
            for (int col = 0; col < nc; ++col)
                for (int row = 0; row < nc; ++row) {
                    const double* s = &tmp[(((size_t)c * 9 + d) * nc + col) * nc * 2 + (size_t)row * 2];
                    double* dd = &res[(((size_t)cl * 9 + d) * nc + row) * nc * 2 + (size_t)col * 2];
                    dd[0] = s[0];
                    dd[1] = s[1];
                }
    }
    if (is_device_ptr(out)) {
        DD_CUDA(cudaMemcpy(out, res.data(), sizeof(double) * res.size(), cudaMemcpyHostToDevice));
    } else {
        std::memcpy(out, res.data(), sizeof(double) * res.size());
    }
    return 0;
}

}  // extern "C"

template <typename T>
static int coarse_solve_T(ddamg_handle* h, const double* in, double* out, int n_rhs, int fixed) {
    const size_t cn = (size_t)h->NB * h->nc;
    DD_TRY(h->ws_fine[5].ensure(sizeof(cplx<T>) * cn * n_rhs * 2));
    cplx<T>* a = h->ws_fine[5].as<cplx<T>>();
    cplx<T>* o = a + cn * n_rhs;
    DD_TRY(coarse_in<T>(h, in, n_rhs, a));
    h->coarse_iters = 0;
    DD_TRY(coarse_solve<T>(h, a, o, n_rhs, fixed));
    DD_TRY(coarse_out<T>(h, o, out, n_rhs));
    return tc_check(h);
}

extern "C" {
int ddamg_coarse_solve(ddamg_handle* h, const double* in, double* out, int n_rhs, int fixed_iters) {
    DD_TRY(check_ready(h));
    if (!in || !out || n_rhs < 1) return DDAMG_ERR_INVALID_ARG;
    return h->single() ? coarse_solve_T<float>(h, in, out, n_rhs, fixed_iters) : coarse_solve_T<double>(h, in, out, n_rhs, fixed_iters);
}

}  // extern "C"

template <typename T>
static int vcycle_T(ddamg_handle* h, const double* in, double* out, int n_rhs, int fixed) {
    const size_t fld = (size_t)12 * h->V;
    DD_TRY(h->ws_fine[5].ensure(sizeof(cplx<T>) * fld * n_rhs * 2));
    cplx<T>* a = h->ws_fine[5].as<cplx<T>>();
    cplx<T>* o = a + fld * n_rhs;
    DD_TRY(fine_in<T>(h, in, n_rhs, h->ws_io[0], a));
    DD_TRY(vcycle<T>(h, a, o, n_rhs, fixed));
    return fine_out<T>(h, o, out, n_rhs);
}

extern "C" {
int ddamg_vcycle(ddamg_handle* h, const double* in, double* out, int n_rhs, int coarse_fixed_iters) {
    DD_TRY(check_ready(h));
    if (!in || !out || n_rhs < 1) return DDAMG_ERR_INVALID_ARG;
    return h->single() ? vcycle_T<float>(h, in, out, n_rhs, coarse_fixed_iters) : vcycle_T<double>(h, in, out, n_rhs, coarse_fixed_iters);
}

int ddamg_set_mass(ddamg_handle* h, double m0) {
    if (!h) return DDAMG_ERR_INVALID_ARG;
    // site terms: rebuild with the new mass (the clover part does not depend on it)
    const double old_m0 = h->m0;
    h->m0 = m0;
    DD_TRY(launch_clover(h->g, h->U64, m0, h->csw, h->clov64, h->clovinv64, h->stream));
    if (h->single()) {
        DD_TRY((convert<float, double>(h->clov64, h->clov32, (size_t)h->V * 72, h->stream)));
        DD_TRY((convert<float, double>(h->clovinv64, h->clovinv32, (size_t)h->V * 72, h->stream)));
        DD_TRY(launch_to_dw(h->clov64, h->clovdw, (size_t)h->V * 72, h->stream));
        DD_TRY(clover_to_aos(h->clov32, h->clov_aos, h->V, h->stream));
        DD_TRY(clover_to_aos(h->clovinv32, h->clovinv_aos, h->V, h->stream));
        if (h->half() && h->p.smoother_fp16) {
            DD_TRY(clover_to_aos16(h->clov32, h->clov_aos16, h->V, h->stream));
            DD_TRY(clover_to_aos16(h->clovinv32, h->clovinv_aos16, h->V, h->stream));
        }
    }
    if (h->ready) {
        // mass re-use (Sec. 6.3): P is kept, D_c moves by (m0' - m0) I, only the inverses are redone
        const double delta = m0 - old_m0;
        shift_coarse_diag_kernel<<<ceil_div((long long)h->NB * h->nc, 256), 256, 0, h->stream>>>(h->B64, h->NB, h->nc, delta);
        DD_CHECK_LAUNCH();
        DD_TRY(finish_coarse(h));
    }
    DD_CUDA(cudaStreamSynchronize(h->stream));
    return 0;
}

int ddamg_set_stream(ddamg_handle* h, void* s) {
    if (!h) return DDAMG_ERR_INVALID_ARG;
    h->stream = s ? reinterpret_cast<cudaStream_t>(s) : h->own_stream;
    return 0;
}

int ddamg_info(const ddamg_handle* h, long long* n_sites, long long* n_coarse, int* dof) {
    if (!h) return DDAMG_ERR_INVALID_ARG;
    if (n_sites) *n_sites = h->V;
    if (n_coarse) *n_coarse = h->NB;
    if (dof) *dof = h->nc;
    return 0;
}

int ddamg_profile_enable(ddamg_handle* h, int family_mask) {
    if (!h) return DDAMG_ERR_INVALID_ARG;
    h->prof_mask = family_mask;
    return 0;
}

int ddamg_profile_families(char* names, int len) {
    std::string all;
    for (int f = 0; f < PF_COUNT; ++f) {
        if (f) all += ",";
        all += kPfNames[f];
    }
    if (names && len > 0) {
        std::strncpy(names, all.c_str(), (size_t)len - 1);
        names[len - 1] = 0;
    }
    return PF_COUNT;
}

int ddamg_profile_reset(ddamg_handle* h) {
    if (!h) return DDAMG_ERR_INVALID_ARG;
    DD_CUDA(cudaStreamSynchronize(h->stream));
    for (auto& r : h->prof) {
        h->ev_pool.push_back(r.e0);
        h->ev_pool.push_back(r.e1);
    }
    h->prof.clear();
    return 0;
}

int ddamg_profile_read(ddamg_handle* h, ddamg_kernel_profile* out, int max) {
    if (!h || (!out && max > 0)) return DDAMG_ERR_INVALID_ARG;
    DD_CUDA(cudaStreamSynchronize(h->stream));
    long long n[PF_COUNT] = {0};
    double ms[PF_COUNT] = {0}, by[PF_COUNT] = {0}, fl[PF_COUNT] = {0};
    for (auto& r : h->prof) {
        float t = 0;
        if (cudaEventElapsedTime(&t, r.e0, r.e1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        n[r.fam]++;
        ms[r.fam] += t;
        by[r.fam] += r.bytes;
        fl[r.fam] += r.flops;
    }
    int k = 0;
    for (int f = 0; f < PF_COUNT; ++f) {
        if (!n[f]) continue;
        if (k < max) {
            std::memset(&out[k], 0, sizeof(out[k]));
            std::strncpy(out[k].name, kPfNames[f], sizeof(out[k].name) - 1);
            out[k].launches = n[f];
            out[k].total_ms = ms[f];
            out[k].bytes = by[f];
            out[k].flops = fl[f];
        }
        ++k;
    }
    return k;
}

int ddamg_destroy(ddamg_handle* h) {
    if (!h) return 0;
    if (h->stream) cudaStreamSynchronize(h->stream);
    ml_release(h);
    dfree(h->d_lnbr);
    dfree(h->d_blex);
    dfree(h->d_bnbr);
    dfree(h->d_lex_of);
    dfree(h->d_clex_of);
    dfree(h->d_sites);
    dfree(h->U64);
    dfree(h->clov64);
    dfree(h->clovinv64);
    dfree(h->U32);
    dfree(h->Uaos);
    dfree(h->Uaos16);
    dfree(h->clov_aos16);
    dfree(h->clovinv_aos16);
    dfree(h->clov_aos);
    dfree(h->clovinv_aos);
    dfree(h->clov32);
    dfree(h->clovinv32);
    dfree(h->V64);
    dfree(h->P64);
    dfree(h->P32);
    dfree(h->B64);
    dfree(h->Dinv64);
    dfree(h->B32);
    dfree(h->Dinv32);
    dfree(h->Udw);
    dfree(h->clovdw);
    dfree(h->Bh);
    dfree(h->Dh);
    dfree(h->P16);
    dfree(h->d_flag);
    dfree(h->d_tc_err);
    for (auto& s : h->ws_fine) s.release();
    for (auto& s : h->ws_coarse) s.release();
    for (auto& s : h->ws_io) s.release();
    for (auto& s : h->ws_outer) s.release();
    h->ws_rmax.release();
    dfree(h->slot_b);
    dfree(h->slot_x);
    h->kc.release();
    h->ko.release();
    for (auto& r : h->prof) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
    return 0;
}

}  // extern "C"

#include "multilevel.inc"
