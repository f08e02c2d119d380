// Blocking of the level-1 lattice for the recursion to a third level (Sec. 3: the two-level
// method formulated again for the coarse system; Sec. 6.4: 3 and 4 levels).  Host-only C++.
//
// The level-1 lattice is the lattice of the fine aggregates, with the library's internal coarse
// order: sites whose coordinate sum is even first, then odd, each group lexicographic (x0
// slowest).  Its own lattice blocks serve as the level-1 SAP domains and as the level-1
// aggregates; they become the sites of level 2, numbered by the same rule (blocks with an even
// block-coordinate sum, i.e. red blocks, first).  Inside a block the sites are listed with the
// globally even ones first, each group in lexicographic order: the operator's even sites are the
// ones whose diagonal blocks are inverted (odd-even reduction of the block solves).
#pragma once

#include <array>
#include <vector>

namespace ddamg {

struct MLHostGeom {
    int L1[4] = {0, 0, 0, 0};   // level-1 extents
    int b1[4] = {0, 0, 0, 0};   // block extents on level 1
    int nb1[4] = {0, 0, 0, 0};  // blocks per direction = level-2 extents
    int NB = 0;                 // level-1 sites
    int NB2 = 0;                // level-1 blocks = level-2 sites
    int Vb1 = 0;                // sites per block
    int Vb1e = 0;               // globally even sites per block (the first Vb1e local indices)
    std::vector<int> lex1;      // [NB] lexicographic index of each internal level-1 site
    std::vector<int> nbr1;      // [8][NB] internal index of the neighbour in direction 2 mu + backward
    std::vector<int> sites;     // [NB2][Vb1] internal level-1 site of (block, local index)
    std::vector<int> blk_of;    // [NB] block (level-2 site) of each level-1 site
    std::vector<int> loc_of;    // [NB] local index inside its block
    std::vector<unsigned char> same;  // [8][NB] 1 where the neighbour lies in the same block
    std::vector<int> nbr2;      // [8][NB2] neighbouring level-2 site
    std::vector<int> lex2;      // [NB2] lexicographic index of each internal level-2 site
};

namespace mlg {
inline int lex(const int* L, const std::array<int, 4>& x) { return ((x[0] * L[1] + x[1]) * L[2] + x[2]) * L[3] + x[3]; }
inline std::array<int, 4> coords(const int* L, int q) {
    return {q / (L[1] * L[2] * L[3]), (q / (L[2] * L[3])) % L[1], (q / L[3]) % L[2], q % L[3]};
}
// internal order of a periodic lattice: even coordinate sums first, each group lexicographic
inline void parity_order(const int* L, std::vector<int>& lex_of, std::vector<int>& int_of) {
    const int n = L[0] * L[1] * L[2] * L[3];
    lex_of.assign(n, 0);
    int_of.assign(n, 0);
    int idx = 0;
    for (int par = 0; par < 2; ++par)
        for (int q = 0; q < n; ++q) {
            std::array<int, 4> x = coords(L, q);
            if (((x[0] + x[1] + x[2] + x[3]) & 1) != par) continue;
            lex_of[idx] = q;
            int_of[q] = idx++;
        }
}
}  // namespace mlg

// Fills g; returns 0, or -1 when an extent is not positive, a block extent does not divide the
// lattice, a direction has an odd number of blocks (red-black SAP and the odd-even coarsest
// solve need even counts), or every block extent is odd (a block then holds different numbers
// of even and odd sites).
inline int ml_build_geom(const int L1[4], const int b1[4], MLHostGeom& g) {
    bool any_even = false;
    for (int m = 0; m < 4; ++m) {
        if (L1[m] < 1 || b1[m] < 1 || L1[m] % b1[m]) return -1;
        if ((L1[m] / b1[m]) % 2) return -1;
        any_even = any_even || (b1[m] % 2 == 0);
        g.L1[m] = L1[m];
        g.b1[m] = b1[m];
        g.nb1[m] = L1[m] / b1[m];
    }
    if (!any_even) return -1;
    g.NB = L1[0] * L1[1] * L1[2] * L1[3];
    g.Vb1 = b1[0] * b1[1] * b1[2] * b1[3];
    g.NB2 = g.NB / g.Vb1;
    g.Vb1e = g.Vb1 / 2;
    std::vector<int> int1, int2;
    mlg::parity_order(g.L1, g.lex1, int1);
    mlg::parity_order(g.nb1, g.lex2, int2);
    g.nbr1.assign(8 * (size_t)g.NB, 0);
    g.nbr2.assign(8 * (size_t)g.NB2, 0);
    g.same.assign(8 * (size_t)g.NB, 0);
    g.blk_of.assign(g.NB, 0);
    g.loc_of.assign(g.NB, 0);
    g.sites.assign((size_t)g.NB2 * g.Vb1, 0);
    std::vector<int> fill_e(g.NB2, 0), fill_o(g.NB2, g.Vb1e);
    for (int c = 0; c < g.NB; ++c) {
        std::array<int, 4> x = mlg::coords(g.L1, g.lex1[c]), bc;
        for (int m = 0; m < 4; ++m) bc[m] = x[m] / g.b1[m];
        const int c2 = int2[mlg::lex(g.nb1, bc)];
        const bool even = ((x[0] + x[1] + x[2] + x[3]) & 1) == 0;
        int& slot = even ? fill_e[c2] : fill_o[c2];
        if (slot >= (even ? g.Vb1e : g.Vb1)) return -1;  // not reached when some block extent is even
        g.blk_of[c] = c2;
        g.loc_of[c] = slot;
        g.sites[(size_t)c2 * g.Vb1 + slot] = c;
        ++slot;
        for (int d = 0; d < 8; ++d) {
            const int mu = d >> 1, s = (d & 1) ? -1 : 1;
            std::array<int, 4> y = x;
            y[mu] = (y[mu] + s + g.L1[mu]) % g.L1[mu];
            const int n = int1[mlg::lex(g.L1, y)];
            g.nbr1[(size_t)d * g.NB + c] = n;
            std::array<int, 4> by;
            for (int m = 0; m < 4; ++m) by[m] = y[m] / g.b1[m];
            g.same[(size_t)d * g.NB + c] = (by == bc) ? 1 : 0;
        }
    }
    for (int c2 = 0; c2 < g.NB2; ++c2) {
        std::array<int, 4> bc = mlg::coords(g.nb1, g.lex2[c2]);
        for (int d = 0; d < 8; ++d) {
            const int mu = d >> 1, s = (d & 1) ? -1 : 1;
            std::array<int, 4> y = bc;
            y[mu] = (y[mu] + s + g.nb1[mu]) % g.nb1[mu];
            g.nbr2[(size_t)d * g.NB2 + c2] = int2[mlg::lex(g.nb1, y)];
        }
    }
    return 0;
}

}  // namespace ddamg
