// Smoothed-aggregation algebraic multigrid (internal): the preconditioner of
// the FP64 conjugate-gradient solves of K (Eq. (7)) and of M_delta (Eq. (19))
// selected by qpat_params.multigrid.
//
// The method is the textbook smoothed aggregation of Vanek, Mandel and
// Brezina (Computing 56, 1996): aggregates of the matrix graph, a piecewise-
// constant tentative prolongator smoothed by one damped Jacobi step,
// P = (I - omega D^-1 A) P_tent with omega = 4 / (3 rho(D^-1 A)), Galerkin
// coarse operators A_c = P^T A P, Chebyshev smoothing in D^-1 A on each level
// and an exact solve on the coarsest level; applied as one symmetric V-cycle
// per CG iteration.
//
// Split of the work:
//  * symbolic (host, once per mesh and matrix pattern, amg_setup.cpp): the
//    aggregates depend only on the pattern, so every level's pattern, P, R
//    = P^T, and the index plans of the numeric products are fixed per mesh;
//  * numeric (device, once per assembled operator, amg.cu): P's values from
//    A's, A P, P^T (A P), the inverse diagonals, the spectral bounds and the
//    coarsest inverse -- gathers in a fixed order, so every value is the
//    same from run to run;
//  * solve (device, amg.cu): conjugate gradients with the V-cycle, R right-
//    hand sides node-major, deterministic reductions.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace qpat {

// A sparse pattern in one of two layouts.  Sliced ELLPACK with 32-row
// slices (rowmajor = false): entry k of row i sits at
// (ptr[i / 32] + k) * 32 + i % 32, so the 32 rows of a warp read 32
// consecutive entries; padding entries repeat the row's own id (value 0).
// Row-major (rowmajor = true, for rows of a few dozen entries and more,
// which several lanes share): entry k of row i sits at ptr[i] + k.  Rows
// hold len[i] entries.  The patterns this file builds keep each row sorted
// by column; the fine level keeps the mesh's SELL order.
struct SellPattern {
    int64_t n = 0;         // rows
    int64_t nslices = 0;   // SELL: slices of 32 rows
    bool rowmajor = false;
    std::vector<int64_t> ptr;   // SELL: nslices + 1, in units of 32 entries; row-major: n + 1
    std::vector<int32_t> col;   // entries()
    std::vector<uint16_t> len;  // SELL: 32 * nslices (0 past row n - 1); row-major: n
    int64_t entries() const {
        if (ptr.empty()) return 0;
        return rowmajor ? ptr.back() : 32 * ptr.back();
    }
    int64_t pos(int64_t row, int k) const {
        return rowmajor ? ptr[size_t(row)] + k : (ptr[size_t(row / 32)] + k) * 32 + row % 32;
    }
    int maxlen = 0;
};

// Rows of at least this many entries on average are stored row-major and
// applied by 8 lanes per row.
constexpr int kAmgRowMajorLen = 24;

// Host plan of one level: the level's operator pattern and, except on the
// coarsest level, the transfer to the next one.
struct AmgLevelPlan {
    SellPattern A;                 // operator pattern (global column ids)
    std::vector<int32_t> diag;     // k of the diagonal entry of each row
    int64_t nc = 0;                // rows of the next level (0 on the coarsest)
    std::vector<int32_t> agg;      // aggregate of each row
    SellPattern P;                 // prolongator pattern (n rows, next-level columns)
    std::vector<uint16_t> a2p;      // per A entry (SELL position): slot in its row of P holding agg(col)
    std::vector<uint16_t> pself;    // per row: slot of agg(row) in its row of P
    // A P (n rows, next-level columns; CSR, columns sorted): the product's
    // pattern and, per row i, for every A entry k < len(i) and every P entry
    // kk < len_P(col_k), the slot of that P entry's column in row i of A P.
    std::vector<int64_t> ap_ptr;
    std::vector<int32_t> ap_col;
    std::vector<int64_t> ap_sptr;  // n + 1
    std::vector<uint16_t> ap_slot;
    // R = P^T (nc rows, fine columns sorted); r_src: the P SELL position of
    // each stored R entry (-1 on padding).
    SellPattern R;
    std::vector<int64_t> r_src;
    // Galerkin plan: for coarse row I, for every R entry k < len_R(I) (fine
    // row i) and every entry of row i of A P, the slot of that column in row
    // I of the next level's pattern.
    std::vector<int64_t> g_ptr;    // nc + 1
    std::vector<uint16_t> g_slot;
};

struct AmgPlan {
    std::vector<AmgLevelPlan> levels;  // levels[0] is the fine operator
    std::string error;                 // non-empty: no hierarchy (the caller keeps its other preconditioner)
};

// Largest coarsest level solved exactly (dense inverse in one CTA).
constexpr int kAmgCoarsest = 128;
// Most levels of a hierarchy.
constexpr int kAmgMaxLevels = 12;

// Builds the plan from the fine pattern in SELL form with global column ids
// (entries of a row in any order, the diagonal present, the pattern
// symmetric).  The fine level's A keeps the given positions, so the assembled
// values of the mesh's pattern serve as level 0 unchanged.
AmgPlan amg_build_plan(const SellPattern& fine);

// Checks every invariant the device kernels rely on (diagonal slots,
// non-empty aggregates, P, a2p, pself, the A P and Galerkin slots, R = P^T,
// symmetric coarse patterns, the coarsest size); "" if all hold.
std::string amg_check_plan(const AmgPlan& plan);

// The fine pattern of a prepared host mesh (K: prior = 0; the prior's
// stiffness-only pattern: prior = 1) with global column ids.
struct HostMesh;
SellPattern amg_fine_pattern(const HostMesh& h, int prior);

}  // namespace qpat
