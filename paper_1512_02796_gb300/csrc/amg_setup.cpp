// Host side of the smoothed-aggregation hierarchy (see amg.h): aggregates
// of the matrix graph, the patterns of P, A P, R = P^T and P^T A P on every
// level, and the index plans that let the device form their values with
// plain gathers.  Everything here depends on the pattern only, is computed
// once per mesh and pattern, and is deterministic (row loops are split over
// host threads in fixed contiguous ranges and concatenated in order).
#include "amg.h"
#include "qpat_internal.h"

#include <algorithm>
#include <thread>

namespace qpat {
namespace {

int host_threads() {
    const unsigned h = std::thread::hardware_concurrency();
    return int(std::max(1u, std::min(h, 16u)));
}

// fn(t, begin, end) over nt contiguous ranges of [0, n).
template <typename F>
void parallel_ranges(int64_t n, int nt, const F& fn) {
    if (nt <= 1 || n < 8192) {
        fn(0, int64_t(0), n);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(nt);
    for (int t = 0; t < nt; ++t) {
        const int64_t b = n * t / nt, e = n * (t + 1) / nt;
        th.emplace_back([&fn, t, b, e] { fn(t, b, e); });
    }
    for (auto& x : th) x.join();
}

struct Csr {
    int64_t n = 0;
    std::vector<int64_t> ptr;
    std::vector<int32_t> col;
    int64_t len(int64_t i) const { return ptr[i + 1] - ptr[i]; }
};

// Distinct column ids of one row, collected in O(1) each.
struct Marker {
    std::vector<int64_t> stamp;
    std::vector<int32_t> list;
    explicit Marker(int64_t ncols) : stamp(size_t(ncols), -1) {}
    void begin() { list.clear(); }
    void add(int32_t c, int64_t row) {
        if (stamp[size_t(c)] != row) {
            stamp[size_t(c)] = row;
            list.push_back(c);
        }
    }
};

// CSR of n rows over ncols columns; row i = sorted distinct ids that
// gather(i, marker) adds.
template <typename G>
Csr build_rows(int64_t n, int64_t ncols, const G& gather) {
    const int nt = n < 8192 ? 1 : host_threads();
    std::vector<std::vector<int32_t>> cols(static_cast<size_t>(nt));
    std::vector<std::vector<int64_t>> lens(static_cast<size_t>(nt));
    parallel_ranges(n, nt, [&](int t, int64_t b, int64_t e) {
        Marker mk(ncols);
        auto& c = cols[size_t(t)];
        auto& l = lens[size_t(t)];
        l.reserve(size_t(e - b));
        for (int64_t i = b; i < e; ++i) {
            mk.begin();
            gather(i, mk);
            std::sort(mk.list.begin(), mk.list.end());
            c.insert(c.end(), mk.list.begin(), mk.list.end());
            l.push_back(int64_t(mk.list.size()));
        }
    });
    Csr out;
    out.n = n;
    out.ptr.assign(size_t(n + 1), 0);
    int64_t row = 0;
    for (int t = 0; t < nt; ++t)
        for (int64_t L : lens[size_t(t)]) {
            out.ptr[size_t(row + 1)] = out.ptr[size_t(row)] + L;
            ++row;
        }
    out.col.reserve(size_t(out.ptr[size_t(n)]));
    for (int t = 0; t < nt; ++t) out.col.insert(out.col.end(), cols[size_t(t)].begin(), cols[size_t(t)].end());
    return out;
}

// Position of column c in the sorted row [b, e) of col (the caller knows it is there).
inline int slot_of(const int32_t* col, int64_t b, int64_t e, int32_t c) {
    return int(std::lower_bound(col + b, col + e, c) - (col + b));
}

bool sell_from_csr(const Csr& c, SellPattern& s, std::string& err) {
    if (c.n > 0 && c.ptr[size_t(c.n)] >= int64_t(kAmgRowMajorLen) * c.n) {
        // long rows: row-major, so that the lanes sharing a row read consecutive entries
        s.n = c.n;
        s.nslices = 0;
        s.rowmajor = true;
        s.ptr = c.ptr;
        s.col = c.col;
        s.len.assign(size_t(c.n), 0);
        s.maxlen = 0;
        for (int64_t i = 0; i < c.n; ++i) {
            if (c.len(i) > 65535) {
                err = "multigrid: a row of a level holds more than 65535 entries";
                return false;
            }
            s.len[size_t(i)] = uint16_t(c.len(i));
            s.maxlen = std::max(s.maxlen, int(c.len(i)));
        }
        return true;
    }
    s.n = c.n;
    s.rowmajor = false;
    s.nslices = (c.n + 31) / 32;
    s.ptr.assign(size_t(s.nslices + 1), 0);
    s.len.assign(size_t(32 * s.nslices), 0);
    s.maxlen = 0;
    for (int64_t sl = 0; sl < s.nslices; ++sl) {
        int64_t w = 0;
        for (int64_t i = 32 * sl; i < std::min(c.n, 32 * sl + 32); ++i) w = std::max(w, c.len(i));
        if (w > 65535) {
            err = "multigrid: a row of a level holds more than 65535 entries";
            return false;
        }
        s.ptr[size_t(sl + 1)] = s.ptr[size_t(sl)] + w;
        s.maxlen = std::max(s.maxlen, int(w));
    }
    s.col.assign(size_t(32 * s.ptr[size_t(s.nslices)]), 0);
    for (int64_t sl = 0; sl < s.nslices; ++sl) {
        const int64_t w = s.ptr[size_t(sl + 1)] - s.ptr[size_t(sl)];
        for (int lane = 0; lane < 32; ++lane) {
            const int64_t i = 32 * sl + lane;
            const int64_t L = i < c.n ? c.len(i) : 0;
            if (i < c.n) s.len[size_t(i)] = uint16_t(L);
            for (int64_t k = 0; k < w; ++k)
                s.col[size_t((s.ptr[size_t(sl)] + k) * 32 + lane)] =
                    k < L ? c.col[size_t(c.ptr[size_t(i)] + k)] : int32_t(i < c.n ? i : 0);
        }
    }
    return true;
}

// Aggregates of the graph of A (Vanek, Mandel, Brezina 1996, without a
// strength threshold: the pattern alone decides).  1: every node whose
// neighbours are all free forms an aggregate with them; 2: a free node joins
// the aggregate of step 1 it has most neighbours in (ties: the lower id);
// 3: what is left forms aggregates with its free neighbours.
std::vector<int32_t> aggregate(const SellPattern& A, int64_t& nagg) {
    const int64_t n = A.n;
    std::vector<int32_t> agg(size_t(n), -1);
    int32_t na = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (agg[size_t(i)] >= 0) continue;
        bool free_ = true;
        for (int k = 0; k < A.len[size_t(i)] && free_; ++k) {
            const int32_t j = A.col[size_t(A.pos(i, k))];
            if (j != i && agg[size_t(j)] >= 0) free_ = false;
        }
        if (!free_) continue;
        agg[size_t(i)] = na;
        for (int k = 0; k < A.len[size_t(i)]; ++k) agg[size_t(A.col[size_t(A.pos(i, k))])] = na;
        ++na;
    }
    const std::vector<int32_t> agg1 = agg;
    std::vector<std::pair<int32_t, int>> cnt;
    for (int64_t i = 0; i < n; ++i) {
        if (agg1[size_t(i)] >= 0) continue;
        cnt.clear();
        for (int k = 0; k < A.len[size_t(i)]; ++k) {
            const int32_t j = A.col[size_t(A.pos(i, k))];
            const int32_t a = j == i ? -1 : agg1[size_t(j)];
            if (a < 0) continue;
            auto it = std::find_if(cnt.begin(), cnt.end(), [a](const std::pair<int32_t, int>& p) { return p.first == a; });
            if (it == cnt.end())
                cnt.push_back({a, 1});
            else
                ++it->second;
        }
        if (cnt.empty()) continue;
        std::pair<int32_t, int> best = cnt[0];
        for (const auto& p : cnt)
            if (p.second > best.second || (p.second == best.second && p.first < best.first)) best = p;
        agg[size_t(i)] = best.first;
    }
    for (int64_t i = 0; i < n; ++i) {
        if (agg[size_t(i)] >= 0) continue;
        agg[size_t(i)] = na;
        for (int k = 0; k < A.len[size_t(i)]; ++k) {
            const int32_t j = A.col[size_t(A.pos(i, k))];
            if (agg[size_t(j)] < 0) agg[size_t(j)] = na;
        }
        ++na;
    }
    nagg = na;
    return agg;
}

}  // namespace

namespace {

bool set_diag(AmgLevelPlan& L) {
    const SellPattern& A = L.A;
    L.diag.assign(size_t(A.n), -1);
    for (int64_t i = 0; i < A.n; ++i)
        for (int k = 0; k < A.len[size_t(i)]; ++k)
            if (A.col[size_t(A.pos(i, k))] == i) {
                L.diag[size_t(i)] = k;
                break;
            }
    return std::find(L.diag.begin(), L.diag.end(), -1) == L.diag.end();
}

// The transfer from level L to the next one; `coarse` receives the next
// level's pattern (rows sorted).
bool build_transfer(AmgLevelPlan& L, Csr& coarse, std::string& err) {
    const SellPattern& A = L.A;
    const int64_t n = A.n;
    const int nt = n < 8192 ? 1 : host_threads();
    int64_t nc = 0;
    L.agg = aggregate(A, nc);
    L.nc = nc;
    if (nc <= 0 || nc >= n) {
        err = "multigrid: aggregation made no progress";
        return false;
    }
    // P = (I - omega D^-1 A) P_tent: row i holds the aggregates of i's row of A
    const Csr Pc = build_rows(n, nc, [&](int64_t i, Marker& mk) {
        for (int k = 0; k < A.len[size_t(i)]; ++k) mk.add(L.agg[size_t(A.col[size_t(A.pos(i, k))])], i);
    });
    if (!sell_from_csr(Pc, L.P, err)) return false;
    L.a2p.assign(size_t(A.entries()), 0);
    L.pself.assign(size_t(n), 0);
    parallel_ranges(n, nt, [&](int, int64_t b, int64_t e) {
        for (int64_t i = b; i < e; ++i) {
            const int64_t pb = Pc.ptr[size_t(i)], pe = Pc.ptr[size_t(i + 1)];
            for (int k = 0; k < A.len[size_t(i)]; ++k) {
                const int64_t at = A.pos(i, k);
                L.a2p[size_t(at)] = uint16_t(slot_of(Pc.col.data(), pb, pe, L.agg[size_t(A.col[size_t(at)])]));
            }
            L.pself[size_t(i)] = uint16_t(slot_of(Pc.col.data(), pb, pe, L.agg[size_t(i)]));
        }
    });
    // A P: row i is the union of the P rows of i's neighbours
    Csr APc = build_rows(n, nc, [&](int64_t i, Marker& mk) {
        for (int k = 0; k < A.len[size_t(i)]; ++k) {
            const int32_t j = A.col[size_t(A.pos(i, k))];
            for (int64_t q = Pc.ptr[size_t(j)]; q < Pc.ptr[size_t(j + 1)]; ++q) mk.add(Pc.col[size_t(q)], i);
        }
    });
    for (int64_t i = 0; i < n; ++i)
        if (APc.len(i) > 65535) {
            err = "multigrid: a row of A P holds more than 65535 entries";
            return false;
        }
    L.ap_sptr.assign(size_t(n + 1), 0);
    for (int64_t i = 0; i < n; ++i) {
        int64_t s = 0;
        for (int k = 0; k < A.len[size_t(i)]; ++k) s += Pc.len(A.col[size_t(A.pos(i, k))]);
        L.ap_sptr[size_t(i + 1)] = L.ap_sptr[size_t(i)] + s;
    }
    L.ap_slot.assign(size_t(L.ap_sptr[size_t(n)]), 0);
    parallel_ranges(n, nt, [&](int, int64_t b, int64_t e) {
        for (int64_t i = b; i < e; ++i) {
            int64_t o = L.ap_sptr[size_t(i)];
            for (int k = 0; k < A.len[size_t(i)]; ++k) {
                const int32_t j = A.col[size_t(A.pos(i, k))];
                for (int64_t q = Pc.ptr[size_t(j)]; q < Pc.ptr[size_t(j + 1)]; ++q)
                    L.ap_slot[size_t(o++)] = uint16_t(
                        slot_of(APc.col.data(), APc.ptr[size_t(i)], APc.ptr[size_t(i + 1)], Pc.col[size_t(q)]));
            }
        }
    });
    // R = P^T: coarse row I lists the fine rows whose P row holds I, ascending
    Csr Rc;
    Rc.n = nc;
    Rc.ptr.assign(size_t(nc + 1), 0);
    for (int32_t I : Pc.col) ++Rc.ptr[size_t(I + 1)];
    for (int64_t I = 0; I < nc; ++I) Rc.ptr[size_t(I + 1)] += Rc.ptr[size_t(I)];
    Rc.col.assign(Pc.col.size(), 0);
    std::vector<int64_t> rsrc(Pc.col.size(), -1);
    {
        std::vector<int64_t> next(Rc.ptr.begin(), Rc.ptr.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t q = Pc.ptr[size_t(i)]; q < Pc.ptr[size_t(i + 1)]; ++q) {
                const int64_t at = next[size_t(Pc.col[size_t(q)])]++;
                Rc.col[size_t(at)] = int32_t(i);
                rsrc[size_t(at)] = L.P.pos(i, int(q - Pc.ptr[size_t(i)]));
            }
    }
    if (!sell_from_csr(Rc, L.R, err)) return false;
    L.r_src.assign(size_t(L.R.entries()), -1);
    for (int64_t I = 0; I < nc; ++I)
        for (int k = 0; k < L.R.len[size_t(I)]; ++k) L.r_src[size_t(L.R.pos(I, k))] = rsrc[size_t(Rc.ptr[size_t(I)] + k)];
    // P^T A P: coarse row I is the union of the A P rows of R's row I
    coarse = build_rows(nc, nc, [&](int64_t I, Marker& mk) {
        for (int64_t q = Rc.ptr[size_t(I)]; q < Rc.ptr[size_t(I + 1)]; ++q) {
            const int32_t i = Rc.col[size_t(q)];
            for (int64_t a = APc.ptr[size_t(i)]; a < APc.ptr[size_t(i + 1)]; ++a) mk.add(APc.col[size_t(a)], I);
        }
    });
    L.g_ptr.assign(size_t(nc + 1), 0);
    for (int64_t I = 0; I < nc; ++I) {
        int64_t s = 0;
        for (int64_t q = Rc.ptr[size_t(I)]; q < Rc.ptr[size_t(I + 1)]; ++q) s += APc.len(Rc.col[size_t(q)]);
        L.g_ptr[size_t(I + 1)] = L.g_ptr[size_t(I)] + s;
    }
    L.g_slot.assign(size_t(L.g_ptr[size_t(nc)]), 0);
    parallel_ranges(nc, nc < 8192 ? 1 : nt, [&](int, int64_t b, int64_t e) {
        for (int64_t I = b; I < e; ++I) {
            int64_t o = L.g_ptr[size_t(I)];
            for (int64_t q = Rc.ptr[size_t(I)]; q < Rc.ptr[size_t(I + 1)]; ++q) {
                const int32_t i = Rc.col[size_t(q)];
                for (int64_t a = APc.ptr[size_t(i)]; a < APc.ptr[size_t(i + 1)]; ++a)
                    L.g_slot[size_t(o++)] = uint16_t(slot_of(coarse.col.data(), coarse.ptr[size_t(I)],
                                                             coarse.ptr[size_t(I + 1)], APc.col[size_t(a)]));
            }
        }
    });
    L.ap_ptr = std::move(APc.ptr);
    L.ap_col = std::move(APc.col);
    return true;
}

}  // namespace

AmgPlan amg_build_plan(const SellPattern& fine) {
    AmgPlan plan;
    plan.levels.reserve(kAmgMaxLevels);
    plan.levels.emplace_back();
    plan.levels[0].A = fine;
    if (!set_diag(plan.levels[0])) {
        plan.error = "multigrid: a row of the pattern has no diagonal entry";
        return plan;
    }
    while (plan.levels.back().A.n > kAmgCoarsest) {
        if (int(plan.levels.size()) >= kAmgMaxLevels) {
            plan.error = "multigrid: no coarsest level of at most 128 rows within 12 levels";
            return plan;
        }
        Csr coarse;
        if (!build_transfer(plan.levels.back(), coarse, plan.error)) return plan;
        plan.levels.emplace_back();
        if (!sell_from_csr(coarse, plan.levels.back().A, plan.error)) return plan;
        if (!set_diag(plan.levels.back())) {
            plan.error = "multigrid: a coarse row has no diagonal entry";
            return plan;
        }
    }
    return plan;
}

}  // namespace qpat

namespace qpat {

SellPattern amg_fine_pattern(const HostMesh& h, int prior) {
    const auto& ptr = prior ? h.psell_ptr : h.sell_ptr;
    const auto& col = prior ? h.psell_col : h.sell_col;
    const auto& len = prior ? h.psell_len : h.sell_len;
    SellPattern f;
    f.n = h.N;
    f.nslices = int64_t(ptr.size()) - 1;
    f.ptr = ptr;
    f.col.assign(size_t(32 * ptr.back()), 0);
    f.len.assign(len.begin(), len.end());
    f.maxlen = 0;
    for (int64_t s = 0; s < f.nslices; ++s) {
        const int64_t w = ptr[size_t(s + 1)] - ptr[size_t(s)];
        f.maxlen = std::max(f.maxlen, int(w));
        const int p = h.patch_of_slice[size_t(s)];
        const int nb = h.node_ptr[size_t(p)];
        for (int lane = 0; lane < 32; ++lane) {
            const int64_t g = 32 * s + lane;
            for (int64_t k = 0; k < w; ++k) {
                const int64_t at = (ptr[size_t(s)] + k) * 32 + lane;
                f.col[size_t(at)] = g < h.N ? h.nodes[size_t(nb + col[size_t(at)])] : 0;
            }
        }
    }
    return f;
}


std::string amg_check_plan(const AmgPlan& plan) {
    if (!plan.error.empty()) return plan.error;
    if (plan.levels.empty()) return "no levels";
    for (size_t l = 0; l < plan.levels.size(); ++l) {
        const AmgLevelPlan& L = plan.levels[l];
        const SellPattern& A = L.A;
        const std::string at = "level " + std::to_string(l) + ": ";
        for (int64_t i = 0; i < A.n; ++i)
            if (L.diag[size_t(i)] < 0 || A.col[size_t(A.pos(i, L.diag[size_t(i)]))] != i) return at + "diagonal slot";
        if (l + 1 == plan.levels.size()) {
            if (L.nc != 0) return at + "coarsest level with a transfer";
            if (A.n > kAmgCoarsest) return at + "coarsest level too large";
            break;
        }
        const SellPattern& C = plan.levels[l + 1].A;
        if (L.nc != C.n || L.nc >= A.n) return at + "coarse size";
        // every aggregate non-empty
        std::vector<int> members(size_t(L.nc), 0);
        for (int32_t a : L.agg) {
            if (a < 0 || a >= L.nc) return at + "aggregate id";
            ++members[size_t(a)];
        }
        if (std::find(members.begin(), members.end(), 0) != members.end()) return at + "empty aggregate";
        // P rows: the aggregates of the row's neighbours, a2p and pself point at them
        for (int64_t i = 0; i < A.n; ++i) {
            const int LP = L.P.len[size_t(i)];
            for (int k = 1; k < LP; ++k)
                if (L.P.col[size_t(L.P.pos(i, k - 1))] >= L.P.col[size_t(L.P.pos(i, k))]) return at + "P row order";
            if (L.pself[size_t(i)] >= LP || L.P.col[size_t(L.P.pos(i, L.pself[size_t(i)]))] != L.agg[size_t(i)])
                return at + "pself";
            for (int k = 0; k < A.len[size_t(i)]; ++k) {
                const int64_t e = A.pos(i, k);
                const int s = L.a2p[size_t(e)];
                if (s >= LP || L.P.col[size_t(L.P.pos(i, s))] != L.agg[size_t(A.col[size_t(e)])]) return at + "a2p";
            }
        }
        // A P slots name the P entry's column
        for (int64_t i = 0; i < A.n; ++i) {
            int64_t o = L.ap_sptr[size_t(i)];
            const int64_t b = L.ap_ptr[size_t(i)], e = L.ap_ptr[size_t(i + 1)];
            for (int k = 0; k < A.len[size_t(i)]; ++k) {
                const int32_t j = A.col[size_t(A.pos(i, k))];
                for (int kk = 0; kk < L.P.len[size_t(j)]; ++kk) {
                    const int s = L.ap_slot[size_t(o++)];
                    if (s >= e - b || L.ap_col[size_t(b + s)] != L.P.col[size_t(L.P.pos(j, kk))]) return at + "ap_slot";
                }
            }
            if (o != L.ap_sptr[size_t(i + 1)]) return at + "ap_sptr";
        }
        // R = P^T: every P entry exactly once, at the right row and column
        std::vector<char> seen(size_t(L.P.entries()), 0);
        int64_t count = 0;
        for (int64_t I = 0; I < L.nc; ++I)
            for (int k = 0; k < L.R.len[size_t(I)]; ++k) {
                const int64_t e = L.R.pos(I, k);
                const int64_t src = L.r_src[size_t(e)];
                const int32_t i = L.R.col[size_t(e)];
                if (src < 0 || src >= L.P.entries() || seen[size_t(src)]) return at + "r_src";
                seen[size_t(src)] = 1;
                ++count;
                // src must lie in row i of P and hold column I
                bool ok = false;
                for (int kk = 0; kk < L.P.len[size_t(i)] && !ok; ++kk) ok = L.P.pos(i, kk) == src && L.P.col[size_t(src)] == I;
                if (!ok) return at + "R is not P^T";
            }
        int64_t pentries = 0;
        for (int64_t i = 0; i < A.n; ++i) pentries += L.P.len[size_t(i)];
        if (count != pentries) return at + "R misses P entries";
        // Galerkin slots name the A P column in the coarse row
        for (int64_t I = 0; I < L.nc; ++I) {
            int64_t o = L.g_ptr[size_t(I)];
            for (int k = 0; k < L.R.len[size_t(I)]; ++k) {
                const int32_t i = L.R.col[size_t(L.R.pos(I, k))];
                for (int64_t a = L.ap_ptr[size_t(i)]; a < L.ap_ptr[size_t(i + 1)]; ++a) {
                    const int s = L.g_slot[size_t(o++)];
                    if (s >= C.len[size_t(I)] || C.col[size_t(C.pos(I, s))] != L.ap_col[size_t(a)]) return at + "g_slot";
                }
            }
            if (o != L.g_ptr[size_t(I + 1)]) return at + "g_ptr";
        }
        // the coarse pattern is symmetric
        for (int64_t I = 0; I < C.n; ++I)
            for (int k = 0; k < C.len[size_t(I)]; ++k) {
                const int32_t J = C.col[size_t(C.pos(I, k))];
                bool found = false;
                for (int kk = 0; kk < C.len[size_t(J)] && !found; ++kk) found = C.col[size_t(C.pos(J, kk))] == I;
                if (!found) return at + "coarse pattern not symmetric";
            }
    }
    return "";
}

}  // namespace qpat
