// Host-side mesh preparation: boundary faces in canonical order, Morton
// locality order of the nodes and the owned-node CTA patches used by every
// element kernel.  The P1 basis of Eq. (5) lives on this mesh; the boundary
// faces carry the Robin term and the illumination of Eq. (1).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>

#include "qpat_internal.h"

namespace qpat {

namespace {

uint64_t spread3(uint64_t v) {
    // spread the low 21 bits of v to every third bit
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
}

struct Face {
    int32_t v[3];
    int32_t tet;
};

}  // namespace

std::string build_host_mesh(const double* xyz, int64_t N, const int32_t* tets,
                            int64_t E, int patch_nodes, int patch_multiple, HostMesh& m) {
    if (N <= 0 || E <= 0 || xyz == nullptr || tets == nullptr)
        return "qpat_mesh: empty mesh or NULL array";
    if (N >= (int64_t(1) << 31) || E >= (int64_t(1) << 29))
        return "qpat_mesh: mesh too large for 32-bit ids";
    if (patch_nodes < 32 || patch_nodes > 8192 || patch_nodes % 32 != 0)
        return "qpat_mesh: patch_nodes must be a multiple of 32 in [32, 8192]";
    for (int64_t i = 0; i < 4 * E; ++i)
        if (tets[i] < 0 || tets[i] >= N) return "qpat_mesh: tet node id out of range";
    for (int64_t i = 0; i < 3 * N; ++i)
        if (!std::isfinite(xyz[i])) return "qpat_mesh: non-finite coordinate";

    m = HostMesh();
    m.N = N;
    m.E = E;
    m.patch_nodes = patch_nodes;

    // ---- degenerate tets
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* t = tets + 4 * e;
        double d[3][3];
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) d[a][c] = xyz[3 * t[a + 1] + c] - xyz[3 * t[0] + c];
        double det = d[0][0] * (d[1][1] * d[2][2] - d[1][2] * d[2][1]) -
                     d[0][1] * (d[1][0] * d[2][2] - d[1][2] * d[2][0]) +
                     d[0][2] * (d[1][0] * d[2][1] - d[1][1] * d[2][0]);
        double scale = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) scale = std::max(scale, std::fabs(d[a][c]));
        if (!(std::fabs(det) > 1e-12 * scale * scale * scale))
            return "qpat_mesh: degenerate tetrahedron " + std::to_string(e);
    }

    // ---- boundary faces, canonical order (sorted caller triples, lexicographic)
    {
        std::vector<Face> f(4 * E);
        static const int omit[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
        for (int64_t e = 0; e < E; ++e)
            for (int k = 0; k < 4; ++k) {
                Face& q = f[4 * e + k];
                for (int a = 0; a < 3; ++a) q.v[a] = tets[4 * e + omit[k][a]];
                std::sort(q.v, q.v + 3);
                q.tet = int32_t(e);
            }
        std::sort(f.begin(), f.end(), [](const Face& a, const Face& b) {
            if (a.v[0] != b.v[0]) return a.v[0] < b.v[0];
            if (a.v[1] != b.v[1]) return a.v[1] < b.v[1];
            return a.v[2] < b.v[2];
        });
        auto same = [](const Face& a, const Face& b) {
            return a.v[0] == b.v[0] && a.v[1] == b.v[1] && a.v[2] == b.v[2];
        };
        for (size_t i = 0; i < f.size();) {
            size_t j = i + 1;
            while (j < f.size() && same(f[i], f[j])) ++j;
            if (j - i > 2) return "qpat_mesh: a face is shared by more than two tets";
            if (j - i == 1)
                for (int a = 0; a < 3; ++a) m.faces_caller.push_back(f[i].v[a]);
            i = j;
        }
        m.F = int64_t(m.faces_caller.size() / 3);
    }

    // ---- Morton order of the nodes
    double lo[3] = {xyz[0], xyz[1], xyz[2]}, hi[3] = {xyz[0], xyz[1], xyz[2]};
    for (int64_t i = 0; i < N; ++i)
        for (int c = 0; c < 3; ++c) {
            lo[c] = std::min(lo[c], xyz[3 * i + c]);
            hi[c] = std::max(hi[c], xyz[3 * i + c]);
        }
    double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
    m.extent = ext;
    std::vector<std::pair<uint64_t, int32_t>> key(N);
    for (int64_t i = 0; i < N; ++i) {
        uint64_t code = 0;
        for (int c = 0; c < 3; ++c) {
            double s = (xyz[3 * i + c] - lo[c]) / ext;
            uint64_t q = uint64_t(std::min(std::max(s, 0.0), 1.0) * double((1u << 21) - 1) + 0.5);
            code |= spread3(q) << c;
        }
        key[i] = {code, int32_t(i)};
    }
    std::sort(key.begin(), key.end());
    m.perm.resize(N);
    m.iperm.resize(N);
    for (int64_t i = 0; i < N; ++i) {
        m.perm[i] = key[i].second;
        m.iperm[key[i].second] = int32_t(i);
    }
    m.xyz.resize(3 * N);
    for (int64_t i = 0; i < N; ++i)
        for (int c = 0; c < 3; ++c) m.xyz[3 * i + c] = xyz[3 * m.perm[i] + c];
    m.tets.resize(4 * E);
    for (int64_t i = 0; i < 4 * E; ++i) m.tets[i] = m.iperm[tets[i]];
    m.faces_lib.resize(3 * m.F);
    m.farea.resize(m.F);
    for (int64_t f = 0; f < m.F; ++f) {
        for (int a = 0; a < 3; ++a) m.faces_lib[3 * f + a] = m.iperm[m.faces_caller[3 * f + a]];
        const double* p0 = &m.xyz[3 * m.faces_lib[3 * f + 0]];
        const double* p1 = &m.xyz[3 * m.faces_lib[3 * f + 1]];
        const double* p2 = &m.xyz[3 * m.faces_lib[3 * f + 2]];
        double a[3], b[3];
        for (int c = 0; c < 3; ++c) {
            a[c] = p1[c] - p0[c];
            b[c] = p2[c] - p0[c];
        }
        double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2],
               cz = a[0] * b[1] - a[1] * b[0];
        m.farea[f] = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    }

    // ---- node -> incident tets, node -> incident boundary faces
    std::vector<int32_t> nt_ptr(N + 1, 0), nt(4 * E);
    for (int64_t i = 0; i < 4 * E; ++i) nt_ptr[m.tets[i] + 1]++;
    for (int64_t i = 0; i < N; ++i) nt_ptr[i + 1] += nt_ptr[i];
    {
        std::vector<int32_t> fill(nt_ptr.begin(), nt_ptr.end() - 1);
        for (int64_t e = 0; e < E; ++e)
            for (int k = 0; k < 4; ++k) nt[fill[m.tets[4 * e + k]]++] = int32_t(e);
    }
    std::vector<int32_t> nf_ptr(N + 1, 0), nf(3 * m.F);
    for (int64_t i = 0; i < 3 * m.F; ++i) nf_ptr[m.faces_lib[i] + 1]++;
    for (int64_t i = 0; i < N; ++i) nf_ptr[i + 1] += nf_ptr[i];
    {
        std::vector<int32_t> fill(nf_ptr.begin(), nf_ptr.end() - 1);
        for (int64_t f = 0; f < m.F; ++f)
            for (int k = 0; k < 3; ++k) nf[fill[m.faces_lib[3 * f + k]]++] = int32_t(f);
    }
    m.nface_ptr = nf_ptr;
    m.nface = nf;

    // ---- patches: P balanced ranges of whole 32-node slices.  With
    // patch_multiple > 0 the count is rounded up to a multiple of it (the
    // resident CTA count of the persistent solver) so that every CTA owns the
    // same number of patches and the patches differ by at most one slice.
    const int64_t S = (N + 31) / 32;
    int64_t Pl = (N + patch_nodes - 1) / patch_nodes;
    if (patch_multiple > 0) Pl = ((Pl + patch_multiple - 1) / patch_multiple) * patch_multiple;
    Pl = std::max<int64_t>(1, std::min(Pl, S));
    const int P = int(Pl);
    m.P = P;
    m.own_begin.resize(P + 1);
    m.patch_of_slice.resize(S);
    for (int p = 0; p <= P; ++p) m.own_begin[p] = int32_t(std::min<int64_t>(32 * ((S * p) / P), N));
    for (int p = 0; p < P; ++p)
        for (int64_t s = (S * p) / P; s < (S * (p + 1)) / P; ++s) m.patch_of_slice[s] = p;
    m.node_ptr.assign(1, 0);
    m.tet_ptr.assign(1, 0);
    m.face_ptr.assign(1, 0);
    m.tcol_beg.assign(1, 0);
    m.fcol_beg.assign(1, 0);
    m.tcol_off.clear();
    m.fcol_off.clear();
    std::vector<int32_t> tet_stamp(E, -1), face_stamp(m.F, -1), node_local(N, -1);
    std::vector<int32_t> ptets, pfaces, halo;
    std::vector<std::vector<uint16_t>> rows(N);   // local column ids of every row
    std::vector<std::vector<uint16_t>> srows(N);  // the subset with a non-zero gradient coupling
    for (int p = 0; p < P; ++p) {
        const int32_t b = m.own_begin[p], e = m.own_begin[p + 1];
        const int nown = e - b;
        ptets.clear();
        pfaces.clear();
        halo.clear();
        for (int32_t g = b; g < e; ++g) {
            for (int32_t q = nt_ptr[g]; q < nt_ptr[g + 1]; ++q) {
                int32_t t = nt[q];
                if (tet_stamp[t] != p) {
                    tet_stamp[t] = p;
                    ptets.push_back(t);
                }
            }
            for (int32_t q = nf_ptr[g]; q < nf_ptr[g + 1]; ++q) {
                int32_t f = nf[q];
                if (face_stamp[f] != p) {
                    face_stamp[f] = p;
                    pfaces.push_back(f);
                }
            }
        }
        for (int32_t g = b; g < e; ++g) node_local[g] = g - b;
        for (int32_t t : ptets)
            for (int k = 0; k < 4; ++k) {
                int32_t g = m.tets[4 * t + k];
                if ((g < b || g >= e) && node_local[g] == -1) {
                    node_local[g] = -2;  // seen
                    halo.push_back(g);
                }
            }
        std::sort(halo.begin(), halo.end());
        for (size_t i = 0; i < halo.size(); ++i) node_local[halo[i]] = int32_t(nown + i);
        const int ntouch = nown + int(halo.size());
        if (ntouch > 65535) return "qpat_mesh: a patch touches more than 65535 nodes";
        for (int32_t g = b; g < e; ++g) m.nodes.push_back(g);
        for (int32_t g : halo) m.nodes.push_back(g);
        // greedy colours: a tet (face) takes the lowest colour that no earlier
        // tet (face) sharing one of its owned vertices has; then the lists are
        // sorted by colour (stable, so the order inside a colour is kept)
        auto colour = [&](std::vector<int32_t>& items, int nv, const int32_t* conn, std::vector<int32_t>& beg,
                          std::vector<int32_t>& off, int32_t base) -> int {
            std::vector<std::array<uint64_t, 4>> used(size_t(nown), std::array<uint64_t, 4>{0, 0, 0, 0});
            std::vector<int> col(items.size());
            int ncol = 0;
            for (size_t i = 0; i < items.size(); ++i) {
                std::array<uint64_t, 4> u{0, 0, 0, 0};
                for (int k = 0; k < nv; ++k) {
                    const int32_t l = node_local[conn[size_t(nv) * items[i] + k]];
                    if (l >= 0 && l < nown)
                        for (int w = 0; w < 4; ++w) u[w] |= used[l][w];
                }
                int c = 0;
                while (c < 256 && ((u[c >> 6] >> (c & 63)) & 1u)) ++c;
                if (c == 256) return -1;
                col[i] = c;
                ncol = std::max(ncol, c + 1);
                for (int k = 0; k < nv; ++k) {
                    const int32_t l = node_local[conn[size_t(nv) * items[i] + k]];
                    if (l >= 0 && l < nown) used[l][c >> 6] |= uint64_t(1) << (c & 63);
                }
            }
            std::vector<int32_t> sorted;
            sorted.reserve(items.size());
            int32_t pos = base;
            for (int c = 0; c < ncol; ++c) {
                off.push_back(pos);
                for (size_t i = 0; i < items.size(); ++i)
                    if (col[i] == c) {
                        sorted.push_back(items[i]);
                        ++pos;
                    }
            }
            off.push_back(pos);
            beg.push_back(int32_t(off.size()));
            items.swap(sorted);
            return ncol;
        };
        const int ntc = colour(ptets, 4, m.tets.data(), m.tcol_beg, m.tcol_off, int32_t(m.tet_loc.size() / 4));
        const int nfc = colour(pfaces, 3, m.faces_lib.data(), m.fcol_beg, m.fcol_off, int32_t(m.face_loc.size() / 4));
        if (ntc < 0 || nfc < 0) return "qpat_mesh: more than 256 element colours in a patch";
        m.max_tcolors = std::max(m.max_tcolors, ntc);
        for (int32_t t : ptets) {
            int32_t lv[4];
            for (int k = 0; k < 4; ++k) {
                lv[k] = node_local[m.tets[4 * t + k]];
                m.tet_loc.push_back(uint16_t(lv[k]));
            }
            // gradient couplings of the tet: cofactor vectors c_k (grad lambda_k
            // times the determinant); a pair couples in a stiffness operator iff
            // c_a . c_b is not zero up to rounding
            double cof[4][3];
            {
                const double* q0 = &m.xyz[3 * m.tets[4 * t]];
                double ed[3][3];
                for (int k = 1; k < 4; ++k)
                    for (int d = 0; d < 3; ++d) ed[k - 1][d] = m.xyz[3 * m.tets[4 * t + k] + d] - q0[d];
                auto cross = [](const double* x, const double* y, double* z) {
                    z[0] = x[1] * y[2] - x[2] * y[1];
                    z[1] = x[2] * y[0] - x[0] * y[2];
                    z[2] = x[0] * y[1] - x[1] * y[0];
                };
                cross(ed[1], ed[2], cof[1]);
                cross(ed[2], ed[0], cof[2]);
                cross(ed[0], ed[1], cof[3]);
                for (int d = 0; d < 3; ++d) cof[0][d] = -(cof[1][d] + cof[2][d] + cof[3][d]);
            }
            for (int a = 0; a < 4; ++a)
                if (lv[a] < nown)
                    for (int c = 0; c < 4; ++c) {
                        rows[b + lv[a]].push_back(uint16_t(lv[c]));
                        const double dot = cof[a][0] * cof[c][0] + cof[a][1] * cof[c][1] + cof[a][2] * cof[c][2];
                        const double na = std::sqrt(cof[a][0] * cof[a][0] + cof[a][1] * cof[a][1] + cof[a][2] * cof[a][2]);
                        const double nc = std::sqrt(cof[c][0] * cof[c][0] + cof[c][1] * cof[c][1] + cof[c][2] * cof[c][2]);
                        if (a == c || std::fabs(dot) > 1e-12 * na * nc) srows[b + lv[a]].push_back(uint16_t(lv[c]));
                    }
        }
        for (int32_t g = b; g < e; ++g) {
            for (auto* rp : {&rows[g], &srows[g]}) {
                auto& r = *rp;
                std::sort(r.begin(), r.end());
                r.erase(std::unique(r.begin(), r.end()), r.end());
            }
            if (rows[g].size() > 255) return "qpat_mesh: a node has more than 254 neighbours";
        }
        for (int32_t f : pfaces) {
            for (int k = 0; k < 3; ++k) m.face_loc.push_back(uint16_t(node_local[m.faces_lib[3 * f + k]]));
            m.face_loc.push_back(0);
            m.pface_area.push_back(m.farea[f]);
        }
        m.node_ptr.push_back(int32_t(m.nodes.size()));
        m.tet_ptr.push_back(int32_t(m.tet_loc.size() / 4));
        m.face_ptr.push_back(int32_t(m.face_loc.size() / 4));
        m.max_touched = std::max(m.max_touched, ntouch);
        m.max_own = std::max(m.max_own, nown);
        m.max_ptets = std::max(m.max_ptets, int(ptets.size()));
        m.max_pfaces = std::max(m.max_pfaces, int(pfaces.size()));
        for (int32_t g = b; g < e; ++g) node_local[g] = -1;
        for (int32_t g : halo) node_local[g] = -1;
    }

    // ---- sliced ELLPACK patterns (slices never straddle patches: patch_nodes % 32 == 0)
    m.nslices = (N + 31) / 32;
    auto build_sell = [&](const std::vector<std::vector<uint16_t>>& rr, std::vector<int64_t>& ptr,
                          std::vector<uint16_t>& col, std::vector<uint8_t>& len, std::vector<int32_t>& diag,
                          int& wmax) -> const char* {
        ptr.assign(m.nslices + 1, 0);
        len.assign(size_t(32) * m.nslices, 0);
        diag.resize(N);
        wmax = 0;
        for (int64_t s = 0; s < m.nslices; ++s) {
            size_t w = 0;
            for (int64_t g = 32 * s; g < std::min<int64_t>(N, 32 * s + 32); ++g) w = std::max(w, rr[g].size());
            ptr[s + 1] = ptr[s] + int64_t(w);
            wmax = std::max(wmax, int(w));
        }
        col.assign(size_t(32) * ptr[m.nslices], 0);
        for (int64_t s = 0; s < m.nslices; ++s) {
            const int64_t w = ptr[s + 1] - ptr[s];
            for (int lane = 0; lane < 32; ++lane) {
                const int64_t g = 32 * s + lane;
                uint16_t self = 0;
                if (g < N) {
                    const int p = m.patch_of_slice[g >> 5];
                    self = uint16_t(g - m.own_begin[p]);
                    len[g] = uint8_t(rr[g].size());
                    diag[g] = -1;
                }
                for (int64_t k = 0; k < w; ++k) {
                    uint16_t c = self;
                    if (g < N && k < int64_t(rr[g].size())) c = rr[g][k];
                    col[(ptr[s] + k) * 32 + lane] = c;
                    if (g < N && k < int64_t(rr[g].size()) && c == self) diag[g] = int32_t(k);
                }
                if (g < N && diag[g] < 0) return "qpat_mesh: a node belongs to no tetrahedron";
            }
        }
        return nullptr;
    };
    if (const char* err = build_sell(rows, m.sell_ptr, m.sell_col, m.sell_len, m.sell_diag, m.sell_wmax)) return err;
    if (const char* err = build_sell(srows, m.psell_ptr, m.psell_col, m.psell_len, m.psell_diag, m.psell_wmax))
        return err;
    return "";
}

void flux_patch_host(const HostMesh& m, const double c[3], const double n[3],
                     double half_w, double amp, double* flux_face) {
    const double tol = 1e-9 * m.extent;
    double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double u[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
    for (int64_t f = 0; f < m.F; ++f) {
        bool on = true;
        double cen[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) {
            const double* p = &m.xyz[3 * m.faces_lib[3 * f + a]];
            double d = (p[0] - c[0]) * u[0] + (p[1] - c[1]) * u[1] + (p[2] - c[2]) * u[2];
            if (std::fabs(d) > tol) on = false;
            for (int k = 0; k < 3; ++k) cen[k] += p[k] / 3.0;
        }
        double r[3] = {cen[0] - c[0], cen[1] - c[1], cen[2] - c[2]};
        double rn = r[0] * u[0] + r[1] * u[1] + r[2] * u[2];
        double inf = 0.0;
        for (int k = 0; k < 3; ++k) inf = std::max(inf, std::fabs(r[k] - rn * u[k]));
        flux_face[f] = (on && inf <= half_w + tol) ? amp : 0.0;
    }
}

void flux_side_host(const HostMesh& m, const double c[3], const double axis[3], const double ref[3],
                    double radius, double theta0, double half_w, double amp, double* flux_face) {
    const double tol = 1e-9 * m.extent;
    const double pi = 3.14159265358979323846;
    auto dot = [](const double* x, const double* y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; };
    // orthonormal frame: u along the axis, e1 = ref without its axial part, e2 = u x e1
    const double an = std::sqrt(dot(axis, axis));
    const double u[3] = {axis[0] / an, axis[1] / an, axis[2] / an};
    const double ru = dot(ref, u);
    double e1[3] = {ref[0] - ru * u[0], ref[1] - ru * u[1], ref[2] - ru * u[2]};
    const double e1n = std::sqrt(dot(e1, e1));
    for (double& v : e1) v /= e1n;
    const double e2[3] = {u[1] * e1[2] - u[2] * e1[1], u[2] * e1[0] - u[0] * e1[2], u[0] * e1[1] - u[1] * e1[0]};
    for (int64_t f = 0; f < m.F; ++f) {
        bool side = true;
        double cen[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) {
            const double* p = &m.xyz[3 * m.faces_lib[3 * f + a]];
            const double d[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
            const double t = dot(d, u);
            const double rr[3] = {d[0] - t * u[0], d[1] - t * u[1], d[2] - t * u[2]};
            if (std::fabs(std::sqrt(dot(rr, rr)) - radius) > tol) side = false;
            for (int k = 0; k < 3; ++k) cen[k] += d[k] / 3.0;
        }
        double val = 0.0;
        if (side) {
            // polar angle of the centroid, its offset from theta0 wrapped to (-pi, pi]
            double dth = std::atan2(dot(cen, e2), dot(cen, e1)) - theta0;
            dth = std::remainder(dth, 2.0 * pi);
            if (dth <= -pi) dth += 2.0 * pi;
            if (std::fabs(dth) <= half_w) val = amp * std::cos(0.5 * pi * dth / half_w);
        }
        flux_face[f] = val;
    }
}

}  // namespace qpat
