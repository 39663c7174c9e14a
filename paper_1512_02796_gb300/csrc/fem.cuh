// Element-level device code shared by every patch kernel.
//
// All element operators are written with the cofactor vectors of a tet:
// with edges e_j = p_j - p_0 (j = 1..3), c_1 = e_2 x e_3, c_2 = e_3 x e_1,
// c_3 = e_1 x e_2, c_0 = -(c_1 + c_2 + c_3) and det = e_1 . c_1, the P1
// barycentric gradients are grad(lambda_i) = c_i / det and |T| = |det| / 6.
// For a P1 field x_h on the tet, G_x = sum_j x_j c_j = sum_{j>=1} (x_j - x_0) c_j
// is det * grad(x_h), so |T| grad(lambda_i) . grad(x_h) = (c_i . G_x) / (6 |det|).
//
// The mass term with a P1 coefficient mu uses the exact integral of
// lambda_i lambda_j lambda_k (|T|/20, /60, /120 for 3, 2, 1 distinct
// indices), summed in closed form:
//   (M(mu) x)_i = |T|/120 [ (S_mu + mu_i)(S_x + x_i) + mu.x + mu_i x_i ],
// S_mu, S_x the sums over the 4 vertices.  The Robin boundary term
// 1/2 integral x v (Appendix weak form) on a face F adds |F|/24 (S_x^F + x_i).
#pragma once

#include <cuda_runtime.h>

#include "qpat_internal.h"

namespace qpat {

// OP_K / OP_PRIOR: matrix-free element operators recomputed from the
// geometry on every apply.  OP_CSR1 / OP_CSR2: the same operators assembled
// once per linearisation into the sliced-ELLPACK pattern of the mesh (one
// value array shared by all right-hand sides, or one per prior block).
enum OpKind { OP_K = 0, OP_PRIOR = 1, OP_CSR1 = 2, OP_CSR2 = 3 };

constexpr int kThreads = 256;

template <typename T>
struct OpParams {
    const T* c1;     // OP_K: nodal kappa (or kappa o s1); OP_PRIOR: u for block 0 (kappa_tilde)
    const T* c2;     // OP_K: nodal mu (or mu o s2);      OP_PRIOR: u for block 1 (mu_tilde)
    T inv_T2;        // OP_PRIOR: 1 / T^2 of the Perona-Malik weight (Eq. (10), (14))
    T scale1;        // OP_PRIOR: b / a on block 1 (Eq. (16))
    T delta;         // OP_PRIOR: delta of M_delta (Eq. (19))
    int robin;       // OP_K: include the Robin boundary term
    const T* v0;     // OP_CSR*: assembled values (block 0 / all RHS)
    const T* v1;     // OP_CSR2: assembled values of block 1
    int prior_kind = 0;   // OP_PRIOR: r(t) of the prior (see prior_weight)
    T prior_q = T(1);     // OP_PRIOR: exponent q of the smoothed TV^q prior
};

// Lagged-diffusivity weight r'(t)/t of the prior R(u) = integral r(|grad u|)
// (Eq. (9)) at t^2 = g2; the lagged step (Eq. (14)) uses it per tet.
//   kind 0, Perona-Malik (Eq. (10)): r(t) = T^2/2 log(1 + t^2/T^2)  ->  1 / (1 + t^2/T^2)
//   kind 1, smoothed TV^q (named after Eq. (10)): r(t) = (t^2 + T^2)^(q/2) / q
//                                              ->  (t^2 + T^2)^(q/2 - 1)
// (q = 1 is smoothed total variation; q = 2 gives weight 1, the plain Laplacian.)
template <typename T>
__host__ __device__ inline T prior_weight(int kind, T g2, T inv_T2, T q) {
    if (kind == 0) return T(1) / (T(1) + g2 * inv_T2);
    const T e = q * T(0.5) - T(1);
    return e == T(0) ? T(1) : pow(g2 + T(1) / inv_T2, e);
}

// Slot of local column c in library row g of the sliced-ELLPACK pattern.
__device__ __forceinline__ int64_t sell_slot(const MeshDev& m, int g, int c) {
    const int64_t base = m.sell_ptr[g >> 5];
    const int lane = g & 31, len = m.sell_len[g];
    for (int k = 0; k < len; ++k) {
        const int64_t idx = (base + k) * 32 + lane;
        if (m.sell_col[idx] == c) return idx;
    }
    return -1;
}

// Rows [ob, ob + nown) of an assembled operator applied to staged input
// xin (touched x R, node-major), R right-hand sides; result written by
// `emit(i, r, value)` with i the owned local row.
template <typename T, int R, int NV, class Emit>
__device__ __forceinline__ void csr_rows(const MeshDev& m, int ob, int nown, const T* __restrict__ v0,
                                         const T* __restrict__ v1, const T* xin, Emit emit) {
    for (int i = threadIdx.x; i < nown; i += blockDim.x) {
        const int g = ob + i;
        const int64_t base = m.sell_ptr[g >> 5] * 32 + (g & 31);
        const int len = m.sell_len[g];
        T acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = T(0);
        for (int k = 0; k < len; ++k) {
            const int64_t idx = base + int64_t(k) * 32;
            const int c = m.sell_col[idx];
            if constexpr (NV == 1) {
                const T v = __ldg(v0 + idx);
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] += v * xin[c * R + r];
            } else {
                static_assert(R == 2, "two value sets mean two blocks");
                acc[0] += __ldg(v0 + idx) * xin[c * 2];
                acc[1] += __ldg(v1 + idx) * xin[c * 2 + 1];
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) emit(i, r, acc[r]);
    }
}

template <typename T>
__device__ __forceinline__ void tet_cofactors(const T p[4][3], T c[4][3], T& ad) {
    T e1[3], e2[3], e3[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        e1[k] = p[1][k] - p[0][k];
        e2[k] = p[2][k] - p[0][k];
        e3[k] = p[3][k] - p[0][k];
    }
    c[1][0] = e2[1] * e3[2] - e2[2] * e3[1];
    c[1][1] = e2[2] * e3[0] - e2[0] * e3[2];
    c[1][2] = e2[0] * e3[1] - e2[1] * e3[0];
    c[2][0] = e3[1] * e1[2] - e3[2] * e1[1];
    c[2][1] = e3[2] * e1[0] - e3[0] * e1[2];
    c[2][2] = e3[0] * e1[1] - e3[1] * e1[0];
    c[3][0] = e1[1] * e2[2] - e1[2] * e2[1];
    c[3][1] = e1[2] * e2[0] - e1[0] * e2[2];
    c[3][2] = e1[0] * e2[1] - e1[1] * e2[0];
#pragma unroll
    for (int k = 0; k < 3; ++k) c[0][k] = -(c[1][k] + c[2][k] + c[3][k]);
    T det = e1[0] * c[1][0] + e1[1] * c[1][1] + e1[2] * c[1][2];
    ad = fabs(det);
}

// G_x = sum_{j>=1} (x_j - x_0) c_j
template <typename T>
__device__ __forceinline__ void grad_vec(const T c[4][3], const T x[4], T G[3]) {
    const T d1 = x[1] - x[0], d2 = x[2] - x[0], d3 = x[3] - x[0];
#pragma unroll
    for (int k = 0; k < 3; ++k) G[k] = d1 * c[1][k] + d2 * c[2][k] + d3 * c[3][k];
}

// y_i = sk (c_i . G) for i = 0..3 (c_0 term from the others)
template <typename T>
__device__ __forceinline__ void stiff_rows(const T c[4][3], const T G[3], T sk, T y[4]) {
    T s1 = sk * (c[1][0] * G[0] + c[1][1] * G[1] + c[1][2] * G[2]);
    T s2 = sk * (c[2][0] * G[0] + c[2][1] * G[1] + c[2][2] * G[2]);
    T s3 = sk * (c[3][0] * G[0] + c[3][1] * G[1] + c[3][2] * G[2]);
    y[0] = -(s1 + s2 + s3);
    y[1] = s1;
    y[2] = s2;
    y[3] = s3;
}

// y_i += vm [ (S_m + m_i)(S_x + x_i) + m.x + m_i x_i ],  vm = |T| / 120
template <typename T>
__device__ __forceinline__ void mass_rows_add(const T m[4], T Sm, const T x[4], T vm, T y[4]) {
    const T Sx = x[0] + x[1] + x[2] + x[3];
    const T mx = m[0] * x[0] + m[1] * x[1] + m[2] * x[2] + m[3] * x[3];
#pragma unroll
    for (int i = 0; i < 4; ++i) y[i] += vm * ((Sm + m[i]) * (Sx + x[i]) + mx + m[i] * x[i]);
}

// Shared-memory staging of one patch.  Strides use the mesh-wide maxima so
// that the layout is fixed for the kernel.
template <typename T, int R>
struct PatchSmem {
    T* px;
    T* py;
    T* pz;
    T* c1;
    T* c2;
    T* xin;   // touched x R, node-major
    T* yout;  // owned x R, node-major
    __device__ void carve(T* base, int MT, int MO) {
        px = base;
        py = px + MT;
        pz = py + MT;
        c1 = pz + MT;
        c2 = c1 + MT;
        xin = c2 + MT;
        yout = xin + size_t(MT) * R;
        (void)MO;
    }
    static size_t bytes(int MT, int MO) { return sizeof(T) * (size_t(MT) * (5 + R) + size_t(MO) * R); }
};

template <typename T>
__device__ __forceinline__ const T* xyz_of(const MeshDev& m);
template <>
__device__ __forceinline__ const double* xyz_of<double>(const MeshDev& m) { return m.xyz64; }
template <>
__device__ __forceinline__ const float* xyz_of<float>(const MeshDev& m) { return m.xyz32; }

template <typename T>
__device__ __forceinline__ T face_area_of(const MeshDev& m, int i);
template <>
__device__ __forceinline__ double face_area_of<double>(const MeshDev& m, int i) { return __ldg(m.pface_area64 + i); }
template <>
__device__ __forceinline__ float face_area_of<float>(const MeshDev& m, int i) { return __ldg(m.pface_area32 + i); }

// Stage coordinates and the two nodal coefficients of the touched nodes.
template <typename T, int R>
__device__ __forceinline__ void stage_static(const MeshDev& m, int nb, int nt, const PatchSmem<T, R>& s,
                                             const OpParams<T>& op) {
    const T* xyz = xyz_of<T>(m);
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
        const int g = __ldg(m.nodes + nb + i);
        s.px[i] = __ldg(xyz + 3 * g + 0);
        s.py[i] = __ldg(xyz + 3 * g + 1);
        s.pz[i] = __ldg(xyz + 3 * g + 2);
        s.c1[i] = __ldg(op.c1 + g);
        s.c2[i] = __ldg(op.c2 + g);
    }
}

template <typename T, int R>
__device__ __forceinline__ void load_tet(const PatchSmem<T, R>& s, const ushort4 lv, T p[4][3]) {
    const int v[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        p[a][0] = s.px[v[a]];
        p[a][1] = s.py[v[a]];
        p[a][2] = s.pz[v[a]];
    }
}

// f(e) for every element of patch p, one colour after the other with a
// block-wide barrier after each (beg / off: HostMesh's tcol_* or fcol_*).
// Elements of one colour share no owned vertex, so the sums into owned rows
// need no atomics and add up in the same order on every run.
template <class F>
__device__ __forceinline__ void for_each_coloured(const int* beg, const int* off, int p, F&& f) {
    const int j0 = __ldg(beg + p), j1 = __ldg(beg + p + 1);
    for (int j = j0; j + 1 < j1; ++j) {
        const int e1 = __ldg(off + j + 1);
        for (int e = __ldg(off + j) + threadIdx.x; e < e1; e += blockDim.x) f(e);
        __syncthreads();
    }
}

// y += v into an owned-row accumulator: plain in a coloured loop, atomic otherwise
template <bool kColoured, typename T>
__device__ __forceinline__ void acc_add(T* y, T v) {
    if constexpr (kColoured) {
        *y += v;
    } else {
        atomicAdd(y, v);
    }
}

// Element loop of one patch: yout[owned] += (operator) xin.  xin, the
// coordinates and the coefficients must be staged and yout zeroed.
// kColoured: colour by colour (run-to-run identical sums, a barrier per
// colour); otherwise all elements at once with shared-memory atomics (the
// matrix-free FP32 PCG, where a barrier per colour and iteration would cost
// more than it buys).
template <typename T, int R, int OP, bool kColoured = false>
__device__ __forceinline__ void patch_elements(const MeshDev& m, int p, int nown, const PatchSmem<T, R>& s,
                                               const OpParams<T>& op) {
    auto tet = [&](int t) {
        const ushort4 lv = m.tet_loc[t];
        const int v[4] = {lv.x, lv.y, lv.z, lv.w};
        T pc[4][3], c[4][3], ad;
        load_tet(s, lv, pc);
        tet_cofactors(pc, c, ad);
        if constexpr (OP == OP_K) {
            T mu[4], Sm = T(0), ks = T(0);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                ks += s.c1[v[a]];
                mu[a] = s.c2[v[a]];
                Sm += mu[a];
            }
            const T sk = ks / (T(24) * ad);  // (S_kappa / 4) / (6 |det|)
            const T vm = ad / T(720);        // |T| / 120
#pragma unroll
            for (int r = 0; r < R; ++r) {
                T x[4], G[3], y[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) x[a] = s.xin[v[a] * R + r];
                grad_vec(c, x, G);
                stiff_rows(c, G, sk, y);
                mass_rows_add(mu, Sm, x, vm, y);
#pragma unroll
                for (int a = 0; a < 4; ++a)
                    if (v[a] < nown) acc_add<kColoured>(&s.yout[v[a] * R + r], y[a]);
            }
        } else {
            static_assert(R == 2, "the prior operator has two blocks");
            const T inv6ad = T(1) / (T(6) * ad);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const T* uc = r == 0 ? s.c1 : s.c2;
                T u[4], Gu[3], x[4], G[3], y[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    u[a] = uc[v[a]];
                    x[a] = s.xin[v[a] * 2 + r];
                }
                grad_vec(c, u, Gu);
                // |grad u|^2 = |G_u|^2 / det^2 ; c_T = r'(|grad u|) / |grad u|
                const T g2 = (Gu[0] * Gu[0] + Gu[1] * Gu[1] + Gu[2] * Gu[2]) / (ad * ad);
                const T cT = prior_weight<T>(op.prior_kind, g2, op.inv_T2, op.prior_q);
                const T sk = (r == 0 ? T(1) : op.scale1) * cT * inv6ad;
                grad_vec(c, x, G);
                stiff_rows(c, G, sk, y);
#pragma unroll
                for (int a = 0; a < 4; ++a)
                    if (v[a] < nown) acc_add<kColoured>(&s.yout[v[a] * 2 + r], y[a]);
            }
        }
    };
    if constexpr (kColoured) {
        for_each_coloured(m.tcol_beg, m.tcol_off, p, tet);
    } else {
        const int tb = __ldg(m.tet_ptr + p), te = __ldg(m.tet_ptr + p + 1);
        for (int t = tb + threadIdx.x; t < te; t += blockDim.x) tet(t);
    }
    if constexpr (OP == OP_K) {
        if (op.robin) {
            auto face = [&](int f) {
                const ushort4 lv = m.face_loc[f];
                const int v[3] = {lv.x, lv.y, lv.z};
                const T w = face_area_of<T>(m, f) / T(24);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    T x[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) x[a] = s.xin[v[a] * R + r];
                    const T Sx = x[0] + x[1] + x[2];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        if (v[a] < nown) acc_add<kColoured>(&s.yout[v[a] * R + r], w * (Sx + x[a]));
                }
            };
            if constexpr (kColoured) {
                for_each_coloured(m.fcol_beg, m.fcol_off, p, face);
            } else {
                const int fb = __ldg(m.face_ptr + p), fe = __ldg(m.face_ptr + p + 1);
                for (int f = fb + threadIdx.x; f < fe; f += blockDim.x) face(f);
            }
        }
    }
}

// Deterministic block reduction of NS doubles per thread; result valid in
// thread 0 (out[s]).  scratch: at least 32 * NS doubles of shared memory.
template <int NS>
__device__ __forceinline__ void block_reduce(double (&v)[NS], double* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[s] += __shfl_down_sync(0xffffffffu, v[s], o);
    }
    if (lane == 0)
        for (int s = 0; s < NS; ++s) scratch[warp * NS + s] = v[s];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            double a = 0.0;
            for (int w = 0; w < nw; ++w) a += scratch[w * NS + s];
            v[s] = a;
        }
    }
    __syncthreads();
}

}  // namespace qpat
