// Device side of the smoothed-aggregation multigrid preconditioner (see
// amg.h): the numeric set-up of the hierarchy from the assembled FP64
// operator, the V-cycle, and the conjugate-gradient driver that uses it.
//
// Layout: vectors are node-major with R right-hand sides interleaved
// (x[i * R + r]), as everywhere in the library.  The K operator has one value
// set for all right-hand sides; M_delta has two (its blocks, R = 2, column r
// uses set r), and every level of its hierarchy keeps two sets over one
// pattern.  All sums run in a fixed order: results are identical from run
// to run.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "abi_internal.h"
#include "amg.h"

namespace qpat {

struct SellDev {
    int64_t n = 0;
    const int64_t* ptr = nullptr;
    const int32_t* col = nullptr;
    const uint16_t* len = nullptr;
    int64_t entries = 0;
    int maxlen = 0;
    int rowmajor = 0;  // layout (see SellPattern); row-major rows are applied by 8 lanes each
};

struct LevelDev {
    SellDev A;
    const int32_t* diag = nullptr;
    int64_t nc = 0;
    SellDev P;
    const uint16_t* a2p = nullptr;
    const uint16_t* pself = nullptr;
    const int64_t* ap_ptr = nullptr;
    const int32_t* ap_col = nullptr;
    const int64_t* ap_sptr = nullptr;
    const uint16_t* ap_slot = nullptr;
    int64_t ap_nnz = 0;
    int ap_maxlen = 0;
    SellDev R;
    const int64_t* r_src = nullptr;
    const int64_t* g_ptr = nullptr;
    const uint16_t* g_slot = nullptr;
};

namespace {

__device__ __forceinline__ int64_t spos(const SellDev& S, int64_t row, int k) {
    return S.rowmajor ? S.ptr[row] + k : (S.ptr[row >> 5] + k) * 32 + (row & 31);
}

// ---------------------------------------------------------------- set-up kernels

// Inverse diagonal (n x NV, interleaved) and the Gershgorin bound
// max_i sum_j |a_ij| / a_ii of D^-1 A per value set (hi must start at 0; the
// bound is >= 1, so the bits of the positive doubles order like integers).
template <int NV>
__global__ void __launch_bounds__(256) k_dinv_hi(SellDev A, const int32_t* diag, const double* v0, const double* v1,
                                                 double* dinv, double* hi) {
    __shared__ double bmax[NV][8];
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double ratio = 0.0;
        if (i < A.n) {
            const double* val = v == 0 ? v0 : v1;
            const int L = A.len[i];
            double s = 0.0;
            for (int k = 0; k < L; ++k) s += fabs(val[spos(A, i, k)]);
            const double d = val[spos(A, i, diag[i])];
            dinv[i * NV + v] = 1.0 / d;
            ratio = s / fabs(d);
        }
        // the largest ratio of the block (max is exact in any order), then one atomic per block
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ratio = fmax(ratio, __shfl_xor_sync(0xffffffffu, ratio, o));
        if (lane == 0) bmax[v][warp] = ratio;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double m = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) m = fmax(m, bmax[threadIdx.x][w]);
        atomicMax(reinterpret_cast<unsigned long long*>(hi + threadIdx.x), __double_as_longlong(m));
    }
}

// P = (I - omega D^-1 A) P_tent, omega = 4 / (3 hi): row i of P from row i of A.
template <int NV>
__global__ void k_prolong(SellDev A, SellDev P, const uint16_t* a2p, const uint16_t* pself, const double* v0,
                          const double* v1, const double* dinv, const double* hi, double* p0, double* p1) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= A.n) return;
    const int L = A.len[i], LP = P.len[i];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const double* val = v == 0 ? v0 : v1;
        double* pv = v == 0 ? p0 : p1;
        const double w = (4.0 / 3.0) / hi[v] * dinv[i * NV + v];
        for (int k = 0; k < LP; ++k) pv[spos(P, i, k)] = 0.0;
        pv[spos(P, i, pself[i])] = 1.0;
        for (int k = 0; k < L; ++k) {
            const int64_t at = spos(A, i, k);
            pv[spos(P, i, a2p[at])] -= w * val[at];
        }
    }
}

// Row i of A P = sum over the entries a_ij of row i of A of a_ij (row j of
// P), 8 lanes per row and value set (4 rows per warp): the entries of row i
// of A are taken one after the other and the 8 lanes add a_ij P[j, :] into
// the row's shared accumulator; the columns of one P row differ, so no two
// lanes meet on a slot and every value is summed in the same order on every
// run.
constexpr int kApLanes = 8;
template <int NV>
__global__ void k_ap(SellDev A, SellDev P, const int64_t* ap_ptr, const int64_t* ap_sptr, const uint16_t* ap_slot,
                     int64_t ap_nnz, int ap_maxlen, const double* v0, const double* v1, const double* p0,
                     const double* p1, double* ap) {
    extern __shared__ double acc_all[];
    const int grp = threadIdx.x / kApLanes, sub = threadIdx.x % kApLanes;
    const int64_t task = blockIdx.x * int64_t(blockDim.x / kApLanes) + grp;
    const bool valid = task < A.n * NV;
    const int64_t i = valid ? task / NV : 0;
    const int v = valid ? int(task % NV) : 0;
    double* acc = acc_all + int64_t(grp) * ap_maxlen;
    const double* val = v == 0 ? v0 : v1;
    const double* pv = v == 0 ? p0 : p1;
    double* out = ap + v * ap_nnz;
    const int64_t b = valid ? ap_ptr[i] : 0, cnt = valid ? ap_ptr[i + 1] - b : 0;
    for (int64_t t = sub; t < cnt; t += kApLanes) acc[t] = 0.0;
    __syncwarp();
    int64_t o = valid ? ap_sptr[i] : 0;
    const int L = valid ? A.len[i] : 0;
    // the longest row of the warp sets the step count, so that every lane reaches each __syncwarp
    int Lw = L;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) Lw = max(Lw, __shfl_xor_sync(0xffffffffu, Lw, s));
    for (int k = 0; k < Lw; ++k) {
        if (k < L) {
            const int64_t at = spos(A, i, k);
            const int64_t j = A.col[at];
            const double a = val[at];
            const int LPj = P.len[j];
            for (int kk = sub; kk < LPj; kk += kApLanes) acc[ap_slot[o + kk]] += a * pv[spos(P, j, kk)];
            o += LPj;
        }
        __syncwarp();
    }
    for (int64_t t = sub; t < cnt; t += kApLanes) out[b + t] = acc[t];
}

// R = P^T values gathered from P (padding 0).
template <int NV>
__global__ void k_rvals(int64_t entries, const int64_t* r_src, const double* p0, const double* p1, double* r0,
                        double* r1) {
    const int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (e >= entries) return;
    const int64_t s = r_src[e];
    r0[e] = s >= 0 ? p0[s] : 0.0;
    if (NV == 2) r1[e] = s >= 0 ? p1[s] : 0.0;
}

// Coarse row I of P^T (A P), one warp per row and value set: the R entries
// (fine rows i, ascending) are taken one after the other and the lanes add
// the entries of row i of A P into the row's shared accumulator; within one
// fine row the columns differ, so no two lanes meet on a slot and every
// coarse value is summed in the same order on every run.
template <int NV>
__global__ void k_galerkin(SellDev R, SellDev C, const int64_t* r_src, const int64_t* ap_ptr, const int64_t* g_ptr,
                           const uint16_t* g_slot, int64_t ap_nnz, const double* p0, const double* p1,
                           const double* ap, double* c0, double* c1) {
    extern __shared__ double acc_all[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int64_t task = blockIdx.x * int64_t(wpb) + warp;
    if (task >= C.n * NV) return;
    const int64_t I = task / NV;
    const int v = int(task % NV);
    double* acc = acc_all + int64_t(warp) * C.maxlen;
    const double* pv = v == 0 ? p0 : p1;
    const double* apv = ap + v * ap_nnz;
    double* out = v == 0 ? c0 : c1;
    const int LC = C.len[I], LR = R.len[I];
    for (int k = lane; k < LC; k += 32) acc[k] = 0.0;
    __syncwarp();
    int64_t o = g_ptr[I];
    for (int k = 0; k < LR; ++k) {
        const int64_t at = spos(R, I, k);
        const int64_t i = R.col[at];
        const double p = pv[r_src[at]];
        const int64_t b = ap_ptr[i], cnt = ap_ptr[i + 1] - b;
        for (int64_t t = lane; t < cnt; t += 32) acc[g_slot[o + t]] += p * apv[b + t];
        o += cnt;
        __syncwarp();
    }
    for (int k = lane; k < LC; k += 32) out[spos(C, I, k)] = acc[k];
}

// In-place Gauss-Jordan inversion of the (symmetric positive definite)
// coarsest operator, one CTA per value set, without pivoting: the pivots of
// an SPD matrix are its positive Schur complements.
template <int NV>
__global__ void k_dense_inv(SellDev A, const double* v0, const double* v1, double* inv) {
    extern __shared__ double a[];
    const int n = int(A.n);
    const int v = blockIdx.x;
    const double* val = v == 0 ? v0 : v1;
    double* fcol = a + n * n;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) a[t] = 0.0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int k = 0; k < A.len[i]; ++k) {
            const int64_t at = spos(A, i, k);
            a[i * n + A.col[at]] += val[at];
        }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        const double rp = 1.0 / a[k * n + k];
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) a[k * n + j] = j == k ? rp : a[k * n + j] * rp;
        for (int i = threadIdx.x; i < n; i += blockDim.x) fcol[i] = a[i * n + k];
        __syncthreads();
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            const int i = t / n, j = t % n;
            if (i == k) continue;
            a[t] = j == k ? -fcol[i] * a[k * n + k] : a[t] - fcol[i] * a[k * n + j];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) inv[int64_t(v) * n * n + t] = a[t];
}

__global__ void k_d2f(int64_t n, const double* in, float* out) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i < n) out[i] = float(in[i]);
}

}  // namespace

namespace {

// ---------------------------------------------------------------- solve kernels

constexpr int kRedMaxGrid = 1024;  // blocks of the reducing vector kernels

template <typename T, int R>
__device__ __forceinline__ void ldR(const T* p, T* v) {
    if constexpr (std::is_same<T, double>::value && R % 2 == 0) {
#pragma unroll
        for (int r = 0; r < R; r += 2) {
            const double2 t = *reinterpret_cast<const double2*>(p + r);
            v[r] = t.x;
            v[r + 1] = t.y;
        }
    } else if constexpr (std::is_same<T, float>::value && R % 4 == 0) {
#pragma unroll
        for (int r = 0; r < R; r += 4) {
            const float4 t = *reinterpret_cast<const float4*>(p + r);
            v[r] = t.x;
            v[r + 1] = t.y;
            v[r + 2] = t.z;
            v[r + 3] = t.w;
        }
    } else if constexpr (std::is_same<T, float>::value && R == 2) {
        const float2 t = *reinterpret_cast<const float2*>(p);
        v[0] = t.x;
        v[1] = t.y;
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = p[r];
    }
}

template <typename T, int R>
__device__ __forceinline__ void stR(T* p, const T* v) {
    if constexpr (std::is_same<T, double>::value && R % 2 == 0) {
#pragma unroll
        for (int r = 0; r < R; r += 2) *reinterpret_cast<double2*>(p + r) = make_double2(v[r], v[r + 1]);
    } else if constexpr (std::is_same<T, float>::value && R % 4 == 0) {
#pragma unroll
        for (int r = 0; r < R; r += 4) *reinterpret_cast<float4*>(p + r) = make_float4(v[r], v[r + 1], v[r + 2], v[r + 3]);
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) p[r] = v[r];
    }
}

// acc = (A x)_i for the R columns of row i (NV = 2: column r uses value set
// r).  G lanes share a row (G = 1: one thread per row; G = 8 for rows of a
// few dozen entries and more): lane `sub` takes entries sub, sub + G, ...
// and the group's sums are combined by a fixed xor tree, so every lane of
// the group ends with the same, run-to-run identical, total.  Lanes past the
// last row (valid = false) take part in the shuffles only.
template <typename T, int R, int NV, int G>
__device__ __forceinline__ void row_apply(const SellDev& A, const T* v0, const T* v1, const T* x, int64_t i, int sub,
                                          bool valid, T* acc) {
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = T(0);
    const int L = valid ? A.len[i] : 0;
    const int64_t base = !valid ? 0 : A.rowmajor ? A.ptr[i] : A.ptr[i >> 5] * 32 + (i & 31);
    const int64_t stride = A.rowmajor ? 1 : 32;
    for (int k = sub; k < L; k += G) {
        const int64_t at = base + int64_t(k) * stride;
        const int64_t c = A.col[at];
        T xv[R];
        ldR<T, R>(x + c * R, xv);
        if constexpr (NV == 1) {
            const T a = v0[at];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = fma(a, xv[r], acc[r]);
        } else {
            acc[0] = fma(v0[at], xv[0], acc[0]);
            acc[1] = fma(v1[at], xv[1], acc[1]);
        }
    }
    if constexpr (G > 1) {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    }
}

// MODE 0: y = A x;  1: y = b - A x;  2: y = b + A x (b may be y).
template <typename T, int R, int NV, int MODE, int G>
__global__ void __launch_bounds__(256) k_spmv(SellDev A, const T* v0, const T* v1, const T* x, const T* b, T* y) {
    const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t i = t / G;
    const int sub = int(t % G);
    const bool valid = i < A.n;
    if (G == 1 && !valid) return;
    T acc[R];
    row_apply<T, R, NV, G>(A, v0, v1, x, i, sub, valid, acc);
    if (!valid || sub != 0) return;
    if constexpr (MODE != 0) {
        T bv[R];
        ldR<T, R>(b + i * R, bv);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = MODE == 1 ? bv[r] - acc[r] : bv[r] + acc[r];
    }
    stR<T, R>(y + i * R, acc);
}

// Chebyshev smoothing step k (of a polynomial in D^-1 A on [hi / ratio, hi]):
//   res = b - A x_in  (FIRST: x_in = 0, res = b),
//   d = c_d d + c_r D^-1 res,  x_out = x_in + d,
// with the coefficients of the three-term recurrence (Saad, Iterative
// Methods for Sparse Linear Systems, Alg. 12.1): theta, delta the centre and
// half-width of the interval, sigma = theta / delta, rho_0 = 1 / sigma,
// rho_k = 1 / (2 sigma - rho_{k-1}); step 0: c_d = 0, c_r = 1 / theta;
// step k: c_d = rho_k rho_{k-1}, c_r = 2 rho_k / delta.
template <typename T, int R, int NV, bool FIRST, int G>
__global__ void __launch_bounds__(256) k_cheb(SellDev A, const T* v0, const T* v1, const T* dinv, const double* hi,
                                              double ratio, int k, const T* x_in, T* x_out, T* d, const T* b) {
    const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t i = t / G;
    const int sub = int(t % G);
    const bool valid = i < A.n;
    if ((G == 1 || FIRST) && !valid) return;
    T res[R];
    if constexpr (!FIRST) row_apply<T, R, NV, G>(A, v0, v1, x_in, i, sub, valid, res);
    if (!valid || sub != 0) return;
    T cd[NV], cr[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const double h = hi[v], lo = h / ratio;
        const double theta = 0.5 * (h + lo), delta = 0.5 * (h - lo), sigma = theta / delta;
        double rho_prev = 1.0 / sigma, rho = rho_prev;
        for (int j = 1; j <= k; ++j) {
            rho_prev = rho;
            rho = 1.0 / (2.0 * sigma - rho_prev);
        }
        cd[v] = k == 0 ? T(0) : T(rho * rho_prev);
        cr[v] = k == 0 ? T(1.0 / theta) : T(2.0 * rho / delta);
    }
    T bv[R], dv[R], xv[R];
    ldR<T, R>(b + i * R, bv);
    if constexpr (FIRST) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            res[r] = bv[r];
            xv[r] = T(0);
        }
    } else {
        ldR<T, R>(x_in + i * R, xv);
#pragma unroll
        for (int r = 0; r < R; ++r) res[r] = bv[r] - res[r];
    }
    if (k > 0) ldR<T, R>(d + i * R, dv);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = NV == 2 ? r : 0;
        const T di = dinv[i * NV + v];
        const T upd = cr[v] * di * res[r];
        dv[r] = k > 0 ? fma(cd[v], dv[r], upd) : upd;
        xv[r] += dv[r];
    }
    stR<T, R>(d + i * R, dv);
    stR<T, R>(x_out + i * R, xv);
}

// x = A^-1 b on the coarsest level (dense inverse, n <= kAmgCoarsest).
template <typename T, int R, int NV>
__global__ void k_dense_apply(int n, const T* inv, const T* b, T* x) {
    for (int t = threadIdx.x; t < n * R; t += blockDim.x) {
        const int i = t / R, r = t % R;
        const T* row = inv + int64_t(NV == 2 ? r : 0) * n * n + int64_t(i) * n;
        T s = T(0);
        for (int j = 0; j < n; ++j) s = fma(row[j], b[j * R + r], s);
        x[t] = s;
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block totals of Q per-thread values, in a fixed order, to part[blockIdx * Q + q].
template <int Q>
__device__ __forceinline__ void block_partials(double* v, double* part) {
    __shared__ double red[8][Q];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const double t = warp_sum(v[q]);
        if (lane == 0) red[warp][q] = t;
    }
    __syncthreads();
    if (threadIdx.x < Q) {
        double s = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        part[int64_t(blockIdx.x) * Q + threadIdx.x] = s;
    }
}

// Total of quantity q over G block partials (a full warp calls it; every lane gets it).
__device__ __forceinline__ double total_of(const double* part, int G, int Q, int q) {
    double s = 0.0;
    for (int g = threadIdx.x & 31; g < G; g += 32) s += part[int64_t(g) * Q + q];
    return warp_sum(s);
}

// ---- conjugate gradients (FP64), R right-hand sides; ctl[0] status, ctl[1] RHS still running

// x = 0, r = b, partials of b.b
template <int R>
__global__ void __launch_bounds__(256) k_cg_init(int64_t n, const double* b, double* x, double* r, double* part) {
    double acc[R];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[q] = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        double bv[R], z[R];
        ldR<double, R>(b + i * R, bv);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            acc[q] = fma(bv[q], bv[q], acc[q]);
            z[q] = 0.0;
        }
        stR<double, R>(r + i * R, bv);
        stR<double, R>(x + i * R, z);
    }
    block_partials<R>(acc, part);
}

// x = x0, r = b - A x0, partials of b.b (the stopping target stays rtol |b|)
template <int R, int NV>
__global__ void __launch_bounds__(256) k_cg_init_x0(SellDev A, const double* v0, const double* v1, const double* b,
                                                    const double* x0, double* x, double* r, double* part) {
    double acc[R];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[q] = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < A.n; i += int64_t(gridDim.x) * blockDim.x) {
        double bv[R], av[R], xv[R];
        row_apply<double, R, NV, 1>(A, v0, v1, x0, i, 0, true, av);
        ldR<double, R>(b + i * R, bv);
        ldR<double, R>(x0 + i * R, xv);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            acc[q] = fma(bv[q], bv[q], acc[q]);
            av[q] = bv[q] - av[q];
        }
        stR<double, R>(r + i * R, av);
        stR<double, R>(x + i * R, xv);
    }
    block_partials<R>(acc, part);
}

// Control words of a CG solve (int ctl[]): [0] status, [1] right-hand sides
// still running, [2] iterations done, [3] 1 before the first direction,
// [4] iteration cap; the per-RHS running flags follow at ctl + kCtlActive.
constexpr int kCtlActive = 8;

// bb = totals; a right-hand side with b = 0 is solved by x = 0 and never runs
template <int R>
__global__ void k_cg_start(const double* part, int G, double* bb, int* ctl) {
    int* active = ctl + kCtlActive;
    const int r = threadIdx.x >> 5;
    const double t = total_of(part, G, R, r);
    if ((threadIdx.x & 31) == 0) {
        bb[r] = t;
        active[r] = t > 0.0 ? 1 : 0;
        if (!isfinite(t)) atomicExch(ctl, int(QPAT_EINVAL));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int c = 0;
        for (int q = 0; q < R; ++q) c += active[q];
        ctl[1] = c;
        ctl[2] = 0;
        ctl[3] = 1;
    }
}

// q = A p and partials of p.q
template <int R, int NV>
__global__ void __launch_bounds__(256) k_cg_apply(SellDev A, const double* v0, const double* v1, const double* p,
                                                  double* q, double* part) {
    double acc[R];
#pragma unroll
    for (int t = 0; t < R; ++t) acc[t] = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < A.n; i += int64_t(gridDim.x) * blockDim.x) {
        double qv[R], pv[R];
        row_apply<double, R, NV, 1>(A, v0, v1, p, i, 0, true, qv);
        ldR<double, R>(p + i * R, pv);
#pragma unroll
        for (int t = 0; t < R; ++t) acc[t] = fma(pv[t], qv[t], acc[t]);
        stR<double, R>(q + i * R, qv);
    }
    block_partials<R>(acc, part);
}

// alpha = r.z / p.q on the running right-hand sides (0 on the others)
template <int R>
__global__ void k_cg_alpha(const double* part, int G, const double* rz, double* alpha, int* ctl) {
    const int* active = ctl + kCtlActive;
    const int r = threadIdx.x >> 5;
    const double pq = total_of(part, G, R, r);
    if ((threadIdx.x & 31) == 0) {
        double a = 0.0;
        if (active[r]) {
            if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rz[r]))
                atomicExch(ctl, int(QPAT_EBREAKDOWN));
            else
                a = rz[r] / pq;
        }
        alpha[r] = a;
    }
}

// x += alpha p, r -= alpha q, partials of r.r
// The vector passes of the CG give each node's R values to R / C threads
// of C right-hand sides each (C = 8 for R = 16): fewer live registers per
// thread, more loads in flight for these memory-bound passes.
template <int R>
constexpr int kChunk = R > 8 ? 8 : R;

// Block totals of per-thread partials over C right-hand sides when thread t
// holds chunk t % (R / C): an xor tree over the lanes of the same chunk,
// then the warps in order; part[blockIdx * R * NQ + q * R + r] for the NQ
// quantities of acc (acc[q * C + j] belongs to right-hand side chunk * C + j).
template <int R, int NQ>
__device__ __forceinline__ void chunk_partials(const double* acc, double* part) {
    constexpr int C = kChunk<R>, NCH = R / C;
    __shared__ double red[8][NQ * R];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int j = 0; j < C; ++j) {
            double v = acc[q * C + j];
#pragma unroll
            for (int o = 16; o >= NCH; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane < NCH) red[warp][q * R + lane * C + j] = v;
        }
    __syncthreads();
    if (threadIdx.x < NQ * R) {
        double t = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
        part[int64_t(blockIdx.x) * NQ * R + threadIdx.x] = t;
    }
}

// The next cycle's first fine-level smoothing step (from x = 0: x = d =
// c_r D^-1 b with b = r, c_r = 1 / theta as in k_cheb), taken in the CG
// update on the residual it has just written instead of by a separate pass
// over r; for the FP32 cycle also the FP32 copy of r.  The same operations
// in the same order as k_cheb's first step, so the results do not change.
template <typename T, int NV>
struct PreStep {
    const T* dinv = nullptr;      // fine level, n x NV
    const double* hi = nullptr;   // Gershgorin bounds of the fine level, per value set
    double ratio = 30.0;
    T* x = nullptr;               // the cycle's first fine-level buffer (x = d after the step)
    T* d = nullptr;               // null when no later pre-smoothing step reads d (degree 1)
    float* b32 = nullptr;         // FP32 cycle: the fine level's right-hand side
};

template <int R, int NV, typename T>
__global__ void __launch_bounds__(256) k_cg_update(int64_t n, const double* alpha, const double* p, const double* q,
                                                   double* x, double* r, double* part, PreStep<T, NV> pre) {
    constexpr int C = kChunk<R>, NCH = R / C;
    const int c0 = int(threadIdx.x % NCH) * C;
    double al[C], acc[C];
#pragma unroll
    for (int t = 0; t < C; ++t) {
        al[t] = alpha[c0 + t];
        acc[t] = 0.0;
    }
    T cr[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const double h = pre.hi[v], lo = h / pre.ratio;
        cr[v] = T(1.0 / (0.5 * (h + lo)));
    }
    for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < n * NCH;
         g += int64_t(gridDim.x) * blockDim.x) {
        const int64_t node = g / NCH;
        const int64_t o = node * R + c0;
        double pv[C], qv[C], xv[C], rv[C];
        ldR<double, C>(p + o, pv);
        ldR<double, C>(q + o, qv);
        ldR<double, C>(x + o, xv);
        ldR<double, C>(r + o, rv);
#pragma unroll
        for (int t = 0; t < C; ++t) {
            xv[t] = fma(al[t], pv[t], xv[t]);
            rv[t] = fma(-al[t], qv[t], rv[t]);
            acc[t] = fma(rv[t], rv[t], acc[t]);
        }
        stR<double, C>(x + o, xv);
        stR<double, C>(r + o, rv);
        T rc[C], up[C];
#pragma unroll
        for (int t = 0; t < C; ++t) {
            const int v = NV == 2 ? c0 + t : 0;
            rc[t] = T(rv[t]);
            const T upd = cr[v] * pre.dinv[node * NV + v] * rc[t];
            up[t] = T(0) + upd;
        }
        if constexpr (std::is_same<T, float>::value) stR<float, C>(pre.b32 + o, rc);
        if (pre.d) stR<T, C>(pre.d + o, up);
        stR<T, C>(pre.x + o, up);
    }
    chunk_partials<R, 1>(acc, part);
}

// a right-hand side stops once |r| <= rtol |b|; one more iteration is done.
// Inside a graph (use_graph) the kernel also sets the loop's condition: go
// on while some right-hand side runs, the status is clean and the cap is not
// reached (reaching it with a running right-hand side is QPAT_ENOCONV).
template <int R>
__global__ void k_cg_check(const double* part, int G, const double* bb, const double* rtol2, double* rr, int* ctl,
                           cudaGraphConditionalHandle cond, int use_graph) {
    int* active = ctl + kCtlActive;
    const int r = threadIdx.x >> 5;
    const double t = total_of(part, G, R, r);
    if ((threadIdx.x & 31) == 0) {
        rr[r] = t;
        if (!isfinite(t)) atomicExch(ctl, int(QPAT_EBREAKDOWN));
        if (active[r] && t <= *rtol2 * bb[r]) active[r] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int c = 0;
        for (int q = 0; q < R; ++q) c += active[q];
        ctl[1] = c;
        const int it = ++ctl[2];
        if (c > 0 && it >= ctl[4] && ctl[0] == QPAT_OK) ctl[0] = QPAT_ENOCONV;
        if (use_graph) cudaGraphSetConditional(cond, (c > 0 && ctl[0] == QPAT_OK) ? 1u : 0u);
    }
}

// partials of r.z (and, FLEX, of r.z_old)
template <int R, bool FLEX>
__global__ void __launch_bounds__(256) k_cg_dots(int64_t n, const double* r, const double* z, const double* zo,
                                                 double* part) {
    constexpr int C = kChunk<R>, NCH = R / C, NQ = FLEX ? 2 : 1;
    const int c0 = int(threadIdx.x % NCH) * C;
    double acc[NQ * C];
#pragma unroll
    for (int t = 0; t < NQ * C; ++t) acc[t] = 0.0;
    for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < n * NCH;
         g += int64_t(gridDim.x) * blockDim.x) {
        const int64_t o = (g / NCH) * R + c0;
        double rv[C], zv[C];
        ldR<double, C>(r + o, rv);
        ldR<double, C>(z + o, zv);
#pragma unroll
        for (int t = 0; t < C; ++t) acc[t] = fma(rv[t], zv[t], acc[t]);
        if constexpr (FLEX) {
            ldR<double, C>(zo + o, zv);
#pragma unroll
            for (int t = 0; t < C; ++t) acc[C + t] = fma(rv[t], zv[t], acc[C + t]);
        }
    }
    chunk_partials<R, NQ>(acc, part);
}

// beta = r.z / (r.z)_old (FLEX: (r.z - r.z_old) / (r.z)_old, the form that
// tolerates a preconditioner that varies slightly between applications);
// 0 before the first direction (ctl[3], cleared here).  rz <- r.z.
template <int R, bool FLEX>
__global__ void k_cg_beta(const double* part, int G, double* rz, double* beta, int* ctl) {
    constexpr int Q = FLEX ? 2 * R : R;
    const int* active = ctl + kCtlActive;
    const int first = ctl[3];
    const int r = threadIdx.x >> 5;
    const double t = total_of(part, G, Q, r);
    const double to = FLEX ? total_of(part, G, Q, R + r) : 0.0;
    if ((threadIdx.x & 31) == 0) {
        double b = 0.0;
        if (!first && active[r]) b = (t - to) / rz[r];
        if (active[r] && (!isfinite(t) || !(t > 0.0))) atomicExch(ctl, int(QPAT_EBREAKDOWN));
        beta[r] = b;
        rz[r] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) ctl[3] = 0;
}

// p = z + beta p (FLEX: and z_old = z for the next beta)
template <int R, bool FLEX>
__global__ void __launch_bounds__(256) k_cg_dir(int64_t n, const double* beta, const double* z, double* p,
                                                double* zo) {
    constexpr int C = kChunk<R>, NCH = R / C;
    const int c0 = int(threadIdx.x % NCH) * C;
    double be[C];
#pragma unroll
    for (int t = 0; t < C; ++t) be[t] = beta[c0 + t];
    for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < n * NCH;
         g += int64_t(gridDim.x) * blockDim.x) {
        const int64_t o = (g / NCH) * R + c0;
        double zv[C], pv[C];
        ldR<double, C>(z + o, zv);
        ldR<double, C>(p + o, pv);
#pragma unroll
        for (int t = 0; t < C; ++t) pv[t] = fma(be[t], pv[t], zv[t]);
        stR<double, C>(p + o, pv);
        if constexpr (FLEX) stR<double, C>(zo + o, zv);
    }
}

__global__ void k_d2f_vec(int64_t n, const double* in, float* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = float(in[i]);
}
__global__ void k_f2d_vec(int64_t n, const float* in, double* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = double(in[i]);
}

}  // namespace

// ---------------------------------------------------------------- host side

struct AmgHierDev {
    bool tried = false;
    std::string error;
    std::vector<LevelDev> lv;
    std::vector<void*> allocs;
};

struct AmgValues {
    uint64_t stamp = 0;
    bool valid = false;
    bool has32 = false;
    std::vector<std::array<double*, 2>> A, P, R;  // A[0] unused (the operator's own values)
    std::vector<double*> AP, dinv;
    double* hi = nullptr;   // 2 per level
    double* inv = nullptr;  // coarsest inverse, NV x n x n
    std::vector<std::array<float*, 2>> A32, P32, R32;  // A32[0]: FP32 copy of the operator
    std::vector<float*> dinv32;
    float* inv32 = nullptr;
    std::vector<void*> allocs;
};

struct AmgVecs {
    std::vector<void*> b, xa, xb, d, r;
    std::vector<void*> allocs;
};

struct AmgCg {
    double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *zo = nullptr, *part = nullptr;
    double *bb = nullptr, *rz = nullptr, *alpha = nullptr, *beta = nullptr, *rr = nullptr, *rtol2 = nullptr;
    int* ctl = nullptr;  // control words (see k_cg_start)
    std::vector<void*> allocs;
};

// One CG iteration captured once as the body of a graph "while" node, per
// operator values, right-hand-side count and cycle settings; the check
// kernel of the body sets the loop condition on the device.
struct AmgGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int body_kernels = 0;
};

struct AmgState {
    AmgHierDev hier[2];  // 0: the K pattern, 1: the prior's stiffness-only pattern
    std::map<const void*, AmgValues> vals;
    std::map<std::pair<int, int>, AmgVecs> vecs;  // (pattern * 64 + R, FP32 V-cycle)
    std::map<int, AmgCg> cg;                       // R
    std::map<std::string, AmgGraph> graphs;
    cudaStream_t capture = nullptr;                // a non-default stream to capture on
};

namespace {

template <typename T>
T* dalloc(std::vector<void*>& list, size_t count, cudaError_t& e) {
    if (e != cudaSuccess) return nullptr;
    void* p = nullptr;
    e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return nullptr;
    list.push_back(p);
    return static_cast<T*>(p);
}

template <typename T>
const T* upload(std::vector<void*>& list, const std::vector<T>& h, cudaError_t& e) {
    T* d = dalloc<T>(list, h.size(), e);
    if (e == cudaSuccess && !h.empty()) e = cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    return d;
}

SellDev upload_sell(std::vector<void*>& list, const SellPattern& S, cudaError_t& e) {
    SellDev d;
    d.n = S.n;
    d.ptr = upload(list, S.ptr, e);
    d.col = upload(list, S.col, e);
    d.len = upload(list, S.len, e);
    d.entries = S.entries();
    d.maxlen = S.maxlen;
    d.rowmajor = S.rowmajor ? 1 : 0;
    return d;
}

inline int blocks_of(int64_t n, int per = 256) { return int(std::max<int64_t>(1, (n + per - 1) / per)); }

int build_hier(qpat_mesh_s* M, int prior, AmgHierDev& H) {
    H.tried = true;
    const AmgPlan plan = amg_build_plan(amg_fine_pattern(M->h, prior));
    if (!plan.error.empty()) {
        H.error = plan.error;
        return fail(QPAT_EINVAL, plan.error);
    }
    cudaError_t e = cudaSuccess;
    for (const AmgLevelPlan& L : plan.levels) {
        LevelDev d;
        d.A = upload_sell(H.allocs, L.A, e);
        d.diag = upload(H.allocs, L.diag, e);
        d.nc = L.nc;
        if (L.nc > 0) {
            d.P = upload_sell(H.allocs, L.P, e);
            d.a2p = upload(H.allocs, L.a2p, e);
            d.pself = upload(H.allocs, L.pself, e);
            d.ap_ptr = upload(H.allocs, L.ap_ptr, e);
            d.ap_col = upload(H.allocs, L.ap_col, e);
            d.ap_sptr = upload(H.allocs, L.ap_sptr, e);
            d.ap_slot = upload(H.allocs, L.ap_slot, e);
            d.ap_nnz = int64_t(L.ap_col.size());
            for (size_t i = 0; i + 1 < L.ap_ptr.size(); ++i)
                d.ap_maxlen = std::max<int>(d.ap_maxlen, int(L.ap_ptr[i + 1] - L.ap_ptr[i]));
            d.R = upload_sell(H.allocs, L.R, e);
            d.r_src = upload(H.allocs, L.r_src, e);
            d.g_ptr = upload(H.allocs, L.g_ptr, e);
            d.g_slot = upload(H.allocs, L.g_slot, e);
        }
        H.lv.push_back(d);
    }
    if (e != cudaSuccess) {
        H.error = std::string("multigrid upload: ") + cudaGetErrorString(e);
        return cuda_fail(e, "multigrid upload");
    }
    return QPAT_OK;
}

template <int NV>
cudaError_t numeric_levels(const AmgHierDev& H, const OpState& st, AmgValues& V, cudaStream_t s) {
    const int L = int(H.lv.size());
    cudaError_t e = cudaMemsetAsync(V.hi, 0, sizeof(double) * 2 * L, s);
    if (e != cudaSuccess) return e;
    for (int l = 0; l < L; ++l) {
        const LevelDev& d = H.lv[size_t(l)];
        const double* a0 = l == 0 ? st.v64[0] : V.A[size_t(l)][0];
        const double* a1 = l == 0 ? st.v64[1] : V.A[size_t(l)][1];
        note_launch(1);
        k_dinv_hi<NV><<<blocks_of(d.A.n), 256, 0, s>>>(d.A, d.diag, a0, a1, V.dinv[size_t(l)], V.hi + 2 * l);
        if (l + 1 == L) break;
        const auto& Pv = V.P[size_t(l)];
        const auto& Rv = V.R[size_t(l)];
        note_launch(4);
        k_prolong<NV><<<blocks_of(d.A.n), 256, 0, s>>>(d.A, d.P, d.a2p, d.pself, a0, a1, V.dinv[size_t(l)],
                                                        V.hi + 2 * l, Pv[0], Pv[1]);
        k_rvals<NV><<<blocks_of(d.R.entries), 256, 0, s>>>(d.R.entries, d.r_src, Pv[0], Pv[1], Rv[0], Rv[1]);
        {
            int wpb = 8;  // warps per block, kApLanes lanes per row
            const int rpw = 32 / kApLanes;
            while (wpb > 1 && size_t(wpb * rpw) * size_t(d.ap_maxlen) * sizeof(double) > 96 * 1024) wpb >>= 1;
            const size_t smem = size_t(wpb * rpw) * size_t(d.ap_maxlen) * sizeof(double);
            if ((e = allow_smem(reinterpret_cast<const void*>(&k_ap<NV>), smem)) != cudaSuccess) return e;
            k_ap<NV><<<blocks_of(d.A.n * NV, wpb * rpw), 32 * wpb, smem, s>>>(
                d.A, d.P, d.ap_ptr, d.ap_sptr, d.ap_slot, d.ap_nnz, d.ap_maxlen, a0, a1, Pv[0], Pv[1],
                V.AP[size_t(l)]);
        }
        const LevelDev& c = H.lv[size_t(l + 1)];
        int wpb = 8;
        while (wpb > 1 && size_t(wpb) * size_t(c.A.maxlen) * sizeof(double) > 96 * 1024) wpb >>= 1;
        const size_t smem = size_t(wpb) * size_t(c.A.maxlen) * sizeof(double);
        if ((e = allow_smem(reinterpret_cast<const void*>(&k_galerkin<NV>), smem)) != cudaSuccess) return e;
        k_galerkin<NV><<<blocks_of(c.A.n * NV, wpb), 32 * wpb, smem, s>>>(
            d.R, c.A, d.r_src, d.ap_ptr, d.g_ptr, d.g_slot, d.ap_nnz, Pv[0], Pv[1], V.AP[size_t(l)],
            V.A[size_t(l + 1)][0], V.A[size_t(l + 1)][1]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const LevelDev& c = H.lv[size_t(L - 1)];
    const int n = int(c.A.n);
    const size_t smem = size_t(n) * size_t(n + 1) * sizeof(double);
    if ((e = allow_smem(reinterpret_cast<const void*>(&k_dense_inv<NV>), smem)) != cudaSuccess) return e;
    const double* a0 = L == 1 ? st.v64[0] : V.A[size_t(L - 1)][0];
    const double* a1 = L == 1 ? st.v64[1] : V.A[size_t(L - 1)][1];
    note_launch(1);
    k_dense_inv<NV><<<NV, 256, smem, s>>>(c.A, a0, a1, V.inv);
    return cudaGetLastError();
}

cudaError_t cast_to_f32(const double* in, float* out, int64_t n, cudaStream_t s) {
    note_launch(1);
    k_d2f<<<blocks_of(n), 256, 0, s>>>(n, in, out);
    return cudaGetLastError();
}

// Values of the hierarchy for the operator st (allocated once per operator
// buffer, recomputed when st was prepared again).
int numeric(qpat_mesh_s* M, const AmgHierDev& H, const OpState& st, AmgValues& V, bool need32, cudaStream_t s) {
    const int L = int(H.lv.size());
    const int NV = st.nv;
    cudaError_t e = cudaSuccess;
    if (V.A.empty()) {
        V.A.assign(size_t(L), {nullptr, nullptr});
        V.P.assign(size_t(L), {nullptr, nullptr});
        V.R.assign(size_t(L), {nullptr, nullptr});
        V.AP.assign(size_t(L), nullptr);
        V.dinv.assign(size_t(L), nullptr);
        for (int l = 0; l < L; ++l) {
            const LevelDev& d = H.lv[size_t(l)];
            for (int v = 0; v < NV; ++v) {
                if (l > 0) V.A[size_t(l)][size_t(v)] = dalloc<double>(V.allocs, size_t(d.A.entries), e);
                if (l + 1 < L) {
                    V.P[size_t(l)][size_t(v)] = dalloc<double>(V.allocs, size_t(d.P.entries), e);
                    V.R[size_t(l)][size_t(v)] = dalloc<double>(V.allocs, size_t(d.R.entries), e);
                }
            }
            if (l + 1 < L) V.AP[size_t(l)] = dalloc<double>(V.allocs, size_t(d.ap_nnz) * NV, e);
            V.dinv[size_t(l)] = dalloc<double>(V.allocs, size_t(d.A.n) * NV, e);
        }
        V.hi = dalloc<double>(V.allocs, size_t(2 * L), e);
        const int64_t nco = H.lv.back().A.n;
        V.inv = dalloc<double>(V.allocs, size_t(NV * nco * nco), e);
        if (e != cudaSuccess) return cuda_fail(e, "multigrid workspace");
        // P and A P padding entries are never written: keep them 0
        for (int l = 0; l + 1 < L; ++l)
            for (int v = 0; v < NV; ++v)
                if ((e = cudaMemsetAsync(V.P[size_t(l)][size_t(v)], 0, sizeof(double) * H.lv[size_t(l)].P.entries, s)) !=
                    cudaSuccess)
                    return cuda_fail(e, "multigrid memset");
    }
    if (need32 && !V.has32) {
        V.A32.assign(size_t(L), {nullptr, nullptr});
        V.P32.assign(size_t(L), {nullptr, nullptr});
        V.R32.assign(size_t(L), {nullptr, nullptr});
        V.dinv32.assign(size_t(L), nullptr);
        for (int l = 0; l < L; ++l) {
            const LevelDev& d = H.lv[size_t(l)];
            for (int v = 0; v < NV; ++v) {
                V.A32[size_t(l)][size_t(v)] = dalloc<float>(V.allocs, size_t(d.A.entries), e);
                if (l + 1 < L) {
                    V.P32[size_t(l)][size_t(v)] = dalloc<float>(V.allocs, size_t(d.P.entries), e);
                    V.R32[size_t(l)][size_t(v)] = dalloc<float>(V.allocs, size_t(d.R.entries), e);
                }
            }
            V.dinv32[size_t(l)] = dalloc<float>(V.allocs, size_t(d.A.n) * NV, e);
        }
        const int64_t nco = H.lv.back().A.n;
        V.inv32 = dalloc<float>(V.allocs, size_t(NV * nco * nco), e);
        if (e != cudaSuccess) return cuda_fail(e, "multigrid workspace");
        V.has32 = true;
        V.valid = false;
    }
    if (V.valid && V.stamp == st.stamp) return QPAT_OK;
    e = NV == 1 ? numeric_levels<1>(H, st, V, s) : numeric_levels<2>(H, st, V, s);
    if (e != cudaSuccess) return cuda_fail(e, "multigrid set-up");
    if (V.has32) {
        for (int l = 0; l < L && e == cudaSuccess; ++l) {
            const LevelDev& d = H.lv[size_t(l)];
            for (int v = 0; v < NV && e == cudaSuccess; ++v) {
                const double* a = l == 0 ? st.v64[v] : V.A[size_t(l)][size_t(v)];
                e = cast_to_f32(a, V.A32[size_t(l)][size_t(v)], d.A.entries, s);
                if (e == cudaSuccess && l + 1 < L) e = cast_to_f32(V.P[size_t(l)][size_t(v)], V.P32[size_t(l)][size_t(v)], d.P.entries, s);
                if (e == cudaSuccess && l + 1 < L) e = cast_to_f32(V.R[size_t(l)][size_t(v)], V.R32[size_t(l)][size_t(v)], d.R.entries, s);
            }
            if (e == cudaSuccess) e = cast_to_f32(V.dinv[size_t(l)], V.dinv32[size_t(l)], d.A.n * NV, s);
        }
        const int64_t nco = H.lv.back().A.n;
        if (e == cudaSuccess) e = cast_to_f32(V.inv, V.inv32, NV * nco * nco, s);
        if (e != cudaSuccess) return cuda_fail(e, "multigrid set-up");
    }
    V.stamp = st.stamp;
    V.valid = true;
    (void)M;
    return QPAT_OK;
}

}  // namespace

namespace {

// Optional CUDA-event timing of the fine-level smoothing launches (the
// multigrid cycle's dominant kernel); the events of one cycle are read after
// the next stream synchronisation of the CG loop.
struct FineTimer {
    bool on = false;
    cudaStream_t s = nullptr;
    std::vector<cudaEvent_t> ev;
    int used = 0;
    double ms = 0.0;
    int64_t launches = 0;
    void before() {
        if (!on) return;
        if (used + 2 > int(ev.size())) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            ev.push_back(a);
            ev.push_back(b);
        }
        cudaEventRecord(ev[size_t(used)], s);
    }
    void after() {
        if (!on) return;
        cudaEventRecord(ev[size_t(used + 1)], s);
        used += 2;
    }
    void collect() {  // after a synchronisation of the stream
        for (int k = 0; k < used; k += 2) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, ev[size_t(k)], ev[size_t(k + 1)]) == cudaSuccess) ms += t;
            ++launches;
        }
        used = 0;
    }
    ~FineTimer() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

// One V-cycle x = B b on level l and below (pre-smoothing from x = 0,
// residual, restriction, the coarser cycle, prolongation, post-smoothing
// with the same polynomial: B is symmetric).
template <typename T, int R, int NV>
struct VCycle {
    const AmgHierDev& H;
    const AmgValues& V;
    AmgVecs& W;
    const OpState& st;
    int deg;
    double ratio;
    cudaStream_t s;
    FineTimer* timer = nullptr;
    bool pre_done = false;  // the fine level's first smoothing step was taken by the CG update

    static constexpr bool F64 = std::is_same<T, double>::value;
    const T* av(int l, int v) const {
        if constexpr (F64)
            return l == 0 ? st.v64[v] : V.A[size_t(l)][size_t(v)];
        else
            return V.A32[size_t(l)][size_t(v)];
    }
    const T* pv(int l, int v) const {
        if constexpr (F64) return V.P[size_t(l)][size_t(v)];
        else return V.P32[size_t(l)][size_t(v)];
    }
    const T* rv(int l, int v) const {
        if constexpr (F64) return V.R[size_t(l)][size_t(v)];
        else return V.R32[size_t(l)][size_t(v)];
    }
    const T* dinv(int l) const {
        if constexpr (F64) return V.dinv[size_t(l)];
        else return V.dinv32[size_t(l)];
    }
    const T* inv() const {
        if constexpr (F64) return V.inv;
        else return V.inv32;
    }

    template <int MODE>
    void spmv(const SellDev& A, const T* a0, const T* a1, const T* x, const T* b, T* y) {
        note_launch(1);
        if (A.rowmajor)
            k_spmv<T, R, NV, MODE, 8><<<blocks_of(A.n * 8), 256, 0, s>>>(A, a0, a1, x, b, y);
        else
            k_spmv<T, R, NV, MODE, 1><<<blocks_of(A.n), 256, 0, s>>>(A, a0, a1, x, b, y);
    }
    void cheb(const SellDev& A, const T* a0, const T* a1, const T* di, const double* hi, int k, const T* x_in,
              T* x_out, T* d, const T* b) {
        note_launch(1);
        if (A.rowmajor)
            k_cheb<T, R, NV, false, 8><<<blocks_of(A.n * 8), 256, 0, s>>>(A, a0, a1, di, hi, ratio, k, x_in, x_out, d,
                                                                          b);
        else
            k_cheb<T, R, NV, false, 1><<<blocks_of(A.n), 256, 0, s>>>(A, a0, a1, di, hi, ratio, k, x_in, x_out, d, b);
    }

    // the fine level's first smoothing step on b (before the first iteration)
    void first_fine(const T* b) {
        if (H.lv.size() < 2) return;
        const LevelDev& d = H.lv[0];
        note_launch(1);
        k_cheb<T, R, NV, true, 1><<<blocks_of(d.A.n), 256, 0, s>>>(d.A, av(0, 0), av(0, 1), dinv(0), V.hi, ratio, 0,
                                                                  nullptr, static_cast<T*>(W.xa[0]),
                                                                  static_cast<T*>(W.d[0]), b);
    }

    PreStep<T, NV> pre_step(float* b32) const {
        PreStep<T, NV> p;
        p.dinv = dinv(0);
        p.hi = V.hi;
        p.ratio = ratio;
        p.x = static_cast<T*>(W.xa[0]);
        p.d = deg > 1 ? static_cast<T*>(W.d[0]) : nullptr;
        p.b32 = b32;
        return p;
    }

    const T* run(int l, const T* b) {
        const LevelDev& d = H.lv[size_t(l)];
        const int L = int(H.lv.size());
        T* x = static_cast<T*>(W.xa[size_t(l)]);
        T* y = static_cast<T*>(W.xb[size_t(l)]);
        T* dd = static_cast<T*>(W.d[size_t(l)]);
        if (l == L - 1) {
            note_launch(1);
            k_dense_apply<T, R, NV><<<1, 256, 0, s>>>(int(d.A.n), inv(), b, x);
            return x;
        }
        const double* hi = V.hi + 2 * l;
        const T *a0 = av(l, 0), *a1 = av(l, 1);
        if (!(l == 0 && pre_done)) {
            note_launch(1);
            k_cheb<T, R, NV, true, 1><<<blocks_of(d.A.n), 256, 0, s>>>(d.A, a0, a1, dinv(l), hi, ratio, 0, nullptr,
                                                                      x, dd, b);
        }
        for (int k = 1; k < deg; ++k) {
            if (l == 0 && timer) timer->before();
            cheb(d.A, a0, a1, dinv(l), hi, k, x, y, dd, b);
            if (l == 0 && timer) timer->after();
            std::swap(x, y);
        }
        T* res = static_cast<T*>(W.r[size_t(l)]);
        T* bc = static_cast<T*>(W.b[size_t(l + 1)]);
        spmv<1>(d.A, a0, a1, x, b, res);
        spmv<0>(d.R, rv(l, 0), rv(l, 1), res, nullptr, bc);
        const T* xc = run(l + 1, bc);
        spmv<2>(d.P, pv(l, 0), pv(l, 1), xc, x, x);
        for (int k = 0; k < deg; ++k) {
            if (l == 0 && timer) timer->before();
            cheb(d.A, a0, a1, dinv(l), hi, k, x, y, dd, b);
            if (l == 0 && timer) timer->after();
            std::swap(x, y);
        }
        return x;
    }
};

// Conjugate gradients on the fine operator with one V-cycle per iteration
// as the preconditioner; X0 (or 0) to start, each right-hand side stops at
// |r| <= rtol |b| (the recursive residual, as the persistent PCG does).
// After the start, every iteration is
//   z = B r, beta = r.z / (r.z)_old, p = z + beta p, q = A p,
//   alpha = r.z / p.q, x += alpha p, r -= alpha q, check,
// launched from the host one kernel at a time when the fine-level smoothing
// is being timed, and otherwise replayed from a captured graph whose
// "while" node runs on the device until the check ends it (no host round
// trip per iteration).  Both forms launch the same kernels on the same data.
template <int R, int NV>
struct CgSolve {
    qpat_mesh_s* M;
    const OpState& st;
    const SolveOpts& so;
    const AmgHierDev& H;
    const AmgValues& V;
    bool f32;
    AmgVecs& W;
    AmgCg& C;
    cudaStream_t s;
    FineTimer* timer;
    int64_t n = 0;
    int G = 0;

    // kernels of one iteration: per level above the coarsest 2 deg + 3
    // (smoothing, residual, restriction, prolongation), 1 on the coarsest,
    // 2 casts for the FP32 cycle, 7 of the CG itself
    // (the fine level's first smoothing step, and for the FP32 cycle the cast
    // of r, are taken by the CG update)
    int body_kernels() const {
        const int deg = std::max(1, so.mg_degree);
        const int L = int(H.lv.size());
        return (L - 1) * (2 * deg + 3) - (L > 1 ? 1 : 0) + 1 + (f32 ? 1 : 0) + 7;
    }

    // one iteration on stream t; use_graph: the check sets the loop condition
    void body(cudaStream_t t, cudaGraphConditionalHandle cond, int use_graph) {
        const int deg = std::max(1, so.mg_degree);
        const LevelDev& d0 = H.lv[0];
        const double* z;
        const bool multi = H.lv.size() > 1;
        if (!f32) {
            VCycle<double, R, NV> c{H, V, W, st, deg, so.mg_ratio, t, timer, multi};
            z = c.run(0, C.r);
        } else {
            VCycle<float, R, NV> c{H, V, W, st, deg, so.mg_ratio, t, timer, multi};
            const float* x0 = c.run(0, static_cast<float*>(W.b[0]));
            note_launch(1);
            k_f2d_vec<<<G, 256, 0, t>>>(n * R, x0, C.z);
            z = C.z;
        }
        note_launch(7);
        if (f32) {
            k_cg_dots<R, true><<<G, 256, 0, t>>>(n, C.r, z, C.zo, C.part);
            k_cg_beta<R, true><<<1, 32 * R, 0, t>>>(C.part, G, C.rz, C.beta, C.ctl);
            k_cg_dir<R, true><<<G, 256, 0, t>>>(n, C.beta, z, C.p, C.zo);
        } else {
            k_cg_dots<R, false><<<G, 256, 0, t>>>(n, C.r, z, nullptr, C.part);
            k_cg_beta<R, false><<<1, 32 * R, 0, t>>>(C.part, G, C.rz, C.beta, C.ctl);
            k_cg_dir<R, false><<<G, 256, 0, t>>>(n, C.beta, z, C.p, nullptr);
        }
        k_cg_apply<R, NV><<<G, 256, 0, t>>>(d0.A, st.v64[0], st.v64[1], C.p, C.q, C.part);
        k_cg_alpha<R><<<1, 32 * R, 0, t>>>(C.part, G, C.rz, C.alpha, C.ctl);
        if (!f32) {
            VCycle<double, R, NV> c{H, V, W, st, deg, so.mg_ratio, t, timer};
            k_cg_update<R, NV, double><<<G, 256, 0, t>>>(n, C.alpha, C.p, C.q, C.x, C.r, C.part, c.pre_step(nullptr));
        } else {
            VCycle<float, R, NV> c{H, V, W, st, deg, so.mg_ratio, t, timer};
            float* b0 = static_cast<float*>(W.b[0]);
            k_cg_update<R, NV, float><<<G, 256, 0, t>>>(n, C.alpha, C.p, C.q, C.x, C.r, C.part, c.pre_step(b0));
        }
        k_cg_check<R><<<1, 32 * R, 0, t>>>(C.part, G, C.bb, C.rtol2, C.rr, C.ctl, cond, use_graph);
    }

    int run(AmgState& A, const std::string& key, const double* B, double* X, const double* X0, int* iters) {
        const LevelDev& d0 = H.lv[0];
        n = d0.A.n;
        G = int(std::min<int64_t>(blocks_of(n), kRedMaxGrid));
        int* hc = reinterpret_cast<int*>(M->host_scratch + 240);
        cudaError_t e = cudaSuccess;
        auto read_ctl = [&]() -> cudaError_t {
            cudaError_t x = cudaMemcpyAsync(hc, C.ctl, 3 * sizeof(int), cudaMemcpyDeviceToHost, s);
            if (x == cudaSuccess) x = cudaStreamSynchronize(s);
            return x;
        };
        const double rtol2 = so.rtol * so.rtol;
        const int cap[1] = {so.maxit};
        if ((e = cudaMemsetAsync(C.ctl, 0, 8 * sizeof(int), s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(C.ctl + 4, cap, sizeof(int), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(C.rtol2, &rtol2, sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(C.p, 0, sizeof(double) * n * R, s)) != cudaSuccess)
            return cuda_fail(e, "multigrid start");
        note_launch(2);
        if (X0)
            k_cg_init_x0<R, NV><<<G, 256, 0, s>>>(d0.A, st.v64[0], st.v64[1], B, X0, C.x, C.r, C.part);
        else
            k_cg_init<R><<<G, 256, 0, s>>>(n, B, C.x, C.r, C.part);
        k_cg_start<R><<<1, 32 * R, 0, s>>>(C.part, G, C.bb, C.ctl);
        if ((e = read_ctl()) != cudaSuccess) return cuda_fail(e, "multigrid cg");
        if (hc[0] != QPAT_OK) return fail(hc[0], "multigrid cg: right-hand side not finite");
        if (hc[1] > 0) {
            // the first cycle's first fine smoothing step (later ones come with the CG update)
            const int deg = std::max(1, so.mg_degree);
            if (!f32) {
                VCycle<double, R, NV> c{H, V, W, st, deg, so.mg_ratio, s, timer};
                c.first_fine(C.r);
            } else {
                VCycle<float, R, NV> c{H, V, W, st, deg, so.mg_ratio, s, timer};
                float* b0 = static_cast<float*>(W.b[0]);
                note_launch(1);
                k_d2f_vec<<<G, 256, 0, s>>>(n * R, C.r, b0);
                c.first_fine(b0);
            }
            if (!timer->on) {
                AmgGraph& g = A.graphs[key];
                if (!g.exec) {
                    const int rc = capture(A, g);
                    if (rc != QPAT_OK) return rc;
                }
                if ((e = cudaGraphLaunch(g.exec, s)) != cudaSuccess) return cuda_fail(e, "multigrid graph");
                if ((e = read_ctl()) != cudaSuccess) return cuda_fail(e, "multigrid cg");
                note_launch(hc[2] * g.body_kernels);
            } else {
                while (true) {
                    body(s, 0, 0);
                    if ((e = read_ctl()) != cudaSuccess) return cuda_fail(e, "multigrid cg");
                    timer->collect();
                    if (hc[0] != QPAT_OK || hc[1] == 0) break;
                }
            }
        }
        *iters = hc[2];
        if (hc[0] == QPAT_ENOCONV) return fail(QPAT_ENOCONV, "multigrid cg: iteration cap reached");
        if (hc[0] != QPAT_OK) return fail(hc[0], "multigrid cg: breakdown (p.Ap <= 0 or not finite)");
        if ((e = cudaMemcpyAsync(X, C.x, sizeof(double) * n * R, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return cuda_fail(e, "copy");
        return QPAT_OK;
    }

    int capture(AmgState& A, AmgGraph& g) {
        cudaError_t e = cudaSuccess;
        if (!A.capture && (e = cudaStreamCreateWithFlags(&A.capture, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "multigrid capture stream");
        if ((e = cudaGraphCreate(&g.graph, 0)) != cudaSuccess) return cuda_fail(e, "multigrid graph");
        cudaGraphConditionalHandle cond;
        if ((e = cudaGraphConditionalHandleCreate(&cond, g.graph, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
            return cuda_fail(e, "multigrid graph");
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        if ((e = cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, &np)) != cudaSuccess)
            return cuda_fail(e, "multigrid graph");
        cudaGraph_t bodyg = np.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(A.capture, bodyg, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(e, "multigrid capture");
        body(A.capture, cond, 1);
        g.body_kernels = body_kernels();
        cudaGraph_t out = nullptr;
        const cudaError_t e1 = cudaGetLastError();
        e = cudaStreamEndCapture(A.capture, &out);
        // capturing counted the body's launches once; replays are counted per iteration
        note_launch(-g.body_kernels);
        if (e1 != cudaSuccess) return cuda_fail(e1, "multigrid capture");
        if (e != cudaSuccess) return cuda_fail(e, "multigrid capture");
        if ((e = cudaGraphInstantiate(&g.exec, g.graph, 0)) != cudaSuccess) return cuda_fail(e, "multigrid graph");
        return QPAT_OK;
    }
};

template <int NV>
int dispatch(int R, AmgState& A, const std::string& key, qpat_mesh_s* M, const OpState& st, const SolveOpts& so,
             const AmgHierDev& H, const AmgValues& V, bool f32, AmgVecs& W, AmgCg& C, const double* B, double* X,
             const double* X0, cudaStream_t s, FineTimer* timer, int* iters) {
    if constexpr (NV == 2) {
        return CgSolve<2, 2>{M, st, so, H, V, f32, W, C, s, timer}.run(A, key, B, X, X0, iters);
    } else {
        switch (R) {
            case 1: return CgSolve<1, 1>{M, st, so, H, V, f32, W, C, s, timer}.run(A, key, B, X, X0, iters);
            case 2: return CgSolve<2, 1>{M, st, so, H, V, f32, W, C, s, timer}.run(A, key, B, X, X0, iters);
            case 4: return CgSolve<4, 1>{M, st, so, H, V, f32, W, C, s, timer}.run(A, key, B, X, X0, iters);
            case 8: return CgSolve<8, 1>{M, st, so, H, V, f32, W, C, s, timer}.run(A, key, B, X, X0, iters);
            default: return CgSolve<16, 1>{M, st, so, H, V, f32, W, C, s, timer}.run(A, key, B, X, X0, iters);
        }
    }
}

}  // namespace

int amg_solve(qpat_mesh_s* M, const OpState& st, const SolveOpts& so, int R, const double* B, double* X,
              cudaStream_t s, const double* X0) {
    if (R != 1 && R != 2 && R != 4 && R != 8 && R != 16) return fail(QPAT_EINVAL, "multigrid: R must be 1, 2, 4, 8 or 16");
    if (st.nv == 2 && R != 2) return fail(QPAT_EINVAL, "multigrid: M_delta is solved as 2 right-hand sides");
    if (!(so.mg_ratio > 1.0) || so.mg_degree < 1 || so.mg_degree > 8)
        return fail(QPAT_EINVAL, "multigrid: mg_degree must lie in [1, 8] and mg_ratio exceed 1");
    if (!M->amg) M->amg = new AmgState();
    AmgState& A = *M->amg;
    const int pat = st.kind == OP_PRIOR ? 1 : 0;
    AmgHierDev& H = A.hier[pat];
    if (!H.tried) {
        const int rc = build_hier(M, pat, H);
        if (rc != QPAT_OK) return rc;
    } else if (!H.error.empty()) {
        return fail(QPAT_EINVAL, H.error);
    }
    const bool f32 = so.multigrid == 2 && st.kind == OP_K;
    AmgValues& V = A.vals[st.v64[0]];
    int rc = numeric(M, H, st, V, f32, s);
    if (rc != QPAT_OK) return rc;
    cudaError_t e = cudaSuccess;
    AmgVecs& W = A.vecs[{pat * 64 + R, f32 ? 1 : 0}];
    if (W.xa.empty()) {
        const size_t esz = f32 ? sizeof(float) : sizeof(double);
        for (const LevelDev& d : H.lv) {
            const size_t cnt = size_t(d.A.n) * R * esz;
            W.b.push_back(dalloc<char>(W.allocs, cnt, e));
            W.xa.push_back(dalloc<char>(W.allocs, cnt, e));
            W.xb.push_back(dalloc<char>(W.allocs, cnt, e));
            W.d.push_back(dalloc<char>(W.allocs, cnt, e));
            W.r.push_back(dalloc<char>(W.allocs, cnt, e));
        }
        if (e != cudaSuccess) return cuda_fail(e, "multigrid workspace");
    }
    AmgCg& C = A.cg[R];
    if (!C.r) {
        const size_t nR = size_t(M->h.N) * R;
        C.x = dalloc<double>(C.allocs, nR, e);
        C.r = dalloc<double>(C.allocs, nR, e);
        C.p = dalloc<double>(C.allocs, nR, e);
        C.q = dalloc<double>(C.allocs, nR, e);
        C.z = dalloc<double>(C.allocs, nR, e);
        C.zo = dalloc<double>(C.allocs, nR, e);
        C.part = dalloc<double>(C.allocs, size_t(kRedMaxGrid) * 32, e);
        double* sc = dalloc<double>(C.allocs, 5 * 16 + 1, e);
        C.ctl = dalloc<int>(C.allocs, kCtlActive + 16, e);
        if (e != cudaSuccess) return cuda_fail(e, "multigrid workspace");
        C.bb = sc;
        C.rz = sc + 16;
        C.alpha = sc + 32;
        C.beta = sc + 48;
        C.rr = sc + 64;
        C.rtol2 = sc + 80;
    }
    // the captured iteration depends on these buffers and settings only
    char key[256];
    std::snprintf(key, sizeof key, "%d/%d/%d/%d/%d/%.17g/%p/%p/%p", pat, R, st.nv, int(f32), so.mg_degree, so.mg_ratio,
                  static_cast<const void*>(&V), static_cast<const void*>(st.v64[0]),
                  static_cast<const void*>(st.v64[1]));
    FineTimer timer;
    timer.on = M->timing != 0;
    timer.s = s;
    if (M->timing) cudaEventRecord(M->ev0, s);
    int iters = 0;
    rc = st.nv == 2 ? dispatch<2>(R, A, key, M, st, so, H, V, f32, W, C, B, X, X0, s, &timer, &iters)
                    : dispatch<1>(R, A, key, M, st, so, H, V, f32, W, C, B, X, X0, s, &timer, &iters);
    if (timer.on) {
        cudaStreamSynchronize(s);
        timer.collect();
        M->mg_fine_ms += timer.ms;
        M->mg_fine_launches += timer.launches;
    }
    if ((e = cudaGetLastError()) != cudaSuccess && rc == QPAT_OK) rc = cuda_fail(e, "multigrid launch");
    if (M->timing) {
        cudaEventRecord(M->ev1, s);
        cudaEventSynchronize(M->ev1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, M->ev0, M->ev1);
        M->pcg_ms += ms;
    }
    M->stats.pcg_iters += iters;
    M->stats.rhs_iters += int64_t(iters) * R;
    M->stats.solves += R;
    M->stats.launches += 1;
    return rc;
}

int amg_levels(qpat_mesh_s* M, int prior, int64_t* rows, int max_levels) {
    if (!M->amg) return 0;
    const AmgHierDev& H = M->amg->hier[prior ? 1 : 0];
    const int L = int(H.lv.size());
    for (int l = 0; l < std::min(L, max_levels); ++l) rows[l] = H.lv[size_t(l)].A.n;
    return L;
}

void amg_release(qpat_mesh_s* M) {
    if (!M->amg) return;
    AmgState& A = *M->amg;
    for (auto& H : A.hier)
        for (void* p : H.allocs) cudaFree(p);
    for (auto& kv : A.vals)
        for (void* p : kv.second.allocs) cudaFree(p);
    for (auto& kv : A.vecs)
        for (void* p : kv.second.allocs) cudaFree(p);
    for (auto& kv : A.cg)
        for (void* p : kv.second.allocs) cudaFree(p);
    for (auto& kv : A.graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    if (A.capture) cudaStreamDestroy(A.capture);
    delete M->amg;
    M->amg = nullptr;
}

}  // namespace qpat
