// Persistent fused preconditioned conjugate gradients.
//
// The paper solves with K (Appendix) and with M_delta (Sec. 4, one solve per
// LSQR round) but does not name a solver; both are symmetric positive
// definite, so this library uses preconditioned conjugate gradients.  One
// cooperative launch runs the whole iteration: every CTA owns a fixed set of
// node patches and, per iteration,
//   phase A: forms p = z + beta p_old on its touched nodes in shared memory
//            (z = M^-1 r read from its owner, or D^-1 r formed on the fly),
//            writes p on its owned nodes, applies the operator and keeps
//            q = A p on its owned nodes, accumulating p.q;
//   phase B: x += alpha p, r -= alpha q on its owned nodes, z = M^-1 r
//            (Jacobi D^-1, or the patch-local Chebyshev polynomial below),
//            accumulating r.z and r.r.
// Each phase ends with a grid-wide reduction behind a bounded grid barrier:
// every CTA writes its partial sums, the last CTA to arrive adds all of them
// in a fixed order, publishes the totals and releases the others, so every
// CTA takes the same decisions from bit-identical scalars.  R right-hand
// sides share one launch with their own alpha and beta (block form of the
// stacked illuminations of Sec. 4); node vectors are N x R node-major and
// are moved as 16-byte vectors (4 floats or 2 doubles of consecutive RHS)
// wherever R allows.  Scalars are accumulated in FP64 for either T.
#include <cuda/atomic>
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "launch.h"

namespace qpat {

namespace {

template <typename T>
struct PcgArgs {
    MeshDev m;
    OpParams<T> op;
    const T* invdiag;
    const T* b;
    T* x;
    T* r;
    T* p0;
    T* p1;
    T* q;
    double* partials;
    unsigned* bar;
    int* status;
    int* iters;
    double* stats;
    double rtol2;
    int maxit;
    long long spin_limit;
    T* z;   // optional: z = D^-1 r stored by the owner (two-reduction kernel)
    // optional resume of a previous run (two-reduction kernel, reliable
    // updates): gamma[r] rescales the previous direction to this run's RHS
    // scaling; rz_state[r] and *pbuf carry r.z of the previous direction and
    // the buffer (p0/p1) holding it, and are rewritten at exit
    const double* resume_gamma;
    double* rz_state;
    int* pbuf;
    T* r1;  // single-reduction variant
    T* s0;
    T* s1;
    T* w1;
    // patch-local Chebyshev preconditioner (two-reduction kernel on assembled
    // operators with z stored): degree (0 = Jacobi) and a device pointer to
    // an upper bound of the spectrum of D^-1 A
    int poly_deg = 0;
    const double* poly_hi = nullptr;
};

// kMaxGrid, kMaxNS and kDefaultSpinLimit: launch.h

// ---------------------------------------------------------------- vectors
template <typename T, int VW>
struct VecT;
template <>
struct VecT<float, 4> {
    using type = float4;
};
template <>
struct VecT<double, 2> {
    using type = double2;
};
template <typename T>
struct VecT<T, 1> {
    using type = T;
};

template <typename T, int R, bool kVec>
__host__ __device__ constexpr int vec_width() {
    if (!kVec) return 1;
    if (sizeof(T) == 4) return R % 4 == 0 ? 4 : 1;
    return R % 2 == 0 ? 2 : 1;
}

template <typename T, int VW>
__device__ __forceinline__ void vld_cg(const T* p, T (&v)[VW]) {
    if constexpr (VW == 1) {
        v[0] = __ldcg(p);
    } else {
        const auto t = __ldcg(reinterpret_cast<const typename VecT<T, VW>::type*>(p));
        memcpy(v, &t, sizeof(t));
    }
}
template <typename T, int VW>
__device__ __forceinline__ void vld(const T* p, T (&v)[VW]) {
    if constexpr (VW == 1) {
        v[0] = *p;
    } else {
        const auto t = *reinterpret_cast<const typename VecT<T, VW>::type*>(p);
        memcpy(v, &t, sizeof(t));
    }
}
template <typename T, int VW>
__device__ __forceinline__ void vst(T* p, const T (&v)[VW]) {
    if constexpr (VW == 1) {
        *p = v[0];
    } else {
        typename VecT<T, VW>::type t;
        memcpy(&t, v, sizeof(t));
        *reinterpret_cast<typename VecT<T, VW>::type*>(p) = t;
    }
}

// inverse diagonal of the VW right-hand sides [r0, r0 + VW) of node g
template <typename T, int VW, int OP>
__device__ __forceinline__ void dinv_vec(const T* invdiag, int g, int r0, T (&d)[VW]) {
    if constexpr (OP == OP_PRIOR || OP == OP_CSR2) {
        if constexpr (VW == 1) {
            d[0] = __ldg(invdiag + 2 * g + r0);
        } else {
            const auto t = __ldg(reinterpret_cast<const typename VecT<T, VW>::type*>(invdiag + 2 * g + r0));
            memcpy(d, &t, sizeof(t));
        }
    } else {
        const T v = __ldg(invdiag + g);
#pragma unroll
        for (int c = 0; c < VW; ++c) d[c] = v;
    }
}

// (A x) of owned row g for this thread's right-hand sides [r0, r0 + VW),
// x staged in shared memory (touched x R).  The row's column ids and values
// are fetched kChunk at a time into registers before any is used, so that
// kChunk independent loads per thread are in flight at once (a thread-per-row
// loop that consumes each entry as it arrives waits one memory latency per
// entry).  Entries past the row length are not loaded; their multiply-adds
// run on zeros (predicating them off was measured slower).  Chunk widths: K
// rows of Kuhn meshes hold 15 entries (two chunks of 8), the prior's
// stiffness-only rows 7 (one chunk of 7, no wasted FP64 multiply-add; FP64
// issue slots bound the assembled FP64 solves on GB300).
constexpr int kChunk = 8;
constexpr int kChunkPrior = 7;
constexpr int kChunkK64 = 15;  // FP64 K rows: one chunk of 15 (no multiply-add on padding)
constexpr int kUnroll = 2;  // touched nodes a thread stages at once
//
// kLocal: only the couplings among the patch's owned nodes (local column ids
// below nloc; the owned nodes come first in a patch's node list) take part.
template <typename T, int R, int VW, int OP, bool kLocal = false>
__device__ __forceinline__ void sell_row(const MeshDev& m, const OpParams<T>& op, const T* xs, int g, int r0,
                                         T (&acc)[VW], int nloc = 0) {
    constexpr int NL = OP == OP_CSR2 ? VW : 1;  // distinct value sets this thread reads
    constexpr int CH = OP == OP_CSR2 ? kChunkPrior : (sizeof(T) == 8 ? kChunkK64 : kChunk);
    const int64_t base = m.sell_ptr[g >> 5] * 32 + (g & 31);
    const int len = m.sell_len[g];
    const T* vp[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) vp[q] = (OP == OP_CSR2 && r0 + q == 1) ? op.v1 : op.v0;
#pragma unroll
    for (int c = 0; c < VW; ++c) acc[c] = T(0);
    for (int k0 = 0; k0 < len; k0 += CH) {
        int col[CH];
        T v[CH][NL];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int64_t idx = base + int64_t(k0 + j) * 32;
            const bool ok = k0 + j < len;
            col[j] = ok ? int(__ldg(m.sell_col + idx)) : 0;
#pragma unroll
            for (int q = 0; q < NL; ++q) v[j][q] = ok ? __ldg(vp[q] + idx) : T(0);
        }
        if constexpr (kLocal) {
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                const bool in = col[j] < nloc;
                col[j] = in ? col[j] : 0;
#pragma unroll
                for (int q = 0; q < NL; ++q) v[j][q] = in ? v[j][q] : T(0);
            }
        }
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            T xv[VW];
            vld(xs + col[j] * R + r0, xv);
#pragma unroll
            for (int c = 0; c < VW; ++c) acc[c] += v[j][NL == 1 ? 0 : c] * xv[c];
        }
    }
}

// ---------------------------------------------------------------- grid reduction
// Sum over the grid of NQ x R values; thread t holds acc[q][c] for RHS
// (t % NP) * VW + c.  Totals land in out[q * R + r] (shared) in every CTA.
// Each thread's partial sums (a few terms) and the sums across a warp are
// formed in the solve's own precision T; from the warp totals on, the sums
// (across warps, then across CTAs in a fixed order) run in FP64.  GB300
// issues FP64 at 1/64 of the FP32 rate, so per-element FP64 terms, FP32->FP64
// conversions and FP64 warp shuffles would dominate an FP32 iteration.
template <int NQ, int VW, int NP, typename T>
__device__ __forceinline__ bool grid_reduce(T (&acc)[NQ][VW], double* scratch, double* partials, int& red_id,
                                            unsigned* bar, int* status, long long limit, double* out, int cta,
                                            int ncta) {
    constexpr int R = VW * NP, NS = NQ * R;
    __shared__ int s_last;
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // Warp sums by reduce-scatter: the NQ x VW values of a thread are padded
    // to P2 (a power of two); at each shuffle level the lanes whose level bit
    // is clear keep the lower half of their set and the others the upper
    // half, each adding its partner's copy, so the set halves instead of
    // every lane adding every value at every level.  Lanes that differ in a
    // bit below NP hold different RHS blocks and are never paired.
    constexpr int V = NQ * VW;
    constexpr int P2 = V <= 1 ? 1 : V <= 2 ? 2 : V <= 4 ? 4 : V <= 8 ? 8 : 16;
    static_assert(V <= 16, "at most 16 values per thread");
    T v[P2];
#pragma unroll
    for (int f = 0; f < P2; ++f) v[f] = f < V ? acc[f / VW][f % VW] : T(0);
    int base = 0, nkeep = P2, dup_mask = 0;
#pragma unroll
    for (int o = 16; o >= NP; o >>= 1) {
        if (nkeep > 1) {
            const int h = nkeep / 2;
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const T send = up ? v[i] : v[h + i];
                const T recv = __shfl_xor_sync(0xffffffffu, send, o);
                v[i] = (up ? v[h + i] : v[i]) + recv;
            }
            if (up) base += h;
            nkeep = h;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
            dup_mask |= o;  // both partners now hold the same sum
        }
    }
    if ((lane & dup_mask) == 0) {
        const int part = lane & (NP - 1);
#pragma unroll
        for (int i = 0; i < nkeep; ++i) {
            const int f = base + i;
            if (f < V) scratch[warp * NS + (f / VW) * R + part * VW + (f % VW)] = double(v[i]);
        }
    }
    __syncthreads();
    double* part = partials + size_t(red_id & 1) * kMaxGrid * kMaxNS;
    double* res = partials + size_t(2) * kMaxGrid * kMaxNS + (red_id & 1) * kMaxNS;
    ++red_id;
    if (threadIdx.x < NS) {
        double a = 0.0;
        for (int w = 0; w < nw; ++w) a += scratch[w * NS + threadIdx.x];
        part[size_t(cta) * NS + threadIdx.x] = a;
    }
    __syncthreads();
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(bar[0]);
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> gen(bar[1]);
    unsigned g = 0;
    if (threadIdx.x == 0) {
        g = gen.load(cuda::memory_order_acquire);
        __threadfence();
        const unsigned old = cnt.fetch_add(1u, cuda::memory_order_acq_rel);
        s_last = old == unsigned(ncta) - 1;
        s_ok = 1;
    }
    __syncthreads();
    if (s_last) {
        // the last CTA adds the partials of every CTA in a fixed order
        __threadfence();
        for (int s = warp; s < NS; s += nw) {
            // four independent chains keep four loads per lane in flight
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            int j = lane;
            for (; j + 96 < ncta; j += 128) {
                a0 += __ldcg(part + size_t(j) * NS + s);
                a1 += __ldcg(part + size_t(j + 32) * NS + s);
                a2 += __ldcg(part + size_t(j + 64) * NS + s);
                a3 += __ldcg(part + size_t(j + 96) * NS + s);
            }
            for (; j < ncta; j += 32) a0 += __ldcg(part + size_t(j) * NS + s);
            double a = (a0 + a1) + (a2 + a3);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) res[s] = a;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            cnt.store(0u, cuda::memory_order_relaxed);
            gen.fetch_add(1u, cuda::memory_order_release);
        }
    } else if (threadIdx.x == 0) {
        long long spins = 0;
        while (gen.load(cuda::memory_order_acquire) == g) {
            if (++spins > limit) {
                atomicExch(status, QPAT_ETIMEOUT);
                s_ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
    if (!s_ok) return false;
    if (threadIdx.x < NS) out[threadIdx.x] = __ldcg(res + threadIdx.x);
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------- preconditioner
// Patch-local Chebyshev preconditioner: block Jacobi over the CTA patches,
// each block A_pp (the couplings among a patch's owned nodes) inverted
// approximately by the polynomial of `deg` steps of the Chebyshev iteration
// for A_pp z = r with diagonal scaling, from z = 0, on the interval
// [lo, hi] of B = D^-1 A_pp:  z = p(B) v with v = D^-1 r and p of degree
// deg.  M^-1 = p(B) D^-1 is symmetric (D^-1/2 p(D^-1/2 A_pp D^-1/2) D^-1/2
// per block) and positive definite whenever hi bounds the spectrum (the
// Chebyshev residual polynomial 1 - x p(x) stays inside (-1, 1) on (0, hi]),
// so ordinary PCG applies.  p is evaluated in Horner form,
//   w = a_deg v ;  w = a_j v + B w  (j = deg-1 .. 0) ;  z = w,
// one local operator sweep and two FP64 operations per row and step (FP64
// issue slots are the scarce resource on GB300), and no grid barrier.
constexpr double kPolyRatio = 50.0;  // lo = hi / kPolyRatio

// Monomial coefficients a_0..a_deg of p.  With polynomials in x standing for
// the vectors of the iteration applied to v: the scaled residual
// S_0 = 1, the step D_0 = 1/theta, the iterate P_0 = D_0, and per step
//   S_{k+1} = S_k - x D_k ;  D_{k+1} = rho_{k+1} rho_k D_k + (2 rho_{k+1} / delta) S_{k+1} ;
//   P_{k+1} = P_k + D_{k+1},
// where theta, delta are the centre and half width of [lo, hi],
// rho_0 = delta / theta and rho_{k+1} = 1 / (2 theta / delta - rho_k).
__device__ __forceinline__ void cheb_coeffs(double hi, int deg, double* acoef) {
    if (!(hi > 0.0) || !isfinite(hi)) hi = 2.0;
    hi *= 1.01;  // margin over the FP64 rounding of the bound
    const double lo = hi / kPolyRatio;
    const double th = 0.5 * (hi + lo), dl = 0.5 * (hi - lo), sg = th / dl;
    double S[kMaxPolyDegree + 2] = {}, D[kMaxPolyDegree + 2] = {}, P[kMaxPolyDegree + 2] = {};
    S[0] = 1.0;
    D[0] = 1.0 / th;
    P[0] = D[0];
    double rho = 1.0 / sg;
    for (int k = 0; k < deg; ++k) {
        for (int j = k + 1; j >= 1; --j) S[j] -= D[j - 1];  // S -= x D (D has degree k)
        const double rn = 1.0 / (2.0 * sg - rho);
        const double c1 = rn * rho, c2 = 2.0 * rn / dl;
        for (int j = 0; j <= k + 1; ++j) {
            D[j] = c1 * D[j] + c2 * S[j];
            P[j] += D[j];
        }
        rho = rn;
    }
    // p / |a_deg| instead of p: a positive factor in M^-1 leaves the PCG
    // iterates x unchanged (beta is a ratio of r.z values, alpha absorbs the
    // scale of the direction), and the Horner start w = +-v then needs no
    // multiply.  acoef[deg] = +-1 carries the sign of a_deg.
    for (int j = 0; j <= deg; ++j) acoef[j] = P[j] / fabs(P[deg]);
}

// The deg Horner steps on one patch.  On entry every thread has written, for
// its owned rows (offset li * R + r0), cV = v = D^-1 r and cW0 = a_deg v
// (a_deg = +-1 after the normalisation in cheb_coeffs); on exit the returned
// buffer holds z.  Block-wide barriers separate the steps.
template <typename T, int R, int VW, int NP, int OP>
__device__ __forceinline__ T* cheb_patch(const PcgArgs<T>& a, int ob, int nown, int r0, int deg, const double* acoef,
                                         const T* cV, T* cW0, T* cW1) {
    for (int s = 0; s < deg; ++s) {
        const T* src = (s & 1) ? cW1 : cW0;
        T* dst = (s & 1) ? cW0 : cW1;
        const T aj = T(acoef[deg - 1 - s]);
        __syncthreads();  // w complete
        for (int i = threadIdx.x; i < nown * NP; i += blockDim.x) {
            const int li = i / NP;
            const int g = ob + li;
            const int o = li * R + r0;
            T y[VW], vv[VW], d[VW];
            sell_row<T, R, VW, OP, true>(a.m, a.op, src, g, r0, y, nown);
            vld(cV + o, vv);
            dinv_vec<T, VW, OP>(a.invdiag, g, r0, d);
#pragma unroll
            for (int c = 0; c < VW; ++c) y[c] = aj * vv[c] + d[c] * y[c];
            vst(dst + o, y);
        }
    }
    __syncthreads();  // nobody reads this patch's buffers any more
    return (deg & 1) ? cW1 : cW0;
}

// ---------------------------------------------------------------- the solver
template <typename T, int R, int OP, bool kPoly = false, int NT = kThreads>
__device__ __forceinline__ void pcg_body(const PcgArgs<T>& a, const int cta, const int ncta) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool kCsr = (OP == OP_CSR1 || OP == OP_CSR2);
    constexpr int VW = vec_width<T, R, kCsr>();
    constexpr int NP = R / VW;
    PatchSmem<T, R> s;
    if constexpr (kCsr) {
        s.xin = reinterpret_cast<T*>(smem_raw);  // assembled operators stage p only
    } else {
        s.carve(reinterpret_cast<T*>(smem_raw), a.m.max_touched, a.m.max_own);
    }
    __shared__ double scratch[(NT / 32) * kMaxNS];
    __shared__ double red[kMaxNS];
    __shared__ double bb[R], rz[R], rz_old[R], rr[R], alpha[R], beta[R], zcoef[R];
    __shared__ int s_flag;

    const MeshDev& m = a.m;
    const int P = m.P;
    const int part = threadIdx.x % NP;  // this thread's RHS block [part*VW, part*VW + VW)
    const int r0 = part * VW;
    const bool zs = a.z != nullptr;
    const bool resumed = a.resume_gamma != nullptr;
    const int pb_in = a.pbuf ? *a.pbuf : 0;
    const int off = resumed ? (pb_in == 0 ? 1 : 0) : 0;  // iteration 0 reads p_old from buffer pb_in
    int red_id = 0;

    // patch-local Chebyshev preconditioner: its four owned-row vectors
    // overlay the staged p (phase A is over whenever they are in use)
    const int deg = (kPoly && kCsr && zs) ? a.poly_deg : 0;  // kPoly: a separate instantiation keeps
                                                              // the Jacobi kernel's registers unchanged
    __shared__ double pco[kMaxPolyDegree + 1];
    T *cV = nullptr, *cW0 = nullptr, *cW1 = nullptr;
    bool top_neg = false;  // a_deg = -1: the Horner start is -v
    if (deg > 0) {
        const size_t stride = size_t(m.max_own) * R;
        cV = reinterpret_cast<T*>(smem_raw);
        cW0 = cV + stride;
        cW1 = cW0 + stride;
        if (threadIdx.x == 0) cheb_coeffs(__ldcg(a.poly_hi), deg, pco);
        __syncthreads();
        top_neg = pco[deg] < 0.0;
    }

    // ---- initial residual r = b (x0 = 0)
    {
        T acc[3][VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) acc[0][c] = acc[1][c] = acc[2][c] = 0.0;
        for (int p = cta; p < P; p += ncta) {
            const int ob = __ldg(m.own_begin + p), nown = __ldg(m.own_begin + p + 1) - ob;
            for (int i = threadIdx.x; i < nown * NP; i += blockDim.x) {
                const int g = ob + i / NP;
                const size_t e = size_t(g) * R + r0;
                T bv[VW], d[VW], zero[VW], zv[VW];
                vld(a.b + e, bv);
                dinv_vec<T, VW, OP>(a.invdiag, g, r0, d);
#pragma unroll
                for (int c = 0; c < VW; ++c) {
                    zero[c] = T(0);
                    zv[c] = d[c] * bv[c];
                    acc[0][c] += bv[c] * bv[c];
                    if (deg == 0) acc[1][c] += bv[c] * zv[c];
                }
                vst(a.x + e, zero);
                vst(a.r + e, bv);
                if (deg > 0) {
                    const int o = (i / NP) * R + r0;
                    vst(cV + o, zv);
#pragma unroll
                    for (int c = 0; c < VW; ++c) zv[c] = top_neg ? -zv[c] : zv[c];
                    vst(cW0 + o, zv);
                } else if (a.z) {
                    vst(a.z + e, zv);
                }
            }
            if (deg > 0) {
                const T* zw = cheb_patch<T, R, VW, NP, OP>(a, ob, nown, r0, deg, pco, cV, cW0, cW1);
                for (int i = threadIdx.x; i < nown * NP; i += blockDim.x) {
                    const size_t e = size_t(ob + i / NP) * R + r0;
                    T bv[VW], zv[VW];
                    vld(a.b + e, bv);
                    vld(zw + (i / NP) * R + r0, zv);
#pragma unroll
                    for (int c = 0; c < VW; ++c) acc[1][c] += bv[c] * zv[c];
                    vst(a.z + e, zv);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < VW; ++c) acc[2][c] = acc[0][c];
        if (!grid_reduce<3, VW, NP>(acc, scratch, a.partials, red_id, a.bar, a.status, a.spin_limit, red, cta,
                                    ncta))
            return;
        if (threadIdx.x < R) {
            bb[threadIdx.x] = red[threadIdx.x];
            rz[threadIdx.x] = red[R + threadIdx.x];
            rr[threadIdx.x] = red[2 * R + threadIdx.x];
            // resumed: the previous direction's r.z in this run's scaling
            rz_old[threadIdx.x] = resumed ? a.resume_gamma[threadIdx.x] * a.resume_gamma[threadIdx.x] *
                                                a.rz_state[threadIdx.x]
                                          : 1.0;
        }
        __syncthreads();
    }

    int it = 0;
    for (;;) {
        // ---- convergence / cap (uniform over CTAs)
        if (threadIdx.x == 0) {
            int any = 0;
            for (int r = 0; r < R; ++r) any |= (rr[r] > a.rtol2 * bb[r]) ? 1 : 0;
            s_flag = any;
        }
        __syncthreads();
        if (!s_flag) break;
        if (it >= a.maxit) {
            if (cta == 0 && threadIdx.x == 0) atomicCAS(a.status, 0, QPAT_ENOCONV);
            break;
        }
        const bool prev = it > 0 || resumed;  // a previous direction exists
        if (threadIdx.x < R) {
            const int r = threadIdx.x;
            const bool act = rr[r] > a.rtol2 * bb[r];
            double b_ = (!prev || !act || !(rz_old[r] > 0.0)) ? 0.0 : rz[r] / rz_old[r];
            // resumed run, first step: p = z + beta (gamma p_prev)
            if (it == 0 && resumed) b_ *= a.resume_gamma[r];
            // a converged (frozen) RHS keeps its last direction unchanged, so
            // that a resumed run continues from a conjugate direction
            beta[r] = act ? b_ : (prev ? 1.0 : 0.0);
            zcoef[r] = act ? 1.0 : 0.0;
        }
        __syncthreads();

        T* pc = ((it + off) & 1) ? a.p1 : a.p0;
        const T* pp = ((it + off) & 1) ? a.p0 : a.p1;
        T bt[VW];
        bool zon[VW];  // a select, not an FP64 multiply by 0 / 1
#pragma unroll
        for (int c = 0; c < VW; ++c) {
            bt[c] = T(beta[r0 + c]);
            zon[c] = zcoef[r0 + c] != 0.0;
        }

        // ---- phase A: p = D^-1 r + beta p_old on touched nodes, q = A p on owned nodes
        T accA[1][VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) accA[0][c] = T(0);
        for (int p = cta; p < P; p += ncta) {
            const int nb = __ldg(m.node_ptr + p), nt = __ldg(m.node_ptr + p + 1) - nb;
            const int ob = __ldg(m.own_begin + p), nown = __ldg(m.own_begin + p + 1) - ob;
            if constexpr (!kCsr) stage_static<T, R>(m, nb, nt, s, a.op);
            // kUnroll touched nodes per thread in flight (a spare slot repeats the first node)
            for (int i0 = threadIdx.x; i0 < nt * NP; i0 += kUnroll * blockDim.x) {
                int li[kUnroll];
                T rv[kUnroll][VW], d[kUnroll][VW], po[kUnroll][VW];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const int i = i0 + u * blockDim.x;
                    li[u] = (i < nt * NP ? i : i0) / NP;
                    const int g = __ldg(m.nodes + nb + li[u]);
                    const size_t e = size_t(g) * R + r0;
                    if (zs) {
                        vld_cg(a.z + e, rv[u]);  // z = D^-1 r from its owner
                    } else {
                        vld_cg(a.r + e, rv[u]);
                        dinv_vec<T, VW, OP>(a.invdiag, g, r0, d[u]);
                    }
                    if (prev) vld_cg(pp + e, po[u]);
                }
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    T pv[VW];
#pragma unroll
                    for (int c = 0; c < VW; ++c)
                        pv[c] = (zon[c] ? (zs ? rv[u][c] : d[u][c] * rv[u][c]) : T(0)) +
                                (prev ? bt[c] * po[u][c] : T(0));
                    if (u == 0 || i0 + u * int(blockDim.x) < nt * NP) vst(s.xin + li[u] * R + r0, pv);
                }
            }
            if constexpr (!kCsr)
                for (int i = threadIdx.x; i < nown * R; i += blockDim.x) s.yout[i] = T(0);
            __syncthreads();
            if constexpr (kCsr) {
                // thread per (owned row, RHS block): sliced-ELLPACK row from shared p
                for (int i = threadIdx.x; i < nown * NP; i += blockDim.x) {
                    const int li = i / NP;
                    const int g = ob + li;
                    T acc[VW];
                    sell_row<T, R, VW, OP>(m, a.op, s.xin, g, r0, acc);
                    T pv[VW];
                    vld(s.xin + li * R + r0, pv);
                    const size_t e = size_t(g) * R + r0;
                    vst(pc + e, pv);
                    vst(a.q + e, acc);
#pragma unroll
                    for (int c = 0; c < VW; ++c) accA[0][c] += pv[c] * acc[c];
                }
                __syncthreads();
            } else {
                patch_elements<T, R, OP>(m, p, nown, s, a.op);
                __syncthreads();
                for (int i = threadIdx.x; i < nown * R; i += blockDim.x) {
                    const size_t e = size_t(ob) * R + i;
                    const T pv = s.xin[i];
                    T qv = s.yout[i];
                    if (OP == OP_PRIOR) qv += a.op.delta * pv;
                    pc[e] = pv;
                    a.q[e] = qv;
                    accA[0][0] += pv * qv;
                }
                __syncthreads();
            }
        }
        if (!grid_reduce<1, VW, NP>(accA, scratch, a.partials, red_id, a.bar, a.status, a.spin_limit, red, cta,
                                    ncta))
            return;
        if (threadIdx.x == 0) {
            int bad = 0;
            for (int r = 0; r < R; ++r) {
                const bool act = rr[r] > a.rtol2 * bb[r];
                const double pq = red[r];
                if (act && !(pq > 0.0 && isfinite(pq))) bad = 1;
                alpha[r] = act && pq > 0.0 ? rz[r] / pq : 0.0;
            }
            s_flag = bad;
        }
        __syncthreads();
        if (s_flag) {
            if (cta == 0 && threadIdx.x == 0) atomicCAS(a.status, 0, QPAT_EBREAKDOWN);
            break;
        }

        // ---- phase B: x += alpha p, r -= alpha q; r.D^-1 r and r.r
        T accB[2][VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) accB[0][c] = accB[1][c] = 0.0;
        {
            T al[VW];
#pragma unroll
            for (int c = 0; c < VW; ++c) al[c] = T(alpha[r0 + c]);
            // this CTA's patches in the reverse order of phase A: the patches
            // it handled last there (their operator slices and p, q still
            // partly in L2) come first here, and the next phase A starts
            // again where this one ends
            const int nmine = cta < P ? (P - 1 - cta) / ncta + 1 : 0;
            for (int jp = nmine - 1; jp >= 0; --jp) {
                const int p = cta + jp * ncta;
                const int ob = __ldg(m.own_begin + p), nown = __ldg(m.own_begin + p + 1) - ob;
                for (int i = threadIdx.x; i < nown * NP; i += blockDim.x) {
                    const int g = ob + i / NP;
                    const size_t e = size_t(g) * R + r0;
                    T pv[VW], qv[VW], xv[VW], rv[VW], d[VW];
                    vld(pc + e, pv);
                    vld(a.q + e, qv);
                    vld(a.x + e, xv);
                    vld(a.r + e, rv);
                    dinv_vec<T, VW, OP>(a.invdiag, g, r0, d);
                    T zv[VW];
#pragma unroll
                    for (int c = 0; c < VW; ++c) {
                        xv[c] += al[c] * pv[c];
                        rv[c] -= al[c] * qv[c];
                        zv[c] = d[c] * rv[c];
                        if (deg == 0) accB[0][c] += rv[c] * zv[c];
                        accB[1][c] += rv[c] * rv[c];
                    }
                    vst(a.x + e, xv);
                    vst(a.r + e, rv);
                    if (deg > 0) {
                        const int o = (i / NP) * R + r0;
                        vst(cV + o, zv);
#pragma unroll
                        for (int c = 0; c < VW; ++c) zv[c] = top_neg ? -zv[c] : zv[c];
                        vst(cW0 + o, zv);
                    } else if (zs) {
                        vst(a.z + e, zv);
                    }
                }
                if (deg > 0) {
                    const T* zw = cheb_patch<T, R, VW, NP, OP>(a, ob, nown, r0, deg, pco, cV, cW0, cW1);
                    for (int i = threadIdx.x; i < nown * NP; i += blockDim.x) {
                        const size_t e = size_t(ob + i / NP) * R + r0;
                        T rv[VW], zv[VW];
                        vld(a.r + e, rv);  // written by this thread above
                        vld(zw + (i / NP) * R + r0, zv);
#pragma unroll
                        for (int c = 0; c < VW; ++c) accB[0][c] += rv[c] * zv[c];
                        vst(a.z + e, zv);
                    }
                }
            }
        }
        if (!grid_reduce<2, VW, NP>(accB, scratch, a.partials, red_id, a.bar, a.status, a.spin_limit, red, cta,
                                    ncta))
            return;
        if (threadIdx.x < R) {
            const int r = threadIdx.x;
            const bool act = rr[r] > a.rtol2 * bb[r];
            if (act) {
                rz_old[r] = rz[r];
                rz[r] = red[r];
                rr[r] = red[R + r];
            }
        }
        __syncthreads();
        ++it;
    }
    if (cta == 0 && threadIdx.x < R) {
        a.stats[threadIdx.x] = rr[threadIdx.x];
        a.stats[R + threadIdx.x] = bb[threadIdx.x];
        if (a.rz_state) a.rz_state[threadIdx.x] = rz_old[threadIdx.x];  // r.z that formed the last p
        if (threadIdx.x == 0) {
            *a.iters = it;
            if (a.pbuf && it > 0) *a.pbuf = (it - 1 + off) & 1;
        }
    }
}

// single-reduction kernel on assembled operators: at least 4 resident CTAs
// per SM (a 64-register cap; uncapped it needs ~100 and halves the grid)
template <int OP>
constexpr int min_ctas() {
    return (OP == OP_CSR1 || OP == OP_CSR2) ? 4 : 1;
}

template <typename T, int R, int OP, bool kPoly = false>
__global__ void __launch_bounds__(kThreads) k_pcg(PcgArgs<T> a) {
    pcg_body<T, R, OP, kPoly>(a, blockIdx.x, gridDim.x);
}

// The two-block M_delta solver (R = 2, two value sets, patch-local
// preconditioner) held to three resident CTAs per SM (78 registers, no
// spills): at its unbounded 107 registers only two fit, 16 warps per SM for
// a kernel bound by FP64 issue and shared-memory latency.
template <typename T, int R, int OP, bool kPoly = false>
__global__ void __launch_bounds__(kThreads, 3) k_pcg_occ3(PcgArgs<T> a) {
    pcg_body<T, R, OP, kPoly>(a, blockIdx.x, gridDim.x);
}

// The same solver with kWideThreads threads per CTA, for the launches whose
// shared memory (the staged direction or the preconditioner's owned-row
// vectors of many RHS on large patches) leaves room for one CTA per SM only:
// twice the warps per SM to hide the shared-memory and FP64 latencies.
constexpr int kWideThreads = 2 * kThreads;
template <typename T, int R, int OP, bool kPoly = false>
__global__ void __launch_bounds__(kWideThreads) k_pcg_wide(PcgArgs<T> a) {
    pcg_body<T, R, OP, kPoly, kWideThreads>(a, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------- single-reduction variant
// Chronopoulos-Gear form of the same Jacobi-PCG (assembled operators only):
// with u = D^-1 r, w = A u and s = A p kept by recurrence,
//   x += alpha p,  r -= alpha s,  u = D^-1 r,  w = A u,
//   gamma = r.u,  delta = w.u   (one grid reduction per iteration),
//   beta = gamma / gamma_old,  alpha = gamma / (delta - beta gamma / alpha_old),
//   p = u + beta p,  s = w + beta s.
// r, s and w are read on the halo and double-buffered; every CTA updates s
// and r redundantly on its touched nodes from the previous w, s and r, so the
// new u is staged without a second barrier.  In exact arithmetic the iterates
// equal those of pcg_body.
template <typename T, int R, int OP>
__device__ __forceinline__ void pcg1_body(const PcgArgs<T>& a, const int cta, const int ncta) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int VW = vec_width<T, R, true>();
    constexpr int NP = R / VW;
    T* su = reinterpret_cast<T*>(smem_raw);  // touched x R: the new u
    __shared__ double scratch[(kThreads / 32) * kMaxNS];
    __shared__ double red[kMaxNS];
    __shared__ double bb[R], gam[R], alpha[R], beta[R], rr[R];
    __shared__ int s_flag;

    const MeshDev& m = a.m;
    const int P = m.P;
    const int part = threadIdx.x % NP;
    const int r0 = part * VW;
    int red_id = 0;
    T* const u = a.p1;  // owned u
    T* const p = a.p0;  // owned p

    // ---- start: x = 0, r = b, u = D^-1 b, w = A u; gamma, delta, |b|^2
    {
        T acc[3][VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) acc[0][c] = acc[1][c] = acc[2][c] = 0.0;
        for (int pt = cta; pt < P; pt += ncta) {
            const int nb = __ldg(m.node_ptr + pt), nt = __ldg(m.node_ptr + pt + 1) - nb;
            const int ob = __ldg(m.own_begin + pt), nown = __ldg(m.own_begin + pt + 1) - ob;
            for (int i = threadIdx.x; i < nt * NP; i += blockDim.x) {
                const int li = i / NP;
                const int g = __ldg(m.nodes + nb + li);
                T bv[VW], d[VW], uv[VW];
                vld(a.b + size_t(g) * R + r0, bv);
                dinv_vec<T, VW, OP>(a.invdiag, g, r0, d);
#pragma unroll
                for (int c = 0; c < VW; ++c) uv[c] = d[c] * bv[c];
                vst(su + li * R + r0, uv);
            }
            __syncthreads();
            for (int i = threadIdx.x; i < nown * NP; i += blockDim.x) {
                const int li = i / NP, g = ob + li;
                const size_t e = size_t(g) * R + r0;
                T wv[VW], uv[VW], bv[VW], zero[VW];
                sell_row<T, R, VW, OP>(m, a.op, su, g, r0, wv);
                vld(su + li * R + r0, uv);
                vld(a.b + e, bv);
#pragma unroll
                for (int c = 0; c < VW; ++c) {
                    zero[c] = T(0);
                    acc[0][c] += bv[c] * uv[c];
                    acc[1][c] += wv[c] * uv[c];
                    acc[2][c] += bv[c] * bv[c];
                }
                vst(a.q + e, wv);
                vst(u + e, uv);
                vst(a.r + e, bv);
                vst(a.x + e, zero);
            }
            __syncthreads();
        }
        // r = b, so |r|^2 = |b|^2
        if (!grid_reduce<3, VW, NP>(acc, scratch, a.partials, red_id, a.bar, a.status, a.spin_limit, red, cta, ncta))
            return;
        if (threadIdx.x == 0) {
            int bad = 0;
            for (int r = 0; r < R; ++r) {
                gam[r] = red[r];
                rr[r] = red[2 * R + r];
                bb[r] = rr[r];
                const bool act = rr[r] > a.rtol2 * bb[r];
                const double dl = red[R + r];
                if (act && !(dl > 0.0 && isfinite(dl))) bad = 1;
                alpha[r] = act && dl > 0.0 ? gam[r] / dl : 0.0;
                beta[r] = 0.0;
            }
            s_flag = bad;
        }
        __syncthreads();
        if (s_flag) {
            if (cta == 0 && threadIdx.x == 0) atomicCAS(a.status, 0, QPAT_EBREAKDOWN);
            return;
        }
    }

    int it = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            int any = 0;
            for (int r = 0; r < R; ++r) any |= (rr[r] > a.rtol2 * bb[r]) ? 1 : 0;
            s_flag = any;
        }
        __syncthreads();
        if (!s_flag) break;
        if (it >= a.maxit) {
            if (cta == 0 && threadIdx.x == 0) atomicCAS(a.status, 0, QPAT_ENOCONV);
            break;
        }
        // double buffers by iteration parity (r, w: current / next; s: current / previous)
        const bool odd = it & 1;
        const T* rcur = odd ? a.r1 : a.r;
        T* rnew = odd ? a.r : a.r1;
        const T* wcur = odd ? a.w1 : a.q;
        T* wnew = odd ? a.q : a.w1;
        const T* sold = odd ? a.s0 : a.s1;
        T* scur = odd ? a.s1 : a.s0;
        T al[VW], bt[VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) {
            al[c] = T(alpha[r0 + c]);
            bt[c] = T(beta[r0 + c]);
        }
        T acc[3][VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) acc[0][c] = acc[1][c] = acc[2][c] = 0.0;
        for (int pt = cta; pt < P; pt += ncta) {
            const int nb = __ldg(m.node_ptr + pt), nt = __ldg(m.node_ptr + pt + 1) - nb;
            const int ob = __ldg(m.own_begin + pt), nown = __ldg(m.own_begin + pt + 1) - ob;
            // s = w + beta s_old, r_new = r - alpha s, u_new = D^-1 r_new on the touched nodes
            for (int i0 = threadIdx.x; i0 < nt * NP; i0 += kUnroll * blockDim.x) {
                int li[kUnroll];
                size_t e[kUnroll];
                T wv[kUnroll][VW], rv[kUnroll][VW], sv[kUnroll][VW], d[kUnroll][VW];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const int i = i0 + u * blockDim.x;
                    li[u] = (i < nt * NP ? i : i0) / NP;
                    const int g = __ldg(m.nodes + nb + li[u]);
                    e[u] = size_t(g) * R + r0;
                    vld_cg(wcur + e[u], wv[u]);
                    vld_cg(rcur + e[u], rv[u]);
                    if (it > 0) vld_cg(sold + e[u], sv[u]);
                    dinv_vec<T, VW, OP>(a.invdiag, g, r0, d[u]);
                }
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    if (u > 0 && i0 + u * int(blockDim.x) >= nt * NP) break;
                    T un[VW];
#pragma unroll
                    for (int c = 0; c < VW; ++c) {
                        sv[u][c] = wv[u][c] + (it > 0 ? bt[c] * sv[u][c] : T(0));
                        rv[u][c] -= al[c] * sv[u][c];
                        un[c] = d[u][c] * rv[u][c];
                    }
                    vst(su + li[u] * R + r0, un);
                    if (li[u] < nown) {
                        vst(scur + e[u], sv[u]);
                        vst(rnew + e[u], rv[u]);
                    }
                }
            }
            __syncthreads();
            // owned rows: w_new = A u_new; p = u + beta p; x += alpha p
            for (int i = threadIdx.x; i < nown * NP; i += blockDim.x) {
                const int li = i / NP, g = ob + li;
                const size_t e = size_t(g) * R + r0;
                T wv[VW], un[VW], rn[VW], uo[VW], pv[VW], xv[VW];
                sell_row<T, R, VW, OP>(m, a.op, su, g, r0, wv);
                vld(su + li * R + r0, un);
                vld(rnew + e, rn);
                vld(u + e, uo);
                vld(a.x + e, xv);
                if (it > 0) {
                    vld(p + e, pv);
#pragma unroll
                    for (int c = 0; c < VW; ++c) pv[c] = uo[c] + bt[c] * pv[c];
                } else {
#pragma unroll
                    for (int c = 0; c < VW; ++c) pv[c] = uo[c];
                }
#pragma unroll
                for (int c = 0; c < VW; ++c) {
                    xv[c] += al[c] * pv[c];
                    acc[0][c] += rn[c] * un[c];
                    acc[1][c] += wv[c] * un[c];
                    acc[2][c] += rn[c] * rn[c];
                }
                vst(p + e, pv);
                vst(a.x + e, xv);
                vst(u + e, un);
                vst(wnew + e, wv);
            }
            __syncthreads();
        }
        if (!grid_reduce<3, VW, NP>(acc, scratch, a.partials, red_id, a.bar, a.status, a.spin_limit, red, cta, ncta))
            return;
        if (threadIdx.x == 0) {
            int bad = 0;
            for (int r = 0; r < R; ++r) {
                const bool act = rr[r] > a.rtol2 * bb[r];
                if (!act) {
                    alpha[r] = beta[r] = 0.0;
                    continue;
                }
                rr[r] = red[2 * R + r];
                if (!(rr[r] > a.rtol2 * bb[r])) {
                    // converged now: x holds the final iterate, freeze it
                    alpha[r] = beta[r] = 0.0;
                    continue;
                }
                const double gn = red[r], dn = red[R + r];
                const double b_ = gn / gam[r];
                const double den = dn - b_ * gn / alpha[r];
                if (!(den > 0.0 && isfinite(den) && isfinite(gn))) bad = 1;
                beta[r] = b_;
                alpha[r] = den > 0.0 ? gn / den : 0.0;
                gam[r] = gn;
            }
            s_flag = bad;
        }
        __syncthreads();
        if (s_flag) {
            if (cta == 0 && threadIdx.x == 0) atomicCAS(a.status, 0, QPAT_EBREAKDOWN);
            break;
        }
        ++it;
    }
    if (cta == 0 && threadIdx.x < R) {
        a.stats[threadIdx.x] = rr[threadIdx.x];
        a.stats[R + threadIdx.x] = bb[threadIdx.x];
        if (threadIdx.x == 0) *a.iters = it;
    }
}

template <typename T, int R, int OP>
__global__ void __launch_bounds__(kThreads, min_ctas<OP>()) k_pcg1(PcgArgs<T> a) {
    pcg1_body<T, R, OP>(a, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------- bulk-copy ring variant
// Same iteration as pcg_body (assembled operators), but the operator is not
// read with per-thread loads: one thread streams it, a 32-row slice at a
// time, into a ring of S shared-memory slots with cp.async.bulk copies that
// signal an mbarrier when their bytes have landed (Hopper/Blackwell bulk-copy
// engine: no registers, no per-thread requests).  A slice is the values, the
// local column ids and the row lengths of 32 consecutive rows, which the
// sliced-ELLPACK layout keeps contiguous.  The operator does not change
// between iterations, so the copies for the next iteration's first slices are
// issued while this one finishes: they travel during phase B and both grid
// reductions.  Rows of a slice are computed by all 8 warps: lane = row,
// warp = (RHS block, stride-KS share of the row's entries); the KS partial
// sums meet in shared memory (double-buffered, one __syncthreads per slice).
constexpr int kMaxSlots = 8;
constexpr long long kMbarSpinLimit = 1LL << 22;  // try_wait polls; each may suspend up to ~1 us

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait on phase `parity` of an mbarrier; false after the spin limit
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    for (long long i = 0; i < kMbarSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// shared-memory layout of the ring kernel (byte offsets, 128-aligned)
struct RingLayout {
    int slots;          // S
    int slot_bytes;     // one slice: NV value arrays, column ids, lengths
    int xs_off, red_off, ring_off, total;
};

template <typename T, int R, int OP>
struct RingCfg {
    static constexpr int VW = vec_width<T, R, true>();
    static constexpr int NP = R / VW;
    static constexpr int KS = (kThreads / 32) / NP;  // warps sharing one row's entries
    static constexpr int NV = OP == OP_CSR2 ? 2 : 1;
    static_assert(NP <= kThreads / 32, "one warp per RHS block at least");
};

template <typename T, int R, int OP>
__host__ __device__ inline RingLayout ring_layout(int max_touched, int wmax, int slots) {
    using C = RingCfg<T, R, OP>;
    auto up = [](int b) { return (b + 127) / 128 * 128; };
    RingLayout L;
    L.slots = slots;
    L.slot_bytes = up(C::NV * wmax * 32 * int(sizeof(T)) + wmax * 32 * 2 + 32);
    L.xs_off = 0;
    L.red_off = up(int(sizeof(T)) * max_touched * R);
    // two KS x NP x 32 x VW partial-sum buffers; also the grid reduction's scratch
    int red = 2 * (kThreads / 32) * 32 * C::VW * int(sizeof(T));
    red = red > (kThreads / 32) * kMaxNS * 8 ? red : (kThreads / 32) * kMaxNS * 8;
    L.ring_off = L.red_off + up(red);
    L.total = L.ring_off + slots * L.slot_bytes;
    return L;
}

template <typename T, int R, int OP>
__device__ __forceinline__ void pcg_ring_body(const PcgArgs<T>& a, const RingLayout L, const int cta,
                                              const int ncta) {
    using C = RingCfg<T, R, OP>;
    constexpr int VW = C::VW, NP = C::NP, KS = C::KS, NV = C::NV;
    extern __shared__ __align__(128) unsigned char ring_smem[];
    T* xs = reinterpret_cast<T*>(ring_smem + L.xs_off);
    T* red_s = reinterpret_cast<T*>(ring_smem + L.red_off);
    double* scratch = reinterpret_cast<double*>(ring_smem + L.red_off);
    unsigned char* ring = ring_smem + L.ring_off;
    __shared__ uint64_t full[kMaxSlots];
    __shared__ double red[kMaxNS];
    __shared__ double bb[R], rz[R], rz_old[R], rr[R], alpha[R], beta[R];
    __shared__ double dot_s[NP][VW];
    __shared__ int s_flag;

    const MeshDev& m = a.m;
    const int P = m.P;
    const int S = L.slots;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int rpart = wq % NP, kslot = wq / NP;  // rows pass: RHS block and entry share
    const int r0row = rpart * VW;
    const int spart = threadIdx.x % NP;          // staging and vector phases
    const int r0 = spart * VW;
    const int W = m.sell_wmax;
    int red_id = 0;

    // slices of this CTA per phase (its patches' owned rows, 32 per slice)
    int nsl = 0;
    for (int pt = cta; pt < P; pt += ncta)
        nsl += (__ldg(m.own_begin + pt + 1) - __ldg(m.own_begin + pt) + 31) / 32;
    // sequence number q -> global slice id (the same order every iteration)
    auto slice_of = [&](long long q) {
        int loc = int(q % nsl);
        for (int pt = cta; pt < P; pt += ncta) {
            const int ob = __ldg(m.own_begin + pt);
            const int ns = (__ldg(m.own_begin + pt + 1) - ob + 31) / 32;
            if (loc < ns) return ob / 32 + loc;
            loc -= ns;
        }
        return 0;  // not reached
    };
    auto issue = [&](long long q) {  // one thread
        const int slot = int(q % S);
        const int sl = slice_of(q);
        const int64_t p0 = m.sell_ptr[sl];
        const int w = int(m.sell_ptr[sl + 1] - p0);
        const int64_t e0 = p0 * 32;
        unsigned char* dst = ring + size_t(slot) * L.slot_bytes;
        const unsigned bv = unsigned(w) * 32u * sizeof(T), bc = unsigned(w) * 64u;
        mbar_expect_tx(&full[slot], NV * bv + bc + 32u);
        bulk_g2s(dst, a.op.v0 + e0, bv, &full[slot]);
        if constexpr (NV == 2) bulk_g2s(dst + size_t(W) * 32 * sizeof(T), a.op.v1 + e0, bv, &full[slot]);
        bulk_g2s(dst + size_t(NV) * W * 32 * sizeof(T), m.sell_col + e0, bc, &full[slot]);
        bulk_g2s(dst + size_t(NV) * W * 32 * sizeof(T) + size_t(W) * 64, m.sell_len + size_t(sl) * 32, 32u,
                 &full[slot]);
    };
    long long cons = 0;  // next slice to consume; slices [cons, cons + S) are in flight
    // waits for every copy in flight (bounded), so that no copy outlives the CTA
    auto drain = [&]() {
        for (long long q = cons; q < cons + S; ++q) mbar_wait(&full[q % S], unsigned((q / S) & 1));
    };

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) mbar_init(&full[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (long long q = 0; q < S; ++q) issue(q);

    // ---- initial residual r = b (x0 = 0)
    {
        T acc[3][VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) acc[0][c] = acc[1][c] = acc[2][c] = 0.0;
        for (int pt = cta; pt < P; pt += ncta) {
            const int ob = __ldg(m.own_begin + pt), nown = __ldg(m.own_begin + pt + 1) - ob;
            for (int i = threadIdx.x; i < nown * NP; i += blockDim.x) {
                const int g = ob + i / NP;
                const size_t e = size_t(g) * R + r0;
                T bv[VW], d[VW], zero[VW];
                vld(a.b + e, bv);
                dinv_vec<T, VW, OP>(a.invdiag, g, r0, d);
#pragma unroll
                for (int c = 0; c < VW; ++c) {
                    zero[c] = T(0);
                    acc[0][c] += bv[c] * bv[c];
                    acc[1][c] += bv[c] * (d[c] * bv[c]);
                }
                vst(a.x + e, zero);
                vst(a.r + e, bv);
            }
        }
#pragma unroll
        for (int c = 0; c < VW; ++c) acc[2][c] = acc[0][c];
        if (!grid_reduce<3, VW, NP>(acc, scratch, a.partials, red_id, a.bar, a.status, a.spin_limit, red, cta,
                                    ncta)) {
            drain();
            return;
        }
        if (threadIdx.x < R) {
            bb[threadIdx.x] = red[threadIdx.x];
            rz[threadIdx.x] = red[R + threadIdx.x];
            rr[threadIdx.x] = red[2 * R + threadIdx.x];
            rz_old[threadIdx.x] = 1.0;
        }
        __syncthreads();
    }

    int it = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            int any = 0;
            for (int r = 0; r < R; ++r) any |= (rr[r] > a.rtol2 * bb[r]) ? 1 : 0;
            s_flag = any;
        }
        __syncthreads();
        if (!s_flag) break;
        if (it >= a.maxit) {
            if (cta == 0 && threadIdx.x == 0) atomicCAS(a.status, 0, QPAT_ENOCONV);
            break;
        }
        if (threadIdx.x < R) {
            const int r = threadIdx.x;
            const bool act = rr[r] > a.rtol2 * bb[r];
            beta[r] = (it == 0 || !act) ? 0.0 : rz[r] / rz_old[r];
        }
        __syncthreads();

        T* pc = (it & 1) ? a.p1 : a.p0;
        const T* pp = (it & 1) ? a.p0 : a.p1;
        T bt[VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) bt[c] = T(beta[r0 + c]);

        // ---- phase A: p on the touched nodes (shared), q = A p row slice by row slice
        T dotA[VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) dotA[c] = 0.0;
        bool ok = true;
        for (int pt = cta; pt < P && ok; pt += ncta) {
            const int nb = __ldg(m.node_ptr + pt), nt = __ldg(m.node_ptr + pt + 1) - nb;
            const int ob = __ldg(m.own_begin + pt), nown = __ldg(m.own_begin + pt + 1) - ob;
            for (int i0 = threadIdx.x; i0 < nt * NP; i0 += kUnroll * blockDim.x) {
                int li[kUnroll];
                T rv[kUnroll][VW], d[kUnroll][VW], po[kUnroll][VW];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const int i = i0 + u * blockDim.x;
                    li[u] = (i < nt * NP ? i : i0) / NP;
                    const int g = __ldg(m.nodes + nb + li[u]);
                    const size_t e = size_t(g) * R + r0;
                    vld_cg(a.r + e, rv[u]);
                    dinv_vec<T, VW, OP>(a.invdiag, g, r0, d[u]);
                    if (it > 0) vld_cg(pp + e, po[u]);
                }
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    T pv[VW];
#pragma unroll
                    for (int c = 0; c < VW; ++c) pv[c] = d[u][c] * rv[u][c] + (it > 0 ? bt[c] * po[u][c] : T(0));
                    if (u == 0 || i0 + u * int(blockDim.x) < nt * NP) vst(xs + li[u] * R + r0, pv);
                }
            }
            __syncthreads();
            const int ns = (nown + 31) / 32;
            for (int j = 0; j < ns; ++j, ++cons) {
                const int slot = int(cons % S);
                // a thread that gives up computes nothing (the slot is not
                // valid) and the vote below takes every thread out together
                const bool landed = mbar_wait(&full[slot], unsigned((cons / S) & 1));
                const unsigned char* sb = ring + size_t(slot) * L.slot_bytes;
                const T* vals0 = reinterpret_cast<const T*>(sb);
                const T* vals1 = reinterpret_cast<const T*>(sb + size_t(W) * 32 * sizeof(T));
                const uint16_t* cols = reinterpret_cast<const uint16_t*>(sb + size_t(NV) * W * 32 * sizeof(T));
                const uint8_t* lens = sb + size_t(NV) * W * 32 * sizeof(T) + size_t(W) * 64;
                const int len = landed ? int(lens[lane]) : 0;
                T acc[VW];
#pragma unroll
                for (int c = 0; c < VW; ++c) acc[c] = T(0);
                for (int k = kslot; k < len; k += KS) {
                    const int col = cols[k * 32 + lane];
                    T xv[VW];
                    vld(xs + col * R + r0row, xv);
                    if constexpr (NV == 1) {
                        const T v = vals0[k * 32 + lane];
#pragma unroll
                        for (int c = 0; c < VW; ++c) acc[c] += v * xv[c];
                    } else {
#pragma unroll
                        for (int c = 0; c < VW; ++c) acc[c] += (r0row + c == 0 ? vals0 : vals1)[k * 32 + lane] * xv[c];
                    }
                }
                T* rb = red_s + size_t(cons & 1) * (kThreads / 32) * 32 * VW;
                if constexpr (KS > 1) vst(rb + (wq * 32 + lane) * VW, acc);
                // the slot and this pass's partial sums are complete
                if (!__syncthreads_and(landed)) {
                    if (threadIdx.x == 0) atomicExch(a.status, QPAT_ETIMEOUT);
                    ok = false;
                    break;
                }
                if (threadIdx.x == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue(cons + S);
                }
                if (kslot == 0) {
                    if constexpr (KS > 1) {
#pragma unroll
                        for (int c = 0; c < VW; ++c) acc[c] = T(0);
                        for (int k2 = 0; k2 < KS; ++k2) {
                            T pv[VW];
                            vld(rb + ((k2 * NP + rpart) * 32 + lane) * VW, pv);
#pragma unroll
                            for (int c = 0; c < VW; ++c) acc[c] += pv[c];
                        }
                    }
                    const int li = 32 * j + lane;
                    if (li < nown) {
                        T pv[VW];
                        vld(xs + li * R + r0row, pv);
                        const size_t e = size_t(ob + li) * R + r0row;
                        vst(pc + e, pv);
                        vst(a.q + e, acc);
#pragma unroll
                        for (int c = 0; c < VW; ++c) dotA[c] += pv[c] * acc[c];
                    }
                }
            }
            __syncthreads();  // xs is restaged for the next patch
        }
        if (!ok) {
            drain();
            return;
        }
        // p.q per RHS block: warp sums, then one thread per block feeds the grid reduction
        if (kslot == 0) {
#pragma unroll
            for (int c = 0; c < VW; ++c) {
                double v = double(dotA[c]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) dot_s[rpart][c] = v;
            }
        }
        __syncthreads();
        double accA[1][VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) accA[0][c] = threadIdx.x < NP ? dot_s[threadIdx.x][c] : 0.0;
        if (!grid_reduce<1, VW, NP>(accA, scratch, a.partials, red_id, a.bar, a.status, a.spin_limit, red, cta,
                                    ncta)) {
            drain();
            return;
        }
        if (threadIdx.x == 0) {
            int bad = 0;
            for (int r = 0; r < R; ++r) {
                const bool act = rr[r] > a.rtol2 * bb[r];
                const double pq = red[r];
                if (act && !(pq > 0.0 && isfinite(pq))) bad = 1;
                alpha[r] = act && pq > 0.0 ? rz[r] / pq : 0.0;
            }
            s_flag = bad;
        }
        __syncthreads();
        if (s_flag) {
            if (cta == 0 && threadIdx.x == 0) atomicCAS(a.status, 0, QPAT_EBREAKDOWN);
            break;
        }

        // ---- phase B: x += alpha p, r -= alpha q; r.D^-1 r and r.r
        T accB[2][VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) accB[0][c] = accB[1][c] = 0.0;
        {
            T al[VW];
#pragma unroll
            for (int c = 0; c < VW; ++c) al[c] = T(alpha[r0 + c]);
            for (int pt = cta; pt < P; pt += ncta) {
                const int ob = __ldg(m.own_begin + pt), nown = __ldg(m.own_begin + pt + 1) - ob;
                for (int i0 = threadIdx.x; i0 < nown * NP; i0 += kUnroll * blockDim.x) {
                    T pv[kUnroll][VW], qv[kUnroll][VW], xv[kUnroll][VW], rv[kUnroll][VW], d[kUnroll][VW];
                    size_t e[kUnroll];
#pragma unroll
                    for (int u = 0; u < kUnroll; ++u) {
                        const int i = i0 + u * blockDim.x;
                        const int g = ob + (i < nown * NP ? i : i0) / NP;
                        e[u] = size_t(g) * R + r0;
                        vld(pc + e[u], pv[u]);
                        vld(a.q + e[u], qv[u]);
                        vld(a.x + e[u], xv[u]);
                        vld(a.r + e[u], rv[u]);
                        dinv_vec<T, VW, OP>(a.invdiag, g, r0, d[u]);
                    }
#pragma unroll
                    for (int u = 0; u < kUnroll; ++u) {
                        if (u > 0 && i0 + u * int(blockDim.x) >= nown * NP) break;
#pragma unroll
                        for (int c = 0; c < VW; ++c) {
                            xv[u][c] += al[c] * pv[u][c];
                            rv[u][c] -= al[c] * qv[u][c];
                            accB[0][c] += rv[u][c] * (d[u][c] * rv[u][c]);
                            accB[1][c] += rv[u][c] * rv[u][c];
                        }
                        vst(a.x + e[u], xv[u]);
                        vst(a.r + e[u], rv[u]);
                    }
                }
            }
        }
        if (!grid_reduce<2, VW, NP>(accB, scratch, a.partials, red_id, a.bar, a.status, a.spin_limit, red, cta,
                                    ncta)) {
            drain();
            return;
        }
        if (threadIdx.x < R) {
            const int r = threadIdx.x;
            const bool act = rr[r] > a.rtol2 * bb[r];
            if (act) {
                rz_old[r] = rz[r];
                rz[r] = red[r];
                rr[r] = red[R + r];
            }
        }
        __syncthreads();
        ++it;
    }
    drain();
    if (cta == 0 && threadIdx.x < R) {
        a.stats[threadIdx.x] = rr[threadIdx.x];
        a.stats[R + threadIdx.x] = bb[threadIdx.x];
        if (threadIdx.x == 0) *a.iters = it;
    }
}

template <typename T, int R, int OP>
__global__ void __launch_bounds__(kThreads, 4) k_pcg_ring(PcgArgs<T> a, RingLayout L) {
    pcg_ring_body<T, R, OP>(a, L, blockIdx.x, gridDim.x);
}

// Independent problems (meshes of different sizes) in one cooperative
// launch: CTAs [cta_begin[j], cta_begin[j+1]) solve problem j, and each
// problem's barriers and reductions involve only its own CTAs.
template <typename T, int R, int OP, bool kPoly = false>
__global__ void __launch_bounds__(kThreads) k_pcg_batch(const PcgArgs<T>* __restrict__ probs,
                                                        const int* __restrict__ cta_begin, int nprob) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (cta_begin[mid] <= int(blockIdx.x))
            lo = mid;
        else
            hi = mid - 1;
    }
    const int b0 = cta_begin[lo];
    const PcgArgs<T> a = probs[lo];
    pcg_body<T, R, OP, kPoly>(a, int(blockIdx.x) - b0, cta_begin[lo + 1] - b0);
}

template <int R>
cudaError_t batch_prepare_t(const std::vector<PcgBatchProblem>& probs, PcgBatchPlan& plan) {
    // the patch-local Chebyshev preconditioner when every problem asks for it
    bool poly = !probs.empty();
    for (const auto& p : probs) poly = poly && p.w.poly_deg > 0 && p.w.z && p.w.poly_hi;
    size_t smem = 0;
    for (const auto& p : probs) {
        if (p.w.poly_deg < 0 || p.w.poly_deg > kMaxPolyDegree) return cudaErrorInvalidValue;
        smem = std::max(smem, sizeof(double) * size_t(p.m.max_touched) * R);
        if (poly) smem = std::max(smem, 3 * sizeof(double) * size_t(p.m.max_own) * R);
    }
    auto kern = poly ? k_pcg_batch<double, R, OP_CSR1, true> : k_pcg_batch<double, R, OP_CSR1>;
    cudaError_t err = qpat::allow_smem((const void*)kern, size_t(smem));
    if (err != cudaSuccess) return err;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int nprob = int(probs.size());
    int resident = std::min(per_sm * nsm, kMaxGrid);
    if (resident < nprob) return cudaErrorInvalidConfiguration;
    // CTAs proportional to the work (nodes), at least one per problem and at
    // most one per patch
    double total = 0;
    for (const auto& p : probs) total += double(p.m.N);
    std::vector<int> cnt(nprob);
    int used = 0;
    for (int j = 0; j < nprob; ++j) {
        int c = int(double(resident - nprob) * double(probs[j].m.N) / total) + 1;
        c = std::min(c, probs[j].m.P);
        cnt[j] = c;
        used += c;
    }
    // hand the remaining CTAs to the problems with the most nodes per CTA
    for (int guard = 0; used < resident && guard < resident; ++guard) {
        int best = -1;
        double load = 0;
        for (int j = 0; j < nprob; ++j)
            if (cnt[j] < probs[j].m.P && double(probs[j].m.N) / cnt[j] > load) {
                load = double(probs[j].m.N) / cnt[j];
                best = j;
            }
        if (best < 0) break;
        ++cnt[best];
        ++used;
    }
    std::vector<int> begin(nprob + 1, 0);
    for (int j = 0; j < nprob; ++j) begin[j + 1] = begin[j] + cnt[j];
    std::vector<PcgArgs<double>> args(nprob);
    for (int j = 0; j < nprob; ++j) {
        const auto& p = probs[j];
        PcgArgs<double>& a = args[j];
        a.m = p.m;
        a.op = OpParams<double>{nullptr, nullptr, 0.0, 0.0, 0.0, 1, p.vals, nullptr};
        a.invdiag = p.invdiag;
        a.b = static_cast<const double*>(p.w.b);
        a.x = static_cast<double*>(p.w.x);
        a.r = static_cast<double*>(p.w.r);
        a.p0 = static_cast<double*>(p.w.p0);
        a.p1 = static_cast<double*>(p.w.p1);
        a.q = static_cast<double*>(p.w.q);
        a.partials = p.w.partials;
        a.bar = p.w.bar;
        a.status = p.w.status;
        a.iters = p.w.iters;
        a.stats = p.w.stats;
        a.rtol2 = p.rtol * p.rtol;
        a.maxit = p.maxit;
        a.spin_limit = p.w.spin_limit > 0 ? p.w.spin_limit : kDefaultSpinLimit;
        if (poly) {
            a.z = static_cast<double*>(p.w.z);
            a.poly_deg = p.w.poly_deg;
            a.poly_hi = p.w.poly_hi;
        }
    }
    if ((err = cudaMalloc(&plan.dev_args, sizeof(PcgArgs<double>) * nprob)) != cudaSuccess) return err;
    if ((err = cudaMalloc(reinterpret_cast<void**>(&plan.dev_cta_begin), sizeof(int) * (nprob + 1))) != cudaSuccess)
        return err;
    if ((err = cudaMemcpy(plan.dev_args, args.data(), sizeof(PcgArgs<double>) * nprob, cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return err;
    if ((err = cudaMemcpy(plan.dev_cta_begin, begin.data(), sizeof(int) * (nprob + 1), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return err;
    plan.R = R;
    plan.nprob = nprob;
    plan.grid = begin[nprob];
    plan.smem = smem;
    plan.poly = poly;
    plan.cta_count = cnt;
    return cudaSuccess;
}

template <int R>
cudaError_t batch_launch_t(const PcgBatchPlan& plan, cudaStream_t s) {
    auto kern = plan.poly ? k_pcg_batch<double, R, OP_CSR1, true> : k_pcg_batch<double, R, OP_CSR1>;
    const PcgArgs<double>* pa = static_cast<const PcgArgs<double>*>(plan.dev_args);
    const int* cb = plan.dev_cta_begin;
    int np = plan.nprob;
    void* args[] = {&pa, &cb, &np};
    qpat::note_launch(1);
    return cudaLaunchCooperativeKernel((void*)kern, dim3(plan.grid), dim3(kThreads), args, plan.smem, s);
}

template <typename T, int R, int OP, bool kSingle = false>
cudaError_t launch_pcg_t(const MeshDev& m, const OpParams<T>& op, const T* invdiag, const PcgWork& w,
                         double rtol, int maxit, cudaStream_t s, int* grid_used) {
    constexpr bool kCsr = OP == OP_CSR1 || OP == OP_CSR2;
    const int deg = (kCsr && !kSingle && w.z) ? w.poly_deg : 0;
    if (w.poly_deg < 0 || w.poly_deg > kMaxPolyDegree || (deg > 0 && !w.poly_hi)) return cudaErrorInvalidValue;
    size_t smem = kCsr ? sizeof(T) * size_t(m.max_touched) * R : PatchSmem<T, R>::bytes(m.max_touched, m.max_own);
    if (deg > 0) smem = std::max(smem, 3 * sizeof(T) * size_t(m.max_own) * R);
    void (*kern)(PcgArgs<T>) = nullptr;
    if constexpr (kSingle) {
        kern = k_pcg1<T, R, OP>;
    } else if constexpr (kCsr) {
        kern = deg > 0 ? k_pcg<T, R, OP, true> : k_pcg<T, R, OP>;
        if constexpr (OP == OP_CSR2 && R == 2 && std::is_same<T, double>::value)
            if (deg > 0 && !w.force_narrow) kern = k_pcg_occ3<T, R, OP, true>;
    } else {
        kern = k_pcg<T, R, OP>;
    }
    cudaError_t err = qpat::allow_smem((const void*)kern, size_t(smem));
    if (err != cudaSuccess) return err;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int nthreads = kThreads;
    if constexpr (kCsr && !kSingle && R >= 4) {
        if (per_sm == 1 && !w.force_narrow) {
            // one CTA per SM: the wide variant, if it keeps one resident CTA
            void (*wk)(PcgArgs<T>) = deg > 0 ? k_pcg_wide<T, R, OP, true> : k_pcg_wide<T, R, OP>;
            int pw = 0;
            if (qpat::allow_smem((const void*)wk, size_t(smem)) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pw, wk, kWideThreads, smem) == cudaSuccess &&
                pw >= 1) {
                kern = wk;
                nthreads = kWideThreads;
                per_sm = pw;
            }
            (void)cudaGetLastError();
        }
    }
    int maxres = per_sm * nsm;
    if (maxres > kMaxGrid) maxres = kMaxGrid;
    // equal patch counts per CTA: k = ceil(P / resident), grid = ceil(P / k)
    const int k = (m.P + maxres - 1) / maxres;
    const int grid = (m.P + k - 1) / k;
    if (grid_used) *grid_used = grid;
    PcgArgs<T> a;
    a.m = m;
    a.op = op;
    a.invdiag = invdiag;
    a.b = static_cast<const T*>(w.b);
    a.x = static_cast<T*>(w.x);
    a.r = static_cast<T*>(w.r);
    a.p0 = static_cast<T*>(w.p0);
    a.p1 = static_cast<T*>(w.p1);
    a.q = static_cast<T*>(w.q);
    a.partials = w.partials;
    a.bar = w.bar;
    a.status = w.status;
    a.iters = w.iters;
    a.stats = w.stats;
    a.rtol2 = rtol * rtol;
    a.maxit = maxit;
    a.spin_limit = w.spin_limit > 0 ? w.spin_limit : kDefaultSpinLimit;
    a.z = static_cast<T*>(w.z);
    a.resume_gamma = w.resume_gamma;
    a.rz_state = w.rz_state;
    a.pbuf = w.pbuf;
    a.r1 = static_cast<T*>(w.r1);
    a.s0 = static_cast<T*>(w.s0);
    a.s1 = static_cast<T*>(w.s1);
    a.w1 = static_cast<T*>(w.w1);
    a.poly_deg = deg;
    a.poly_hi = w.poly_hi;
    if (kSingle && !(a.r1 && a.s0 && a.s1 && a.w1)) return cudaErrorInvalidValue;
    err = cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), s);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(w.status, 0, sizeof(int), s);
    if (err != cudaSuccess) return err;
    void* args[] = {&a};
    qpat::note_launch(1);
    return cudaLaunchCooperativeKernel((void*)kern, dim3(grid), dim3(nthreads), args, smem, s);
}

// Ring variant: picks the most slots (<= kMaxSlots) that keep min(4, P / SMs)
// CTAs resident per SM; cudaErrorNotSupported when not even 2 slots fit.
template <typename T, int R, int OP>
cudaError_t launch_pcg_ring_t(const MeshDev& m, const OpParams<T>& op, const T* invdiag, const PcgWork& w,
                              double rtol, int maxit, cudaStream_t s, int* grid_used) {
    auto kern = k_pcg_ring<T, R, OP>;
    int dev = 0, nsm = 0, smem_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaError_t err = cudaFuncGetAttributes(&fa, kern);
    if (err != cudaSuccess) return err;
    const int dyn_max = smem_optin - int(fa.sharedSizeBytes);  // static + dynamic <= opt-in limit
    err = qpat::allow_smem((const void*)kern, size_t(dyn_max));
    if (err != cudaSuccess) return err;
    const int want = std::max(1, std::min(4, (m.P + nsm - 1) / nsm));
    RingLayout L{};
    int per_sm = 0;
    bool found = false;
    for (int S = kMaxSlots; S >= 2 && !found; --S) {
        L = ring_layout<T, R, OP>(m.max_touched, m.sell_wmax, S);
        if (L.total > dyn_max) continue;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, L.total);
        if (err != cudaSuccess) return err;
        found = per_sm >= want;
    }
    if (!found) return cudaErrorNotSupported;
    int maxres = std::min(per_sm * nsm, kMaxGrid);
    const int k = (m.P + maxres - 1) / maxres;
    const int grid = (m.P + k - 1) / k;
    if (grid_used) *grid_used = grid;
    PcgArgs<T> a{};
    a.m = m;
    a.op = op;
    a.invdiag = invdiag;
    a.b = static_cast<const T*>(w.b);
    a.x = static_cast<T*>(w.x);
    a.r = static_cast<T*>(w.r);
    a.p0 = static_cast<T*>(w.p0);
    a.p1 = static_cast<T*>(w.p1);
    a.q = static_cast<T*>(w.q);
    a.partials = w.partials;
    a.bar = w.bar;
    a.status = w.status;
    a.iters = w.iters;
    a.stats = w.stats;
    a.rtol2 = rtol * rtol;
    a.maxit = maxit;
    a.spin_limit = w.spin_limit > 0 ? w.spin_limit : kDefaultSpinLimit;
    err = cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), s);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(w.status, 0, sizeof(int), s);
    if (err != cudaSuccess) return err;
    void* args[] = {&a, &L};
    qpat::note_launch(1);
    return cudaLaunchCooperativeKernel((void*)kern, dim3(grid), dim3(kThreads), args, size_t(L.total), s);
}

}  // namespace

int pcg_max_grid() { return kMaxGrid; }

template <typename T>
cudaError_t launch_pcg_ring(const MeshDev& m, int OP, int R, const OpParams<T>& op, const T* invdiag,
                            const PcgWork& w, double rtol, int maxit, cudaStream_t s, int* grid_used) {
    if (OP == OP_CSR2) {
        if (R != 2) return cudaErrorInvalidValue;
        return launch_pcg_ring_t<T, 2, OP_CSR2>(m, op, invdiag, w, rtol, maxit, s, grid_used);
    }
    if (OP != OP_CSR1) return cudaErrorInvalidValue;
    switch (R) {
        case 1: return launch_pcg_ring_t<T, 1, OP_CSR1>(m, op, invdiag, w, rtol, maxit, s, grid_used);
        case 2: return launch_pcg_ring_t<T, 2, OP_CSR1>(m, op, invdiag, w, rtol, maxit, s, grid_used);
        case 4: return launch_pcg_ring_t<T, 4, OP_CSR1>(m, op, invdiag, w, rtol, maxit, s, grid_used);
        case 8: return launch_pcg_ring_t<T, 8, OP_CSR1>(m, op, invdiag, w, rtol, maxit, s, grid_used);
        case 16: return launch_pcg_ring_t<T, 16, OP_CSR1>(m, op, invdiag, w, rtol, maxit, s, grid_used);
        default: return cudaErrorInvalidValue;
    }
}
template cudaError_t launch_pcg_ring<double>(const MeshDev&, int, int, const OpParams<double>&, const double*,
                                             const PcgWork&, double, int, cudaStream_t, int*);
template cudaError_t launch_pcg_ring<float>(const MeshDev&, int, int, const OpParams<float>&, const float*,
                                            const PcgWork&, double, int, cudaStream_t, int*);

cudaError_t pcg_batch_prepare(int R, const std::vector<PcgBatchProblem>& probs, PcgBatchPlan& plan) {
    switch (R) {
        case 1: return batch_prepare_t<1>(probs, plan);
        case 2: return batch_prepare_t<2>(probs, plan);
        case 4: return batch_prepare_t<4>(probs, plan);
        case 8: return batch_prepare_t<8>(probs, plan);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t pcg_batch_launch(const PcgBatchPlan& plan, cudaStream_t s) {
    switch (plan.R) {
        case 1: return batch_launch_t<1>(plan, s);
        case 2: return batch_launch_t<2>(plan, s);
        case 4: return batch_launch_t<4>(plan, s);
        case 8: return batch_launch_t<8>(plan, s);
        default: return cudaErrorInvalidValue;
    }
}

void pcg_batch_release(PcgBatchPlan& plan) {
    if (plan.dev_args) cudaFree(plan.dev_args);
    if (plan.dev_cta_begin) cudaFree(plan.dev_cta_begin);
    plan.dev_args = nullptr;
    plan.dev_cta_begin = nullptr;
}

size_t pcg_partials_doubles() { return size_t(2) * kMaxGrid * kMaxNS + 2 * kMaxNS; }

template <typename T>
cudaError_t launch_pcg(const MeshDev& m, int OP, int R, const OpParams<T>& op, const T* invdiag,
                       const PcgWork& w, double rtol, int maxit, cudaStream_t s, int* grid_used) {
    if (OP == OP_PRIOR) {
        if (R != 2) return cudaErrorInvalidValue;
        return launch_pcg_t<T, 2, OP_PRIOR>(m, op, invdiag, w, rtol, maxit, s, grid_used);
    }
    if (OP == OP_CSR2) {
        if (R != 2) return cudaErrorInvalidValue;
        return launch_pcg_t<T, 2, OP_CSR2>(m, op, invdiag, w, rtol, maxit, s, grid_used);
    }
    if (OP == OP_CSR1) {
        switch (R) {
            case 1: return launch_pcg_t<T, 1, OP_CSR1>(m, op, invdiag, w, rtol, maxit, s, grid_used);
            case 2: return launch_pcg_t<T, 2, OP_CSR1>(m, op, invdiag, w, rtol, maxit, s, grid_used);
            case 4: return launch_pcg_t<T, 4, OP_CSR1>(m, op, invdiag, w, rtol, maxit, s, grid_used);
            case 8: return launch_pcg_t<T, 8, OP_CSR1>(m, op, invdiag, w, rtol, maxit, s, grid_used);
            case 16: return launch_pcg_t<T, 16, OP_CSR1>(m, op, invdiag, w, rtol, maxit, s, grid_used);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (R) {
        case 1: return launch_pcg_t<T, 1, OP_K>(m, op, invdiag, w, rtol, maxit, s, grid_used);
        case 2: return launch_pcg_t<T, 2, OP_K>(m, op, invdiag, w, rtol, maxit, s, grid_used);
        case 4: return launch_pcg_t<T, 4, OP_K>(m, op, invdiag, w, rtol, maxit, s, grid_used);
        case 8: return launch_pcg_t<T, 8, OP_K>(m, op, invdiag, w, rtol, maxit, s, grid_used);
        case 16: return launch_pcg_t<T, 16, OP_K>(m, op, invdiag, w, rtol, maxit, s, grid_used);
        default: return cudaErrorInvalidValue;
    }
}

// Whether the two-reduction PCG kernel that launch_pcg picks for (OP, R,
// polynomial degree) fits the device's per-block shared memory: the staged
// direction on the touched nodes, the preconditioner's three owned-row
// vectors, or the matrix-free operator's patch geometry, plus the kernel's
// static shared arrays.
template <typename T, int R, int OP>
bool pcg_fits_t(const MeshDev& m, int deg) {
    constexpr bool kCsr = OP == OP_CSR1 || OP == OP_CSR2;
    if (!kCsr) deg = 0;
    size_t smem = kCsr ? sizeof(T) * size_t(m.max_touched) * R : PatchSmem<T, R>::bytes(m.max_touched, m.max_own);
    if (deg > 0) smem = std::max(smem, 3 * sizeof(T) * size_t(m.max_own) * R);
    void (*kern)(PcgArgs<T>) = nullptr;
    if constexpr (kCsr) {
        kern = deg > 0 ? k_pcg<T, R, OP, true> : k_pcg<T, R, OP>;
    } else {
        kern = k_pcg<T, R, OP>;
    }
    cudaFuncAttributes fa{};
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return true;  // let the launch report the error
    }
    return smem + fa.sharedSizeBytes <= size_t(optin);
}

template <typename T>
bool pcg_fits(const MeshDev& m, int OP, int R, int deg) {
    if (OP == OP_PRIOR) return R != 2 || pcg_fits_t<T, 2, OP_PRIOR>(m, deg);
    if (OP == OP_CSR2) return R != 2 || pcg_fits_t<T, 2, OP_CSR2>(m, deg);
    if (OP == OP_CSR1) {
        switch (R) {
            case 1: return pcg_fits_t<T, 1, OP_CSR1>(m, deg);
            case 2: return pcg_fits_t<T, 2, OP_CSR1>(m, deg);
            case 4: return pcg_fits_t<T, 4, OP_CSR1>(m, deg);
            case 8: return pcg_fits_t<T, 8, OP_CSR1>(m, deg);
            case 16: return pcg_fits_t<T, 16, OP_CSR1>(m, deg);
            default: return true;
        }
    }
    switch (R) {
        case 1: return pcg_fits_t<T, 1, OP_K>(m, deg);
        case 2: return pcg_fits_t<T, 2, OP_K>(m, deg);
        case 4: return pcg_fits_t<T, 4, OP_K>(m, deg);
        case 8: return pcg_fits_t<T, 8, OP_K>(m, deg);
        case 16: return pcg_fits_t<T, 16, OP_K>(m, deg);
        default: return true;
    }
}
template bool pcg_fits<double>(const MeshDev&, int, int, int);
template bool pcg_fits<float>(const MeshDev&, int, int, int);

template <typename T>
cudaError_t launch_pcg1(const MeshDev& m, int OP, int R, const OpParams<T>& op, const T* invdiag,
                        const PcgWork& w, double rtol, int maxit, cudaStream_t s, int* grid_used) {
    if (OP == OP_CSR2) {
        if (R != 2) return cudaErrorInvalidValue;
        return launch_pcg_t<T, 2, OP_CSR2, true>(m, op, invdiag, w, rtol, maxit, s, grid_used);
    }
    if (OP != OP_CSR1) return cudaErrorInvalidValue;
    switch (R) {
        case 1: return launch_pcg_t<T, 1, OP_CSR1, true>(m, op, invdiag, w, rtol, maxit, s, grid_used);
        case 2: return launch_pcg_t<T, 2, OP_CSR1, true>(m, op, invdiag, w, rtol, maxit, s, grid_used);
        case 4: return launch_pcg_t<T, 4, OP_CSR1, true>(m, op, invdiag, w, rtol, maxit, s, grid_used);
        case 8: return launch_pcg_t<T, 8, OP_CSR1, true>(m, op, invdiag, w, rtol, maxit, s, grid_used);
        case 16: return launch_pcg_t<T, 16, OP_CSR1, true>(m, op, invdiag, w, rtol, maxit, s, grid_used);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_pcg1<double>(const MeshDev&, int, int, const OpParams<double>&, const double*,
                                         const PcgWork&, double, int, cudaStream_t, int*);
template cudaError_t launch_pcg1<float>(const MeshDev&, int, int, const OpParams<float>&, const float*,
                                        const PcgWork&, double, int, cudaStream_t, int*);
template cudaError_t launch_pcg<double>(const MeshDev&, int, int, const OpParams<double>&, const double*,
                                        const PcgWork&, double, int, cudaStream_t, int*);
template cudaError_t launch_pcg<float>(const MeshDev&, int, int, const OpParams<float>&, const float*,
                                       const PcgWork&, double, int, cudaStream_t, int*);

}  // namespace qpat
