// Persistent fused Jacobi-preconditioned conjugate gradients.
//
// The paper solves with K (Appendix) and with M_delta (Sec. 4, one solve per
// LSQR round) but does not name a solver; both are symmetric positive
// definite, so this library uses preconditioned conjugate gradients.  One
// cooperative launch runs the whole iteration: every CTA owns a fixed set of
// node patches and, per iteration,
//   phase A: forms p = D^-1 r + beta p_old on its touched nodes in shared
//            memory (the z = D^-1 r vector is never stored), writes p on its
//            owned nodes, applies the operator and keeps q = A p on its
//            owned nodes, accumulating p.q;
//   phase B: x += alpha p, r -= alpha q on its owned nodes, accumulating
//            r.D^-1 r and r.r.
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
    T* r1;  // single-reduction variant
    T* s0;
    T* s1;
    T* w1;
};

constexpr int kMaxGrid = 152 * 8;
constexpr int kMaxNS = 48;  // largest reduction: 3 quantities x 16 RHS

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
// entry).  Entries past the row length are not loaded.
constexpr int kChunk = 8;
constexpr int kUnroll = 2;  // touched nodes a thread stages at once
template <typename T, int R, int VW, int OP>
__device__ __forceinline__ void sell_row(const MeshDev& m, const OpParams<T>& op, const T* xs, int g, int r0,
                                         T (&acc)[VW]) {
    constexpr int NL = OP == OP_CSR2 ? VW : 1;  // distinct value sets this thread reads
    const int64_t base = m.sell_ptr[g >> 5] * 32 + (g & 31);
    const int len = m.sell_len[g];
    const T* vp[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) vp[q] = (OP == OP_CSR2 && r0 + q == 1) ? op.v1 : op.v0;
#pragma unroll
    for (int c = 0; c < VW; ++c) acc[c] = T(0);
    for (int k0 = 0; k0 < len; k0 += kChunk) {
        int col[kChunk];
        T v[kChunk][NL];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            const int64_t idx = base + int64_t(k0 + j) * 32;
            const bool ok = k0 + j < len;
            col[j] = ok ? int(__ldg(m.sell_col + idx)) : 0;
#pragma unroll
            for (int q = 0; q < NL; ++q) v[j][q] = ok ? __ldg(vp[q] + idx) : T(0);
        }
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
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
template <int NQ, int VW, int NP>
__device__ __forceinline__ bool grid_reduce(double (&acc)[NQ][VW], double* scratch, double* partials, int& red_id,
                                            unsigned* bar, int* status, long long limit, double* out, int cta,
                                            int ncta) {
    constexpr int R = VW * NP, NS = NQ * R;
    __shared__ int s_last;
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int c = 0; c < VW; ++c)
#pragma unroll
            for (int o = 16; o >= NP; o >>= 1) acc[q][c] += __shfl_down_sync(0xffffffffu, acc[q][c], o);
    if (lane < NP)
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int c = 0; c < VW; ++c) scratch[warp * NS + q * R + lane * VW + c] = acc[q][c];
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

// ---------------------------------------------------------------- the solver
template <typename T, int R, int OP>
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
    __shared__ double scratch[(kThreads / 32) * kMaxNS];
    __shared__ double red[kMaxNS];
    __shared__ double bb[R], rz[R], rz_old[R], rr[R], alpha[R], beta[R];
    __shared__ int s_flag;

    const MeshDev& m = a.m;
    const int P = m.P;
    const int part = threadIdx.x % NP;  // this thread's RHS block [part*VW, part*VW + VW)
    const int r0 = part * VW;
    int red_id = 0;

    // ---- initial residual r = b (x0 = 0)
    {
        double acc[3][VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) acc[0][c] = acc[1][c] = acc[2][c] = 0.0;
        for (int p = cta; p < P; p += ncta) {
            const int ob = __ldg(m.own_begin + p), nown = __ldg(m.own_begin + p + 1) - ob;
            for (int i = threadIdx.x; i < nown * NP; i += blockDim.x) {
                const int g = ob + i / NP;
                const size_t e = size_t(g) * R + r0;
                T bv[VW], d[VW], zero[VW];
                vld(a.b + e, bv);
                dinv_vec<T, VW, OP>(a.invdiag, g, r0, d);
#pragma unroll
                for (int c = 0; c < VW; ++c) {
                    zero[c] = T(0);
                    acc[0][c] += double(bv[c]) * double(bv[c]);
                    acc[1][c] += double(bv[c]) * double(d[c] * bv[c]);
                }
                vst(a.x + e, zero);
                vst(a.r + e, bv);
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
            rz_old[threadIdx.x] = 1.0;
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

        // ---- phase A: p = D^-1 r + beta p_old on touched nodes, q = A p on owned nodes
        double accA[1][VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) accA[0][c] = 0.0;
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
                    vld_cg(a.r + e, rv[u]);
                    dinv_vec<T, VW, OP>(a.invdiag, g, r0, d[u]);
                    if (it > 0) vld_cg(pp + e, po[u]);
                }
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    T pv[VW];
#pragma unroll
                    for (int c = 0; c < VW; ++c) pv[c] = d[u][c] * rv[u][c] + (it > 0 ? bt[c] * po[u][c] : T(0));
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
                    for (int c = 0; c < VW; ++c) accA[0][c] += double(pv[c]) * double(acc[c]);
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
                    accA[0][0] += double(pv) * double(qv);
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
        double accB[2][VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) accB[0][c] = accB[1][c] = 0.0;
        {
            T al[VW];
#pragma unroll
            for (int c = 0; c < VW; ++c) al[c] = T(alpha[r0 + c]);
            for (int p = cta; p < P; p += ncta) {
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
#pragma unroll
                    for (int c = 0; c < VW; ++c) {
                        xv[c] += al[c] * pv[c];
                        rv[c] -= al[c] * qv[c];
                        accB[0][c] += double(rv[c]) * double(d[c] * rv[c]);
                        accB[1][c] += double(rv[c]) * double(rv[c]);
                    }
                    vst(a.x + e, xv);
                    vst(a.r + e, rv);
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
        if (threadIdx.x == 0) *a.iters = it;
    }
}

// single-reduction kernel on assembled operators: at least 4 resident CTAs
// per SM (a 64-register cap; uncapped it needs ~100 and halves the grid)
template <int OP>
constexpr int min_ctas() {
    return (OP == OP_CSR1 || OP == OP_CSR2) ? 4 : 1;
}

template <typename T, int R, int OP>
__global__ void __launch_bounds__(kThreads) k_pcg(PcgArgs<T> a) {
    pcg_body<T, R, OP>(a, blockIdx.x, gridDim.x);
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
        double acc[3][VW];
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
                    acc[0][c] += double(bv[c]) * double(uv[c]);
                    acc[1][c] += double(wv[c]) * double(uv[c]);
                    acc[2][c] += double(bv[c]) * double(bv[c]);
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
        double acc[3][VW];
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
                    acc[0][c] += double(rn[c]) * double(un[c]);
                    acc[1][c] += double(wv[c]) * double(un[c]);
                    acc[2][c] += double(rn[c]) * double(rn[c]);
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

// Independent problems (meshes of different sizes) in one cooperative
// launch: CTAs [cta_begin[j], cta_begin[j+1]) solve problem j, and each
// problem's barriers and reductions involve only its own CTAs.
template <typename T, int R, int OP>
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
    pcg_body<T, R, OP>(a, int(blockIdx.x) - b0, cta_begin[lo + 1] - b0);
}

template <int R>
cudaError_t batch_prepare_t(const std::vector<PcgBatchProblem>& probs, PcgBatchPlan& plan) {
    size_t smem = 0;
    for (const auto& p : probs) smem = std::max(smem, sizeof(double) * size_t(p.m.max_touched) * R);
    auto kern = k_pcg_batch<double, R, OP_CSR1>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
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
        a.spin_limit = 40000000LL;
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
    plan.cta_count = cnt;
    return cudaSuccess;
}

template <int R>
cudaError_t batch_launch_t(const PcgBatchPlan& plan, cudaStream_t s) {
    auto kern = k_pcg_batch<double, R, OP_CSR1>;
    const PcgArgs<double>* pa = static_cast<const PcgArgs<double>*>(plan.dev_args);
    const int* cb = plan.dev_cta_begin;
    int np = plan.nprob;
    void* args[] = {&pa, &cb, &np};
    return cudaLaunchCooperativeKernel((void*)kern, dim3(plan.grid), dim3(kThreads), args, plan.smem, s);
}

template <typename T, int R, int OP, bool kSingle = false>
cudaError_t launch_pcg_t(const MeshDev& m, const OpParams<T>& op, const T* invdiag, const PcgWork& w,
                         double rtol, int maxit, cudaStream_t s, int* grid_used) {
    const size_t smem = (OP == OP_CSR1 || OP == OP_CSR2) ? sizeof(T) * size_t(m.max_touched) * R
                                                         : PatchSmem<T, R>::bytes(m.max_touched, m.max_own);
    void (*kern)(PcgArgs<T>) = nullptr;
    if constexpr (kSingle)
        kern = k_pcg1<T, R, OP>;
    else
        kern = k_pcg<T, R, OP>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (err != cudaSuccess) return err;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
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
    a.spin_limit = 40000000LL;  // about 2 s of __nanosleep(32) spins
    a.r1 = static_cast<T*>(w.r1);
    a.s0 = static_cast<T*>(w.s0);
    a.s1 = static_cast<T*>(w.s1);
    a.w1 = static_cast<T*>(w.w1);
    if (kSingle && !(a.r1 && a.s0 && a.s1 && a.w1)) return cudaErrorInvalidValue;
    err = cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), s);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(w.status, 0, sizeof(int), s);
    if (err != cudaSuccess) return err;
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel((void*)kern, dim3(grid), dim3(kThreads), args, smem, s);
}

}  // namespace

int pcg_max_grid() { return kMaxGrid; }

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
