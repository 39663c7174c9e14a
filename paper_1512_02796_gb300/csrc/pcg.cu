// Persistent fused Jacobi-preconditioned conjugate gradients.
//
// The paper solves with K (Appendix) and with M_delta (Sec. 4, one solve per
// LSQR round) but does not name a solver; both are symmetric positive
// definite, so this library uses preconditioned conjugate gradients.  One
// cooperative launch runs the whole iteration: every CTA owns a fixed set of
// node patches and, per iteration,
//   phase A: forms p = D^-1 r + beta p_old on its touched nodes in shared
//            memory (the z = D^-1 r vector is never stored), writes p on its
//            owned nodes, applies the matrix-free element operator and keeps
//            q = A p on its owned nodes, accumulating p.q;
//   phase B: x += alpha p, r -= alpha q on its owned nodes, accumulating
//            r.D^-1 r and r.r.
// Each phase ends with a grid-wide deterministic reduction (per-CTA
// partials, summed in the same order by every CTA, so every CTA takes the
// same decisions) behind a bounded grid barrier.  R right-hand sides share
// one launch with their own alpha and beta (block form of the stacked
// illuminations of Sec. 4).  Scalars are accumulated in FP64 for either T.
#include <cuda/atomic>

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
};

constexpr int kMaxGrid = 152 * 8;

// Bounded grid barrier: arrive on a counter, the last arrival bumps the
// generation; the others spin (with a limit) until it changes.  On timeout
// the CTA records QPAT_ETIMEOUT and every CTA leaves at its next check.
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* status, long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(bar[0]);
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> gen(bar[1]);
        const unsigned g = gen.load(cuda::memory_order_acquire);
        __threadfence();
        const unsigned old = cnt.fetch_add(1u, cuda::memory_order_acq_rel);
        int ok = 1;
        if (old == gridDim.x - 1) {
            cnt.store(0u, cuda::memory_order_relaxed);
            gen.fetch_add(1u, cuda::memory_order_release);
        } else {
            long long spins = 0;
            while (gen.load(cuda::memory_order_acquire) == g) {
                if (++spins > limit) {
                    atomicExch(status, QPAT_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        cuda::atomic_ref<int, cuda::thread_scope_device> st(*status);
        if (st.load(cuda::memory_order_relaxed) == QPAT_ETIMEOUT) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Grid-wide sum of NQ*R values.  acc[q] belongs to RHS (threadIdx.x % R).
// Result in out[q * R + r] (shared memory) in every CTA.
template <int R, int NQ>
__device__ __forceinline__ bool grid_sum(double (&acc)[NQ], double* scratch, double* partials, int& red_id,
                                         unsigned* bar, int* status, long long limit, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int o = 16; o >= R; o >>= 1) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], o);
    if (lane < R)
#pragma unroll
        for (int q = 0; q < NQ; ++q) scratch[(warp * NQ + q) * R + lane] = acc[q];
    __syncthreads();
    // two buffers of fixed stride (the largest reduction, 3 x 16 values):
    // a slow CTA still reading reduction k never sees reduction k+1's writes
    double* part = partials + size_t(red_id & 1) * kMaxGrid * 48;
    if (threadIdx.x < NQ * R) {
        const int q = threadIdx.x / R, r = threadIdx.x % R;
        double a = 0.0;
        for (int w = 0; w < nw; ++w) a += scratch[(w * NQ + q) * R + r];
        part[size_t(blockIdx.x) * NQ * R + threadIdx.x] = a;
    }
    ++red_id;
    if (!grid_sync(bar, status, limit)) return false;
    // every CTA sums the partials in the same order
    for (int s = warp; s < NQ * R; s += nw) {
        double a = 0.0;
        for (int j = lane; j < gridDim.x; j += 32) a += __ldcg(part + size_t(j) * NQ * R + s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) out[s] = a;
    }
    __syncthreads();
    return true;
}

// Grid-wide sum of NS values held (all of them) by every thread.
template <int NS>
__device__ __forceinline__ bool grid_sum_full(double (&acc)[NS], double* scratch, double* partials, int& red_id,
                                              unsigned* bar, int* status, long long limit, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NS; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NS; ++q) scratch[warp * NS + q] = acc[q];
    __syncthreads();
    double* part = partials + size_t(red_id & 1) * kMaxGrid * 48;
    if (threadIdx.x < NS) {
        double a = 0.0;
        for (int w = 0; w < nw; ++w) a += scratch[w * NS + threadIdx.x];
        part[size_t(blockIdx.x) * NS + threadIdx.x] = a;
    }
    ++red_id;
    if (!grid_sync(bar, status, limit)) return false;
    for (int s = warp; s < NS; s += nw) {
        double a = 0.0;
        for (int j = lane; j < gridDim.x; j += 32) a += __ldcg(part + size_t(j) * NS + s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) out[s] = a;
    }
    __syncthreads();
    return true;
}

template <typename T, int R, int OP>
__device__ __forceinline__ T dinv(const T* invdiag, int g, int r) {
    return (OP == OP_PRIOR || OP == OP_CSR2) ? __ldg(invdiag + 2 * g + r) : __ldg(invdiag + g);
}

template <typename T, int R, int OP>
__global__ void __launch_bounds__(kThreads) k_pcg(PcgArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool kCsr = (OP == OP_CSR1 || OP == OP_CSR2);
    PatchSmem<T, R> s;
    if constexpr (kCsr) {
        s.xin = reinterpret_cast<T*>(smem_raw);  // assembled operators stage p only
    } else {
        s.carve(reinterpret_cast<T*>(smem_raw), a.m.max_touched, a.m.max_own);
    }
    __shared__ double scratch[(kThreads / 32) * 3 * 16];
    __shared__ double red[3 * R];
    __shared__ double bb[R], rz[R], rz_old[R], rr[R], alpha[R], beta[R];
    __shared__ int s_flag;

    const MeshDev& m = a.m;
    const int P = m.P;
    const int myr = threadIdx.x % R;
    int red_id = 0;

    // ---- initial residual r = b (x0 = 0)
    {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int p = blockIdx.x; p < P; p += gridDim.x) {
            const int ob = __ldg(m.own_begin + p), oe = __ldg(m.own_begin + p + 1);
            for (int i = threadIdx.x; i < (oe - ob) * R; i += blockDim.x) {
                const size_t e = size_t(ob) * R + i;
                const T bv = a.b[e];
                a.x[e] = T(0);
                a.r[e] = bv;
                const T z = dinv<T, R, OP>(a.invdiag, ob + i / R, myr) * bv;
                acc[0] += double(bv) * double(bv);
                acc[1] += double(bv) * double(z);
            }
        }
        acc[2] = acc[0];
        if (!grid_sum<R, 3>(acc, scratch, a.partials, red_id, a.bar, a.status, a.spin_limit, red)) return;
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
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(a.status, 0, QPAT_ENOCONV);
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

        // ---- phase A: p = D^-1 r + beta p_old on touched nodes, q = A p on owned nodes
        double accA[1] = {0.0};
        double accF[R];
#pragma unroll
        for (int r = 0; r < R; ++r) accF[r] = 0.0;
        for (int p = blockIdx.x; p < P; p += gridDim.x) {
            const int nb = __ldg(m.node_ptr + p), nt = __ldg(m.node_ptr + p + 1) - nb;
            const int ob = __ldg(m.own_begin + p), nown = __ldg(m.own_begin + p + 1) - ob;
            if constexpr (kCsr) {
                for (int i = threadIdx.x; i < nt * R; i += blockDim.x) {
                    const int g = __ldg(m.nodes + nb + i / R);
                    const size_t e = size_t(g) * R + myr;
                    T pv = dinv<T, R, OP>(a.invdiag, g, myr) * __ldcg(a.r + e);
                    const T bt = T(beta[myr]);
                    if (bt != T(0)) pv += bt * __ldcg(pp + e);
                    s.xin[i] = pv;
                }
                __syncthreads();
                csr_rows<T, R, (OP == OP_CSR2 ? 2 : 1)>(m, ob, nown, a.op.v0, a.op.v1, s.xin,
                                                       [&](int i, int r, T qv) {
                                                           const size_t e = size_t(ob + i) * R + r;
                                                           const T pv = s.xin[i * R + r];
                                                           pc[e] = pv;
                                                           a.q[e] = qv;
                                                           accF[r] += double(pv) * double(qv);
                                                       });
                __syncthreads();
                continue;
            }
            stage_static<T, R>(m, nb, nt, s, a.op);
            for (int i = threadIdx.x; i < nt * R; i += blockDim.x) {
                const int li = i / R;
                const int g = __ldg(m.nodes + nb + li);
                const size_t e = size_t(g) * R + myr;
                T pv = dinv<T, R, OP>(a.invdiag, g, myr) * __ldcg(a.r + e);
                const T bt = T(beta[myr]);
                if (bt != T(0)) pv += bt * __ldcg(pp + e);
                s.xin[i] = pv;
            }
            for (int i = threadIdx.x; i < nown * R; i += blockDim.x) s.yout[i] = T(0);
            __syncthreads();
            if constexpr (!kCsr) {
                patch_elements<T, R, OP>(m, p, nown, s, a.op);
                __syncthreads();
                for (int i = threadIdx.x; i < nown * R; i += blockDim.x) {
                    const size_t e = size_t(ob) * R + i;
                    const T pv = s.xin[i];
                    T qv = s.yout[i];
                    if (OP == OP_PRIOR) qv += a.op.delta * pv;
                    pc[e] = pv;
                    a.q[e] = qv;
                    accA[0] += double(pv) * double(qv);
                }
                __syncthreads();
            }
        }
        if constexpr (kCsr) {
            if (!grid_sum_full<R>(accF, scratch, a.partials, red_id, a.bar, a.status, a.spin_limit, red)) return;
        } else {
            if (!grid_sum<R, 1>(accA, scratch, a.partials, red_id, a.bar, a.status, a.spin_limit, red)) return;
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
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(a.status, 0, QPAT_EBREAKDOWN);
            break;
        }

        // ---- phase B: x += alpha p, r -= alpha q; r.D^-1 r and r.r
        double accB[2] = {0.0, 0.0};
        {
            const T al = T(alpha[myr]);
            for (int p = blockIdx.x; p < P; p += gridDim.x) {
                const int ob = __ldg(m.own_begin + p), oe = __ldg(m.own_begin + p + 1);
                for (int i = threadIdx.x; i < (oe - ob) * R; i += blockDim.x) {
                    const size_t e = size_t(ob) * R + i;
                    const T pv = pc[e], qv = a.q[e];
                    a.x[e] += al * pv;
                    const T rv = a.r[e] - al * qv;
                    a.r[e] = rv;
                    const T z = dinv<T, R, OP>(a.invdiag, ob + i / R, myr) * rv;
                    accB[0] += double(rv) * double(z);
                    accB[1] += double(rv) * double(rv);
                }
            }
        }
        if (!grid_sum<R, 2>(accB, scratch, a.partials, red_id, a.bar, a.status, a.spin_limit, red)) return;
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
    if (blockIdx.x == 0 && threadIdx.x < R) {
        a.stats[threadIdx.x] = rr[threadIdx.x];
        a.stats[R + threadIdx.x] = bb[threadIdx.x];
        if (threadIdx.x == 0) *a.iters = it;
    }
}

template <typename T, int R, int OP>
cudaError_t launch_pcg_t(const MeshDev& m, const OpParams<T>& op, const T* invdiag, const PcgWork& w,
                         double rtol, int maxit, cudaStream_t s, int* grid_used) {
    const size_t smem = (OP == OP_CSR1 || OP == OP_CSR2) ? sizeof(T) * size_t(m.max_touched) * R
                                                         : PatchSmem<T, R>::bytes(m.max_touched, m.max_own);
    auto kern = k_pcg<T, R, OP>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (err != cudaSuccess) return err;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = per_sm * nsm;
    if (grid > kMaxGrid) grid = kMaxGrid;
    if (grid > m.P) grid = m.P;
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
    a.spin_limit = 20000000LL;  // about 2 s of __nanosleep(100) spins
    err = cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), s);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(w.status, 0, sizeof(int), s);
    if (err != cudaSuccess) return err;
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel((void*)kern, dim3(grid), dim3(kThreads), args, smem, s);
}

}  // namespace

int pcg_max_grid() { return kMaxGrid; }

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

template cudaError_t launch_pcg<double>(const MeshDev&, int, int, const OpParams<double>&, const double*,
                                        const PcgWork&, double, int, cudaStream_t, int*);
template cudaError_t launch_pcg<float>(const MeshDev&, int, int, const OpParams<float>&, const float*,
                                       const PcgWork&, double, int, cudaStream_t, int*);

}  // namespace qpat
