// C ABI: mesh handles, workspace, the linear-solve drivers (FP64 PCG and
// FP32 PCG inside FP64 iterative refinement) and the forward / Jacobian /
// prior entry points.  Algorithm 1 lives in recon.cu.
#include <algorithm>
#include <atomic>
#include <set>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "abi_internal.h"
#include "amg.h"

namespace qpat {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    // clear the runtime's last-error slot so that a later launch check does
    // not report this (non-sticky) failure again
    (void)cudaGetLastError();
    return fail(QPAT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void* Workspace::get_bytes(const std::string& name, size_t bytes, cudaStream_t s, cudaError_t* err) {
    *err = cudaSuccess;
    auto it = bufs.find(name);
    if (it != bufs.end() && it->second.second >= bytes) return it->second.first;
    if (it != bufs.end()) {
        cudaStreamSynchronize(s);
        cudaFree(it->second.first);
        bufs.erase(it);
    }
    void* p = nullptr;
    size_t alloc = std::max<size_t>(bytes, 256);
    *err = cudaMalloc(&p, alloc);
    if (*err != cudaSuccess) return nullptr;
    bufs[name] = {p, alloc};
    return p;
}

void Workspace::release() {
    for (auto& kv : bufs) cudaFree(kv.second.first);
    bufs.clear();
}

int round_rhs(int K) {
    if (K <= 1) return 1;
    if (K <= 2) return 2;
    if (K <= 4) return 4;
    if (K <= 8) return 8;
    if (K <= 16) return 16;
    return -1;
}

namespace {

__global__ void k_mul(int64_t n, const double* a, const double* b, double* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = a[i] * b[i];
}

__global__ void k_exp_scale(int64_t n, double c0, const double* u, double* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = c0 * exp(u[i]);
}

// out[l*R + r] = d[l] * x[l*R + r]
__global__ void k_rowscale(int64_t N, int R, const double* d, const double* x, double* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N * R; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = d[i / R] * x[i];
}

// Jv epilogue: out = w o (mu o x + phi o (mu o s2))      (Appendix)
__global__ void k_jv_out(int64_t N, int R, const double* mu, const double* b, const double* x, const double* phi,
                         const double* w, double* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N * R; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t l = i / R;
        const double v = mu[l] * x[i] + phi[i] * b[l];
        out[i] = w ? w[i] * v : v;
    }
}

// J^T epilogue: ok = kappa o y0 ; om = mu o (y1 + sum_r phi_r tw_r)     (Appendix)
__global__ void k_jt_out(int64_t N, int R, const double* kappa, const double* mu, const double* y,
                         const double* phi, const double* tw, double* ok, double* om) {
    for (int64_t l = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; l < N; l += int64_t(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < R; ++r) s += phi[l * R + r] * tw[l * R + r];
        ok[l] = kappa[l] * y[2 * l];
        om[l] = mu[l] * (y[2 * l + 1] + s);
    }
}

// Columns [r0, r0 + Rh) of an N x R node-major block to an N x Rh block and back.
__global__ void k_take_rhs(int64_t N, int R, int r0, int Rh, const double* x, double* xh) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N * Rh; i += int64_t(gridDim.x) * blockDim.x)
        xh[i] = x[(i / Rh) * R + r0 + (i % Rh)];
}
__global__ void k_put_rhs(int64_t N, int R, int r0, int Rh, const double* xh, double* x) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N * Rh; i += int64_t(gridDim.x) * blockDim.x)
        x[(i / Rh) * R + r0 + (i % Rh)] = xh[i];
}

__global__ void k_sqrt_vec(int n, const double* in, double* out) {
    if (threadIdx.x < n) out[threadIdx.x] = sqrt(in[threadIdx.x]);
}

int grid_of(int64_t n) {
    int64_t g = (n + 255) / 256;
    return int(std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16)));
}

}  // namespace

namespace {
__global__ void k_add(int64_t n, const double* a, double* y) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] += a[i];
}
}  // namespace

cudaError_t launch_add(int64_t n, const double* a, double* y, cudaStream_t s) {
    qpat::note_launch(1);
    k_add<<<grid_of(n), 256, 0, s>>>(n, a, y);
    return cudaGetLastError();
}

void k_mul_launch(int64_t n, const double* a, const double* b, double* out, cudaStream_t s) {
    qpat::note_launch(1);
    k_mul<<<grid_of(n), 256, 0, s>>>(n, a, b, out);
}
void k_exp_scale_launch(int64_t n, double c0, const double* u, double* out, cudaStream_t s) {
    qpat::note_launch(1);
    k_exp_scale<<<grid_of(n), 256, 0, s>>>(n, c0, u, out);
}
void k_rowscale_launch(int64_t N, int R, const double* d, const double* x, double* out, cudaStream_t s) {
    qpat::note_launch(1);
    k_rowscale<<<grid_of(N * R), 256, 0, s>>>(N, R, d, x, out);
}
void k_jv_out_launch(int64_t N, int R, const double* mu, const double* b, const double* x, const double* phi,
                     const double* w, double* out, cudaStream_t s) {
    qpat::note_launch(1);
    k_jv_out<<<grid_of(N * R), 256, 0, s>>>(N, R, mu, b, x, phi, w, out);
}
void k_jt_out_launch(int64_t N, int R, const double* kappa, const double* mu, const double* y, const double* phi,
                     const double* tw, double* ok, double* om, cudaStream_t s) {
    qpat::note_launch(1);
    k_jt_out<<<grid_of(N), 256, 0, s>>>(N, R, kappa, mu, y, phi, tw, ok, om);
}

// --------------------------------------------------------------------------
// Linear-solve drivers
// --------------------------------------------------------------------------

uint64_t next_op_stamp() {
    static std::atomic<uint64_t> counter{0};
    return counter.fetch_add(1, std::memory_order_relaxed) + 1;
}

// Operator state of one K(kappa, mu) or M_delta(kt, mt), library order.
int prepare_K(qpat_mesh_s* M, const double* kap_l, const double* mu_l, OpState& st, cudaStream_t s,
              const char* tag) {
    const int64_t N = M->h.N;
    cudaError_t e = cudaSuccess;
    const std::string t(tag);
    st.kind = OP_K;
    st.stamp = next_op_stamp();
    st.c1_64 = kap_l;
    st.c2_64 = mu_l;
    st.c1_32 = M->ws.get<float>(t + ".c1_32", N, s, &e);
    st.c2_32 = M->ws.get<float>(t + ".c2_32", N, s, &e);
    st.inv64 = M->ws.get<double>(t + ".inv64", N, s, &e);
    st.inv32 = M->ws.get<float>(t + ".inv32", N, s, &e);
    st.nv = 1;
    st.v64[0] = M->ws.get<double>(t + ".v64", M->d.sell_entries, s, &e);
    st.v32[0] = M->ws.get<float>(t + ".v32", M->d.sell_entries, s, &e);
    st.gbound = M->ws.get<double>(t + ".gb", 1, s, &e);
    if (e != cudaSuccess) return cuda_fail(e, "workspace");
    if ((e = launch_cast_d2f(N, kap_l, st.c1_32, s)) != cudaSuccess) return cuda_fail(e, "cast");
    if ((e = launch_cast_d2f(N, mu_l, st.c2_32, s)) != cudaSuccess) return cuda_fail(e, "cast");
    if ((e = launch_assemble_K(M->d, kap_l, mu_l, st.v64[0], st.inv64, st.inv32, s, st.gbound)) != cudaSuccess)
        return cuda_fail(e, "assemble_K");
    if ((e = launch_cast_vals(M->d.sell_entries, st.v64[0], st.v32[0], s)) != cudaSuccess)
        return cuda_fail(e, "cast");
    return QPAT_OK;
}

int prepare_prior(qpat_mesh_s* M, const double* kt_l, const double* mt_l, double T, int kind, double q,
                  double b_over_a, double delta,
                  OpState& st, cudaStream_t s) {
    const int64_t N = M->h.N;
    cudaError_t e = cudaSuccess;
    st.kind = OP_PRIOR;
    st.stamp = next_op_stamp();
    st.c1_64 = kt_l;
    st.c2_64 = mt_l;
    st.inv_T2 = 1.0 / (T * T);
    st.prior_kind = kind;
    st.prior_q = q;
    st.scale1 = b_over_a;
    st.delta = delta;
    st.c1_32 = M->ws.get<float>("opP.c1_32", N, s, &e);
    st.c2_32 = M->ws.get<float>("opP.c2_32", N, s, &e);
    st.inv64 = M->ws.get<double>("opP.inv64", 2 * N, s, &e);
    st.inv32 = M->ws.get<float>("opP.inv32", 2 * N, s, &e);
    st.nv = 2;
    st.v64[0] = M->ws.get<double>("opP.v64a", M->dp.sell_entries, s, &e);
    st.v64[1] = M->ws.get<double>("opP.v64b", M->dp.sell_entries, s, &e);
    st.gbound = M->ws.get<double>("opP.gb", 1, s, &e);
    if (e != cudaSuccess) return cuda_fail(e, "workspace");
    if ((e = launch_cast_d2f(N, kt_l, st.c1_32, s)) != cudaSuccess) return cuda_fail(e, "cast");
    if ((e = launch_cast_d2f(N, mt_l, st.c2_32, s)) != cudaSuccess) return cuda_fail(e, "cast");
    if ((e = launch_assemble_prior(M->dp, kt_l, mt_l, st.inv_T2, kind, q, b_over_a, delta, st.v64[0], st.v64[1],
                                   st.inv64, st.inv32, s, st.gbound)) != cudaSuccess)
        return cuda_fail(e, "assemble_prior");
    return QPAT_OK;
}

// FP64 operator apply of the refinement residual: the assembled values
// (two FP64 flops per stored entry; GB300 runs FP64 at ~1/64 of FP32, so the
// element recomputation is kept for FP32 only).
static cudaError_t apply_op64(qpat_mesh_s* M, const OpState& st, int R, const double* x, double* y,
                              cudaStream_t s) {
    return launch_apply_csr<double>(st.kind == OP_PRIOR ? M->dp : M->d, st.nv, R, st.v64[0], st.v64[1], x, y, s);
}

static int pcg_status(int st, const char* what) {
    if (st == QPAT_OK) return QPAT_OK;
    if (st == QPAT_ETIMEOUT) return fail(st, std::string(what) + ": grid barrier timed out");
    if (st == QPAT_EBREAKDOWN) return fail(st, std::string(what) + ": PCG breakdown (p.Ap <= 0 or not finite)");
    if (st == QPAT_ENOCONV) return fail(st, std::string(what) + ": PCG iteration cap reached");
    return fail(st, std::string(what) + ": PCG failed");
}

// Solves A X = B for R right-hand sides (library order, N x R node-major,
// FP64 in and out).  precision 0: FP64 PCG to rtol.  precision 1: X = 0,
// then sweeps of  r = B - A X (FP64 element apply), d = A32^-1 (r / |r|)
// (FP32 PCG to a loose tolerance), X += |r| d,  until |r_j| <= rtol |B_j|.
int solve(qpat_mesh_s* M, const OpState& st, const SolveOpts& so_in, int R, const double* B, double* X,
          cudaStream_t s, const double* X0) {
    // M_delta is solved in FP64 whatever the precision mode: its smallest
    // eigenvalue is delta (constant mode, 1e-6 below the rest) and the
    // lagged weights reach ~1e-5 across edges, beyond what an FP32 inner
    // solve can resolve, so refinement would not contract.
    SolveOpts so = so_in;
    if (st.kind == OP_PRIOR) so.precision = 0;
    // multigrid-preconditioned CG (FP64 iterates whatever the precision mode)
    if (so.multigrid) return amg_solve(M, st, so, R, B, X, s, X0);
    // the prior's assembled blocks live in the stiffness-only pattern
    const MeshDev& md = st.kind == OP_PRIOR ? M->dp : M->d;
    const int64_t N = M->h.N;
    const int64_t n = N * R;
    cudaError_t e = cudaSuccess;
    {
        // More right-hand sides than one launch's shared memory holds on
        // this mesh's patches (e.g. 16 FP64 RHS on ~1000-node patches): the
        // block is solved as two halves of R/2, each RHS with the same
        // arithmetic as in one launch.
        const bool asm_ = so.precision == 0 || so.fp32_assembled;
        const bool poly_ok = asm_ && so.pcg_variant != 2 && so.pcg_variant != 3 && st.gbound;
        const int deg = poly_ok ? (st.kind == OP_PRIOR ? so.poly_prior : so.poly_k) : 0;
        const int op64 = st.kind == OP_K ? OP_CSR1 : OP_CSR2;
        bool fits = pcg_fits<double>(md, op64, R, deg) && (!X0 || apply_csr_fits<double>(md, R));
        if (fits && so.precision == 1)
            fits = pcg_fits<float>(md, so.fp32_assembled ? OP_CSR1 : OP_K, R, deg) && apply_csr_fits<double>(md, R);
        if (!fits && R > 1) {
            const int Rh = R / 2;
            const std::string tag = "split" + std::to_string(R);
            double* Bh = M->ws.get<double>(tag + ".b", N * Rh, s, &e);
            double* Xh = M->ws.get<double>(tag + ".x", N * Rh, s, &e);
            double* X0h = X0 ? M->ws.get<double>(tag + ".x0", N * Rh, s, &e) : nullptr;
            if (e != cudaSuccess) return cuda_fail(e, "workspace");
            for (int half = 0; half < 2; ++half) {
                qpat::note_launch(1);
                k_take_rhs<<<grid_of(N * Rh), 256, 0, s>>>(N, R, half * Rh, Rh, B, Bh);
                if (X0) {
                    qpat::note_launch(1);
                    k_take_rhs<<<grid_of(N * Rh), 256, 0, s>>>(N, R, half * Rh, Rh, X0, X0h);
                }
                if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "split");
                const int rc = solve(M, st, so_in, Rh, Bh, Xh, s, X0h);
                if (rc != QPAT_OK) return rc;
                qpat::note_launch(1);
                k_put_rhs<<<grid_of(N * Rh), 256, 0, s>>>(N, R, half * Rh, Rh, Xh, X);
                if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "split");
            }
            return QPAT_OK;
        }
    }
    PcgWork w{};
    const char* pfx = st.kind == OP_K ? "pcg" : "pcgP";
    auto nm = [&](const char* a) { return std::string(pfx) + "." + a; };
    const size_t esz = so.precision == 0 ? sizeof(double) : sizeof(float);
    w.r = M->ws.get_bytes(nm("r"), n * esz, s, &e);
    w.p0 = M->ws.get_bytes(nm("p0"), n * esz, s, &e);
    w.p1 = M->ws.get_bytes(nm("p1"), n * esz, s, &e);
    w.q = M->ws.get_bytes(nm("q"), n * esz, s, &e);
    w.partials = M->ws.get<double>("pcg.partials", pcg_partials_doubles(), s, &e);
    w.bar = M->ws.get<unsigned>("pcg.bar", 2, s, &e);
    w.status = M->ws.get<int>("pcg.status", 1, s, &e);
    w.iters = M->ws.get<int>("pcg.iters", 1, s, &e);
    w.stats = M->ws.get<double>("pcg.stats", 32, s, &e);
    w.spin_limit = so.spin_limit;
    // PCG variant on the assembled operators (the matrix-free FP32 operator has one)
    const bool assembled = so.precision == 0 || so.fp32_assembled;
    const bool single = assembled && so.pcg_variant == 2;
    const bool ring = assembled && so.pcg_variant == 3;
    // patch-local Chebyshev preconditioner: two-reduction kernel, assembled values
    if (assembled && !single && !ring && st.gbound) {
        w.poly_deg = st.kind == OP_PRIOR ? so.poly_prior : so.poly_k;
        w.poly_hi = st.gbound;
    }
    if (single) {
        w.r1 = M->ws.get_bytes(nm("r1"), n * esz, s, &e);
        w.s0 = M->ws.get_bytes(nm("s0"), n * esz, s, &e);
        w.s1 = M->ws.get_bytes(nm("s1"), n * esz, s, &e);
        w.w1 = M->ws.get_bytes(nm("w1"), n * esz, s, &e);
    }
    double* hpin = M->host_scratch;  // pinned, >= 64 doubles
    if (e != cudaSuccess) return cuda_fail(e, "workspace");
    if (so.precision == 0 && X0) {
        // initial guess: solve A D = B - A X0 with D0 = 0 to the same absolute
        // target |B - A X| <= rtol |B| (per RHS), then X = X0 + D
        double* Bp = M->ws.get<double>(std::string(pfx) + ".b0", n, s, &e);
        double* tmp = M->ws.get<double>(std::string(pfx) + ".t0", n, s, &e);
        double* dpart = M->ws.get<double>("dots.partial", 608 * 16, s, &e);
        double* dn = M->ws.get<double>(std::string(pfx) + ".n0", 64, s, &e);
        if (e != cudaSuccess) return cuda_fail(e, "workspace");
        if ((e = apply_op64(M, st, R, X0, tmp, s)) != cudaSuccess) return cuda_fail(e, "apply64");
        if ((e = launch_sub(n, B, tmp, Bp, s)) != cudaSuccess) return cuda_fail(e, "sub");
        if ((e = launch_dots<double>(N, R, B, B, dpart, dn, s)) != cudaSuccess ||
            (e = launch_dots<double>(N, R, Bp, Bp, dpart, dn + 16, s)) != cudaSuccess)
            return cuda_fail(e, "dots");
        if ((e = cudaMemcpyAsync(hpin, dn, 32 * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(e, "copy");
        double scale = INFINITY;
        for (int r = 0; r < R; ++r)
            if (hpin[16 + r] > 0.0) scale = std::min(scale, std::sqrt(hpin[r] / hpin[16 + r]));
        if (!std::isfinite(scale)) scale = 1.0;
        SolveOpts s2 = so;
        s2.rtol = so.rtol * std::max(scale, 1.0);
        int rc = solve(M, st, s2, R, Bp, X, s, nullptr);
        if (rc != QPAT_OK) return rc;
        if ((e = launch_add(n, X0, X, s)) != cudaSuccess) return cuda_fail(e, "add");
        return QPAT_OK;
    }
    if (so.precision == 0) {
        w.b = const_cast<double*>(B);
        w.x = X;
        // z = D^-1 r kept by the owner: the halo staging then needs one FP64
        // FMA per value instead of a multiply and an FMA
        w.z = M->ws.get_bytes(nm("z"), n * esz, s, &e);
        if (e != cudaSuccess) return cuda_fail(e, "workspace");
        const int OP = st.kind == OP_K ? OP_CSR1 : OP_CSR2;
        OpParams<double> op{st.c1_64, st.c2_64, st.inv_T2, st.scale1, st.delta, 1, st.v64[0], st.v64[1]};
        if (M->timing) cudaEventRecord(M->ev0, s);
        e = cudaErrorNotSupported;
        if (ring) e = launch_pcg_ring<double>(md, OP, R, op, st.inv64, w, so.rtol, so.maxit, s, nullptr);
        if (e == cudaErrorNotSupported) {
            if (so.pcg_variant == 3) return fail(QPAT_EINVAL, "pcg: the bulk-copy ring does not fit this mesh");
            e = single ? launch_pcg1<double>(md, OP, R, op, st.inv64, w, so.rtol, so.maxit, s, nullptr)
                       : launch_pcg<double>(md, OP, R, op, st.inv64, w, so.rtol, so.maxit, s, nullptr);
        }
        if (e != cudaSuccess) return cuda_fail(e, "pcg launch");
        if (M->timing) cudaEventRecord(M->ev1, s);
        int hst[2];
        if ((e = cudaMemcpyAsync(hst, w.status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(hst + 1, w.iters, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(e, "pcg sync");
        if (M->timing) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, M->ev0, M->ev1);
            M->pcg_ms += ms;
        }
        M->stats.pcg_iters += hst[1];
        M->stats.rhs_iters += int64_t(hst[1]) * R;
        M->stats.solves += R;
        M->stats.launches += 1;
        return pcg_status(hst[0], pfx);
    }

    // ---- FP32 PCG inside FP64 refinement.  If the FP32 inner solve breaks
    // down or the refinement stalls (an iterate's coefficients outside the
    // range FP32 resolves), this system is solved again by the FP64 PCG.
    auto refine = [&]() -> int {
        double* Rres = M->ws.get<double>(nm("res64"), n, s, &e);
        double* tmp = M->ws.get<double>(nm("tmp64"), n, s, &e);
        float* b32 = M->ws.get<float>(nm("b32"), n, s, &e);
        float* x32 = M->ws.get<float>(nm("x32"), n, s, &e);
        double* dpart = M->ws.get<double>("dots.partial", 608 * 16, s, &e);
        double* dnorm = M->ws.get<double>(nm("norms"), 64, s, &e);  // [0,R): |r|^2, [16,16+R): |B|^2, [32,..): |r|
        if (e != cudaSuccess) return cuda_fail(e, "workspace");
        w.b = b32;
        w.x = x32;
        if (w.poly_deg > 0) {
            // the polynomial preconditioner keeps z by the owner
            w.z = M->ws.get_bytes(nm("z32"), n * esz, s, &e);
            if (e != cudaSuccess) return cuda_fail(e, "workspace");
        }
        const int OP = so.fp32_assembled ? OP_CSR1 : OP_K;
        OpParams<float> op{st.c1_32, st.c2_32, float(st.inv_T2), float(st.scale1), float(st.delta), 1, st.v32[0],
                           nullptr};
        if (X0) {
            // start from the initial guess: X = X0, r = B - A X0
            if ((e = cudaMemcpyAsync(X, X0, n * sizeof(double), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
                return cuda_fail(e, "copy");
            if ((e = apply_op64(M, st, R, X, tmp, s)) != cudaSuccess) return cuda_fail(e, "apply64");
            if ((e = launch_sub(n, B, tmp, Rres, s)) != cudaSuccess) return cuda_fail(e, "sub");
        } else {
            if ((e = cudaMemsetAsync(X, 0, n * sizeof(double), s)) != cudaSuccess) return cuda_fail(e, "memset");
            if ((e = cudaMemcpyAsync(Rres, B, n * sizeof(double), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
                return cuda_fail(e, "copy");
        }
        if ((e = launch_dots<double>(N, R, B, B, dpart, dnorm + 16, s)) != cudaSuccess) return cuda_fail(e, "dots");
        if ((e = cudaMemcpyAsync(hpin + 16, dnorm + 16, R * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_fail(e, "copy");
        // Reliable updates: each inner run continues the previous one's search
        // direction (rescaled to the new RHS scaling) instead of restarting,
        // with r replaced by the true FP64 residual; the Krylov space built in
        // FP32 is kept across the FP64 corrections.
        const bool reliable = !so.mixed_restart && !single && !ring;
        double* gam = M->ws.get<double>(nm("gamma"), 16, s, &e);
        double* rzst = M->ws.get<double>(nm("rzstate"), 16, s, &e);
        int* pbufp = M->ws.get<int>(nm("pbuf"), 1, s, &e);
        if (e != cudaSuccess) return cuda_fail(e, "workspace");
        double prev_scale[16];
        w.rz_state = reliable ? rzst : nullptr;
        w.pbuf = reliable ? pbufp : nullptr;
        bool resume_next = false;  // set when the last inner run ended normally
        int first_iters = 0;       // iterations of this solve's first inner run
        int sweeps = 0;
        for (;;) {
            if ((e = launch_dots<double>(N, R, Rres, Rres, dpart, dnorm, s)) != cudaSuccess) return cuda_fail(e, "dots");
            if ((e = cudaMemcpyAsync(hpin, dnorm, R * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
                return cuda_fail(e, "copy");
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "sync");
            bool done = true;
            for (int r = 0; r < R; ++r) {
                if (!std::isfinite(hpin[r])) return fail(QPAT_EBREAKDOWN, "refinement: residual not finite");
                if (hpin[r] > so.rtol * so.rtol * hpin[16 + r]) done = false;
            }
            if (done) break;
            if (sweeps >= so.max_sweeps) return fail(QPAT_ENOCONV, "refinement: sweep cap reached");
            w.resume_gamma = nullptr;
            if (reliable && sweeps > 0 && resume_next) {
                // safeguard: continue the previous direction only while the
                // last run cut every residual that was not converged by 10x;
                // otherwise the FP32 recurrence has drifted and a fresh start
                // is better
                bool progress = true;
                for (int r = 0; r < R; ++r) {
                    const double nr = std::sqrt(hpin[r]);
                    if (hpin[r] > so.rtol * so.rtol * hpin[16 + r] && nr > 0.1 * prev_scale[r]) progress = false;
                    hpin[48 + r] = nr > 0.0 ? prev_scale[r] / nr : 0.0;
                }
                if (progress) {
                if ((e = cudaMemcpyAsync(gam, hpin + 48, R * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess)
                    return cuda_fail(e, "copy");
                w.resume_gamma = gam;
                }
            }
            for (int r = 0; r < R; ++r) prev_scale[r] = std::sqrt(hpin[r]);
            ++sweeps;
            qpat::note_launch(1);
            k_sqrt_vec<<<1, 32, 0, s>>>(R, dnorm, dnorm + 32);
            if ((e = launch_cast_d2f_scaled(N, R, Rres, dnorm + 32, b32, s)) != cudaSuccess) return cuda_fail(e, "cast");
            if (M->timing) cudaEventRecord(M->ev0, s);
            // a resumed run that needs far more iterations than the first run
            // has stagnated in FP32: it is cut short and the next run restarts
            const int seg_maxit = w.resume_gamma ? std::min(so.maxit, std::max(100, 2 * first_iters)) : so.maxit;
            e = cudaErrorNotSupported;
            if (ring) e = launch_pcg_ring<float>(M->d, OP, R, op, st.inv32, w, so.inner_rtol, seg_maxit, s, nullptr);
            if (e == cudaErrorNotSupported) {
                if (so.pcg_variant == 3) return fail(QPAT_EINVAL, "pcg32: the bulk-copy ring does not fit this mesh");
                e = single ? launch_pcg1<float>(M->d, OP, R, op, st.inv32, w, so.inner_rtol, seg_maxit, s, nullptr)
                           : launch_pcg<float>(M->d, OP, R, op, st.inv32, w, so.inner_rtol, seg_maxit, s, nullptr);
            }
            if (e != cudaSuccess) return cuda_fail(e, "pcg32 launch");
            if (M->timing) cudaEventRecord(M->ev1, s);
            int hst[2];
            if ((e = cudaMemcpyAsync(hst, w.status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
                (e = cudaMemcpyAsync(hst + 1, w.iters, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
                return cuda_fail(e, "copy");
            if ((e = launch_axpy_f2d_scaled(N, R, x32, dnorm + 32, X, s)) != cudaSuccess) return cuda_fail(e, "axpy");
            if ((e = apply_op64(M, st, R, X, tmp, s)) != cudaSuccess) return cuda_fail(e, "apply64");
            if ((e = launch_sub(n, B, tmp, Rres, s)) != cudaSuccess) return cuda_fail(e, "sub");
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "sync");
            if (M->timing) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, M->ev0, M->ev1);
                M->pcg_ms += ms;
            }
            M->stats.pcg_iters += hst[1];
            M->stats.rhs_iters += int64_t(hst[1]) * R;
            M->stats.launches += 1;
            M->stats.refinements += 1;
            // an inner run that stops at its cap still improves x (the next
            // one then starts afresh); breakdown or timeout is fatal
            if (hst[0] == QPAT_ETIMEOUT || hst[0] == QPAT_EBREAKDOWN) return pcg_status(hst[0], "pcg32");
            resume_next = hst[0] == QPAT_OK;
            if (sweeps == 1) first_iters = hst[1];
        }
        M->stats.solves += R;
        return QPAT_OK;
    };
    const int rc = refine();
    if (rc != QPAT_EBREAKDOWN && rc != QPAT_ENOCONV) return rc;
    M->stats.fp64_fallbacks += 1;
    SolveOpts s64 = so;
    s64.precision = 0;
    return solve(M, st, s64, R, B, X, s, X0);
}

}  // namespace qpat

using namespace qpat;

// --------------------------------------------------------------------------
// Public entry points
// --------------------------------------------------------------------------

namespace qpat {
static std::atomic<long long> g_launches{0};

cudaError_t allow_smem(const void* func, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> raised;  // (device, kernel) -> allowed bytes
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dev, func);
    auto it = raised.find(key);
    if (it == raised.end()) {
        int optin = 0;
        cudaFuncAttributes fa{};
        if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess ||
            (e = cudaFuncGetAttributes(&fa, func)) != cudaSuccess)
            return e;
        const size_t lim = size_t(optin) > fa.sharedSizeBytes ? size_t(optin) - fa.sharedSizeBytes : 0;
        if ((e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, int(lim))) != cudaSuccess)
            return e;
        it = raised.emplace(key, lim).first;
    }
    return smem <= it->second ? cudaSuccess : cudaErrorInvalidValue;
}
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace qpat

extern "C" {

const char* qpat_last_error(void) { return g_err.c_str(); }

int64_t qpat_launch_count(void) { return int64_t(qpat::g_launches.load(std::memory_order_relaxed)); }

void qpat_default_params(qpat_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->T = 5e-3;
    p->b_over_a = 1.0;
    p->delta = 1e-6;
    p->tau = 1e-2;
    p->m0 = 10;
    p->max_lin = 5;
    p->max_lsqr = 50;
    p->fixed_counts = 0;
    p->precision = 0;
    p->max_pcg_iter = 20000;
    p->pcg_rtol = 1e-13;
    p->fit_grid = 9;
    p->fit_gn_steps = 10;
    p->patch_nodes = 0;
    p->prior = 0;
    p->prior_q = 1.0;
    p->poly_degree = 2;        // fastest measured on a 64^3 cube (GB300)
    p->prior_poly_degree = 2;
    p->lsqr_reorth = 1;        // exact-arithmetic LSQR iterates (see qpat.h)
    p->multigrid = 0;
    p->mg_degree = 1;          // fewer FP64 fine-level products per cycle; fastest measured at 64^3 and 128^3
    p->mg_ratio = 30.0;
}

static int mesh_create(const double* xyz, int64_t N, const int32_t* tets, int64_t E, int patch_nodes,
                       int patch_multiple, qpat_mesh_t* out) {
    if (!out) return fail(QPAT_EINVAL, "qpat_mesh: out is NULL");
    *out = nullptr;
    auto* M = new qpat_mesh_s();
    std::string msg = build_host_mesh(xyz, N, tets, E, patch_nodes, patch_multiple, M->h);
    if (!msg.empty()) {
        delete M;
        return fail(QPAT_EINVAL, msg);
    }
    int rc = upload_mesh(M);
    if (rc != QPAT_OK) {
        qpat_mesh_free(M);
        return rc;
    }
    *out = M;
    return QPAT_OK;
}

int qpat_multigrid_host_info(const double* xyz, int64_t N, const int32_t* tets, int64_t E, int patch_nodes,
                             int prior, int64_t* rows, int max_levels) {
    if (max_levels < 0 || (max_levels > 0 && !rows)) return fail(QPAT_EINVAL, "qpat_multigrid_host_info: bad argument");
    HostMesh h;
    std::string msg = build_host_mesh(xyz, N, tets, E, patch_nodes, 0, h);
    if (!msg.empty()) return fail(QPAT_EINVAL, msg);
    const AmgPlan plan = amg_build_plan(amg_fine_pattern(h, prior ? 1 : 0));
    msg = amg_check_plan(plan);
    if (!msg.empty()) return fail(QPAT_EINVAL, "multigrid plan: " + msg);
    const int L = int(plan.levels.size());
    for (int l = 0; l < std::min(L, max_levels); ++l) rows[l] = plan.levels[size_t(l)].A.n;
    return L;
}

int qpat_mesh_host_info(const double* xyz, int64_t N, const int32_t* tets, int64_t E, int patch_nodes,
                        int64_t* info8, int32_t* faces, int32_t* perm) {  // info8: 11 entries
    if (!info8) return fail(QPAT_EINVAL, "qpat_mesh_host_info: info is NULL");
    HostMesh h;
    std::string msg = build_host_mesh(xyz, N, tets, E, patch_nodes, 0, h);
    if (!msg.empty()) return fail(QPAT_EINVAL, msg);
    // self-check of the patch structure: owned ranges tile [0, N); every tet
    // that touches an owned node is listed; local ids map back to the tets
    int64_t dup = 0;
    std::vector<int> stamp(h.N, -1);
    for (int p = 0; p < h.P; ++p) {
        const int ob = h.own_begin[p], oe = h.own_begin[p + 1], nb = h.node_ptr[p];
        // touched nodes are distinct, owned ones first and in order
        for (int i = nb; i < h.node_ptr[p + 1]; ++i) {
            const int g = h.nodes[i];
            if (stamp[g] == p) return fail(QPAT_EINVAL, "host check: duplicate touched node");
            stamp[g] = p;
            if (i - nb < oe - ob && g != ob + (i - nb)) return fail(QPAT_EINVAL, "host check: owned order");
        }
        for (int t = h.tet_ptr[p]; t < h.tet_ptr[p + 1]; ++t) {
            int owned = 0;
            for (int a = 0; a < 4; ++a) {
                const int li = h.tet_loc[4 * t + a];
                if (li >= h.node_ptr[p + 1] - nb) return fail(QPAT_EINVAL, "host check: local id out of range");
                const int g = h.nodes[nb + li];
                if ((li < oe - ob) != (g >= ob && g < oe)) return fail(QPAT_EINVAL, "host check: owned flag wrong");
                owned |= (g >= ob && g < oe);
            }
            if (!owned) return fail(QPAT_EINVAL, "host check: patch tet without owned node");
        }
        dup += h.tet_ptr[p + 1] - h.tet_ptr[p];
        // colours: they tile the patch's tet (face) list in order, and no two
        // elements of one colour share an owned vertex
        auto check_colours = [&](const std::vector<int32_t>& beg, const std::vector<int32_t>& off,
                                 const std::vector<int32_t>& ptr, const std::vector<uint16_t>& loc, int nv) -> bool {
            const int j0 = beg[p], j1 = beg[p + 1];
            if (j1 <= j0 || off[j0] != ptr[p] || off[j1 - 1] != ptr[p + 1]) return false;
            std::vector<int> seen(size_t(oe - ob), -1);
            for (int j = j0; j + 1 < j1; ++j) {
                if (off[j + 1] < off[j]) return false;
                for (int e = off[j]; e < off[j + 1]; ++e)
                    for (int a = 0; a < nv; ++a) {
                        const int li = loc[4 * size_t(e) + a];
                        if (li < oe - ob) {
                            if (seen[li] == j) return false;
                            seen[li] = j;
                        }
                    }
            }
            return true;
        };
        if (!check_colours(h.tcol_beg, h.tcol_off, h.tet_ptr, h.tet_loc, 4) ||
            !check_colours(h.fcol_beg, h.fcol_off, h.face_ptr, h.face_loc, 3))
            return fail(QPAT_EINVAL, "host check: element colours");
    }
    info8[0] = h.F;
    info8[1] = h.P;
    info8[2] = h.max_touched;
    info8[3] = h.max_own;
    info8[4] = h.max_ptets;
    info8[5] = h.max_pfaces;
    info8[6] = dup;  // sum over patches of listed tets (>= E; the excess is border duplication)
    info8[7] = int64_t(h.face_ptr[h.P]);
    info8[10] = h.max_tcolors;
    // the prior's stiffness-only pattern: a subset of the full pattern, with
    // every diagonal, symmetric in global ids
    {
        std::set<std::pair<int, int>> full, sub;
        int64_t nfull = 0, nsub = 0;
        for (int p = 0; p < h.P; ++p) {
            const int nb = h.node_ptr[p];
            for (int g = h.own_begin[p]; g < h.own_begin[p + 1]; ++g) {
                const int64_t b0 = h.sell_ptr[g >> 5] * 32 + (g & 31), b1 = h.psell_ptr[g >> 5] * 32 + (g & 31);
                for (int k = 0; k < h.sell_len[g]; ++k) full.insert({g, h.nodes[nb + h.sell_col[b0 + int64_t(k) * 32]]});
                bool diag = false;
                for (int k = 0; k < h.psell_len[g]; ++k) {
                    const int j = h.nodes[nb + h.psell_col[b1 + int64_t(k) * 32]];
                    sub.insert({g, j});
                    diag |= j == g;
                }
                if (!diag || h.psell_col[b1 + int64_t(h.psell_diag[g]) * 32] != g - h.own_begin[p])
                    return fail(QPAT_EINVAL, "host check: stiffness pattern diagonal");
                nfull += h.sell_len[g];
                nsub += h.psell_len[g];
            }
        }
        for (const auto& e : sub) {
            if (!full.count(e)) return fail(QPAT_EINVAL, "host check: stiffness pattern not a subset");
            if (!sub.count({e.second, e.first})) return fail(QPAT_EINVAL, "host check: stiffness pattern not symmetric");
        }
        info8[8] = nfull;
        info8[9] = nsub;
    }
    if (faces) std::memcpy(faces, h.faces_caller.data(), sizeof(int32_t) * 3 * h.F);
    if (perm) std::memcpy(perm, h.perm.data(), sizeof(int32_t) * h.N);
    // every tet must be listed once per distinct patch owning one of its
    // vertices (node g belongs to the patch of its 32-node slice)
    int64_t expect = 0;
    for (int64_t e = 0; e < h.E; ++e) {
        int pid[4];
        for (int a = 0; a < 4; ++a) pid[a] = h.patch_of_slice[h.tets[4 * e + a] >> 5];
        std::sort(pid, pid + 4);
        expect += 1 + (pid[1] != pid[0]) + (pid[2] != pid[1]) + (pid[3] != pid[2]);
    }
    if (expect != dup) return fail(QPAT_EINVAL, "host check: patch tet lists do not cover the mesh");
    // assembled pattern: row g lists exactly g and its edge neighbours, each once
    std::vector<std::vector<int>> adj(h.N);
    for (int64_t e = 0; e < h.E; ++e)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) adj[h.tets[4 * e + a]].push_back(h.tets[4 * e + b]);
    for (int64_t g = 0; g < h.N; ++g) {
        auto& ref = adj[g];
        std::sort(ref.begin(), ref.end());
        ref.erase(std::unique(ref.begin(), ref.end()), ref.end());
        const int p = h.patch_of_slice[g >> 5], nb = h.node_ptr[p];
        std::vector<int> got;
        for (int k = 0; k < h.sell_len[g]; ++k)
            got.push_back(h.nodes[nb + h.sell_col[(h.sell_ptr[g >> 5] + k) * 32 + (g & 31)]]);
        std::sort(got.begin(), got.end());
        if (got != ref) return fail(QPAT_EINVAL, "host check: assembled pattern row " + std::to_string(g));
        const int64_t d = (h.sell_ptr[g >> 5] + h.sell_diag[g]) * 32 + (g & 31);
        if (h.nodes[nb + h.sell_col[d]] != g) return fail(QPAT_EINVAL, "host check: diagonal slot");
    }
    return QPAT_OK;
}

static constexpr int kPatchesPerSm = 2;

int qpat_mesh(const double* xyz, int64_t N, const int32_t* tets, int64_t E, qpat_mesh_t* out) {
    // default patching: at most 1024 owned nodes per patch and a patch count
    // that is a multiple of 2 CTAs per SM (the residency of the FP64 solver
    // kernels), so that every resident CTA of the persistent solver owns the
    // same number of patches
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess || nsm < 1) {
        (void)cudaGetLastError();
        nsm = 152;
    }
    return mesh_create(xyz, N, tets, E, 1024, kPatchesPerSm * nsm, out);
}

int qpat_mesh_ex(const double* xyz, int64_t N, const int32_t* tets, int64_t E, int patch_nodes, qpat_mesh_t* out) {
    return mesh_create(xyz, N, tets, E, patch_nodes, 0, out);
}

void qpat_mesh_free(qpat_mesh_t M) {
    if (!M) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(M->device);
    if (M->stream) cudaStreamSynchronize(M->stream);
    qpat::amg_release(M);
    M->ws.release();
    if (M->ev0) cudaEventDestroy(M->ev0);
    if (M->ev1) cudaEventDestroy(M->ev1);
    for (void* p : M->dev_allocs) cudaFree(p);
    if (M->host_scratch) cudaFreeHost(M->host_scratch);
    if (M->stream) cudaStreamDestroy(M->stream);
    cudaSetDevice(cur);
    delete M;
}

int64_t qpat_mesh_num_nodes(qpat_mesh_t M) { return M ? M->h.N : -1; }
int64_t qpat_mesh_num_tets(qpat_mesh_t M) { return M ? M->h.E : -1; }
int64_t qpat_mesh_num_faces(qpat_mesh_t M) { return M ? M->h.F : -1; }
int64_t qpat_mesh_num_patches(qpat_mesh_t M) { return M ? M->h.P : -1; }

int64_t qpat_mesh_num_entries(qpat_mesh_t M) {
    if (!M) return -1;
    int64_t n = 0;
    for (uint8_t l : M->h.sell_len) n += l;
    return n;
}

int64_t qpat_mesh_num_prior_entries(qpat_mesh_t M) {
    if (!M) return -1;
    int64_t n = 0;
    for (uint8_t l : M->h.psell_len) n += l;
    return n;
}

int64_t qpat_mesh_num_local_entries(qpat_mesh_t M, int prior) {
    if (!M) return -1;
    const HostMesh& h = M->h;
    const auto& ptr = prior ? h.psell_ptr : h.sell_ptr;
    const auto& col = prior ? h.psell_col : h.sell_col;
    const auto& len = prior ? h.psell_len : h.sell_len;
    int64_t n = 0;
    for (int64_t g = 0; g < h.N; ++g) {
        const int p = h.patch_of_slice[size_t(g >> 5)];
        const int nown = h.own_begin[size_t(p) + 1] - h.own_begin[size_t(p)];
        const int64_t base = ptr[size_t(g >> 5)] * 32 + (g & 31);
        for (int k = 0; k < len[size_t(g)]; ++k)
            if (col[size_t(base + int64_t(k) * 32)] < nown) ++n;
    }
    return n;
}

int qpat_mesh_faces(qpat_mesh_t M, int32_t* faces) {
    if (!M || !faces) return fail(QPAT_EINVAL, "qpat_mesh_faces: NULL argument");
    std::memcpy(faces, M->h.faces_caller.data(), sizeof(int32_t) * 3 * M->h.F);
    return QPAT_OK;
}

int qpat_mesh_permutation(qpat_mesh_t M, int32_t* perm) {
    if (!M || !perm) return fail(QPAT_EINVAL, "qpat_mesh_permutation: NULL argument");
    std::memcpy(perm, M->h.perm.data(), sizeof(int32_t) * M->h.N);
    return QPAT_OK;
}

int qpat_mesh_stats(qpat_mesh_t M, int64_t* out4) {
    if (!M || !out4) return fail(QPAT_EINVAL, "qpat_mesh_stats: NULL argument");
    out4[0] = M->stats.pcg_iters;
    out4[1] = M->stats.solves;
    out4[2] = M->stats.refinements;
    out4[3] = M->stats.launches;
    return QPAT_OK;
}

int64_t qpat_mesh_fp64_fallbacks(qpat_mesh_t M) { return M ? M->stats.fp64_fallbacks : -1; }

int64_t qpat_mesh_rhs_iterations(qpat_mesh_t M) { return M ? M->stats.rhs_iters : -1; }

int qpat_mesh_multigrid_fine_time(qpat_mesh_t M, double* ms, int64_t* launches) {
    if (!M || !ms || !launches) return qpat::fail(QPAT_EINVAL, "qpat_mesh_multigrid_fine_time: bad argument");
    *ms = M->mg_fine_ms;
    *launches = M->mg_fine_launches;
    return QPAT_OK;
}

int qpat_mesh_multigrid_levels(qpat_mesh_t M, int prior, int64_t* rows, int max_levels) {
    if (!M || (max_levels > 0 && !rows) || max_levels < 0) return qpat::fail(QPAT_EINVAL, "qpat_mesh_multigrid_levels: bad argument");
    return qpat::amg_levels(M, prior, rows, max_levels);
}

int qpat_mesh_reset_stats(qpat_mesh_t M) {
    if (!M) return fail(QPAT_EINVAL, "qpat_mesh_reset_stats: NULL mesh");
    M->stats = SolveStats();
    M->pcg_ms = 0.0;
    M->mg_fine_ms = 0.0;
    M->mg_fine_launches = 0;
    return QPAT_OK;
}

int qpat_mesh_set_timing(qpat_mesh_t M, int on) {
    if (!M) return fail(QPAT_EINVAL, "qpat_mesh_set_timing: NULL mesh");
    DeviceGuard dg(M->device);
    if (on && !M->ev0) {
        cudaError_t e = cudaEventCreate(&M->ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&M->ev1);
        if (e != cudaSuccess) return cuda_fail(e, "qpat_mesh_set_timing");
    }
    M->timing = on ? 1 : 0;
    return QPAT_OK;
}

int qpat_mesh_pcg_time(qpat_mesh_t M, double* ms) {
    if (!M || !ms) return fail(QPAT_EINVAL, "qpat_mesh_pcg_time: NULL argument");
    *ms = M->pcg_ms;
    return QPAT_OK;
}

int qpat_flux_patch(qpat_mesh_t M, const double c[3], const double n[3], double half_w, double amp,
                    double* flux_face) {
    if (!M || !c || !n || !flux_face) return fail(QPAT_EINVAL, "qpat_flux_patch: NULL argument");
    if (!(half_w >= 0.0) || (n[0] == 0 && n[1] == 0 && n[2] == 0))
        return fail(QPAT_EINVAL, "qpat_flux_patch: bad half width or zero normal");
    flux_patch_host(M->h, c, n, half_w, amp, flux_face);
    return QPAT_OK;
}

int qpat_flux_side(qpat_mesh_t M, const double c[3], const double axis[3], const double ref[3], double radius,
                   double theta0, double half_w, double amp, double* flux_face) {
    if (!M || !c || !axis || !ref || !flux_face) return fail(QPAT_EINVAL, "qpat_flux_side: NULL argument");
    const double an = std::sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
    if (!(an > 0) || !(radius > 0) || !(half_w > 0)) return fail(QPAT_EINVAL, "qpat_flux_side: bad axis, radius or width");
    const double ra = (ref[0] * axis[0] + ref[1] * axis[1] + ref[2] * axis[2]) / an;
    const double rn2 = ref[0] * ref[0] + ref[1] * ref[1] + ref[2] * ref[2] - ra * ra;
    if (!(rn2 > 1e-24 * (ref[0] * ref[0] + ref[1] * ref[1] + ref[2] * ref[2])))
        return fail(QPAT_EINVAL, "qpat_flux_side: ref is parallel to the axis");
    flux_side_host(M->h, c, axis, ref, radius, theta0, half_w, amp, flux_face);
    return QPAT_OK;
}

int qpat_apply_K_dev(qpat_mesh_t M, int precision, const double* kappa, const double* mu, int R, const double* x,
                     double* y, void* stream) {
    if (!M || !kappa || !mu || !x || !y) return fail(QPAT_EINVAL, "qpat_apply_K_dev: NULL argument");
    const int Rp = round_rhs(R);
    if (R < 1 || Rp < 0) return fail(QPAT_EINVAL, "qpat_apply_K_dev: R must be in [1, 16]");
    if (precision < 0 || precision > 3) return fail(QPAT_EINVAL, "qpat_apply_K_dev: mode must be in [0, 3]");
    DeviceGuard dg(M->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t N = M->h.N;
    cudaError_t e = cudaSuccess;
    double* kl = M->ws.get<double>("ak.k", N, s, &e);
    double* ml = M->ws.get<double>("ak.m", N, s, &e);
    double* xl = M->ws.get<double>("ak.x", N * Rp, s, &e);
    double* yl = M->ws.get<double>("ak.y", N * Rp, s, &e);
    if (e != cudaSuccess) return cuda_fail(e, "workspace");
    // x, y are N x R node-major in caller order
    if ((e = launch_to_lib<double, double>(M->d, 1, 1, kappa, kl, s)) != cudaSuccess) return cuda_fail(e, "to_lib");
    if ((e = launch_to_lib<double, double>(M->d, 1, 1, mu, ml, s)) != cudaSuccess) return cuda_fail(e, "to_lib");
    if ((e = launch_nodemajor_to_lib(M->d, R, Rp, x, xl, s)) != cudaSuccess) return cuda_fail(e, "to_lib");
    if (precision >= 2) {
        OpState st;
        int rc = prepare_K(M, kl, ml, st, s, "akK");
        if (rc != QPAT_OK) return rc;
        if (precision == 2) {
            if ((e = launch_apply_csr<double>(M->d, 1, Rp, st.v64[0], nullptr, xl, yl, s)) != cudaSuccess)
                return cuda_fail(e, "apply_csr");
        } else {
            float* x32 = M->ws.get<float>("ak.x32", N * Rp, s, &e);
            float* y32 = M->ws.get<float>("ak.y32", N * Rp, s, &e);
            if (e != cudaSuccess) return cuda_fail(e, "workspace");
            launch_cast_d2f(N * Rp, xl, x32, s);
            if ((e = launch_apply_csr<float>(M->d, 1, Rp, st.v32[0], nullptr, x32, y32, s)) != cudaSuccess)
                return cuda_fail(e, "apply_csr32");
            if ((e = launch_cast_f2d(N * Rp, y32, yl, s)) != cudaSuccess) return cuda_fail(e, "cast");
        }
    } else if (precision == 0) {
        if ((e = launch_apply_K<double>(M->d, Rp, kl, ml, 1, 1.0, xl, yl, s)) != cudaSuccess)
            return cuda_fail(e, "apply_K");
    } else {
        float* k32 = M->ws.get<float>("ak.k32", N, s, &e);
        float* m32 = M->ws.get<float>("ak.m32", N, s, &e);
        float* x32 = M->ws.get<float>("ak.x32", N * Rp, s, &e);
        float* y32 = M->ws.get<float>("ak.y32", N * Rp, s, &e);
        if (e != cudaSuccess) return cuda_fail(e, "workspace");
        launch_cast_d2f(N, kl, k32, s);
        launch_cast_d2f(N, ml, m32, s);
        launch_cast_d2f(N * Rp, xl, x32, s);
        if ((e = launch_apply_K<float>(M->d, Rp, k32, m32, 1, 1.0f, x32, y32, s)) != cudaSuccess)
            return cuda_fail(e, "apply_K32");
        if ((e = launch_cast_f2d(N * Rp, y32, yl, s)) != cudaSuccess) return cuda_fail(e, "cast");
    }
    if ((e = launch_nodemajor_from_lib(M->d, R, Rp, yl, y, s)) != cudaSuccess) return cuda_fail(e, "from_lib");
    return QPAT_OK;
}

}  // extern "C"
