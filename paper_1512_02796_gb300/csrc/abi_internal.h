// Internal state behind the C ABI (mesh handle, workspace, solve drivers).
#pragma once

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "launch.h"

namespace qpat {

struct Workspace {
    std::map<std::string, std::pair<void*, size_t>> bufs;
    void* get_bytes(const std::string& name, size_t bytes, cudaStream_t s, cudaError_t* err);
    template <typename T>
    T* get(const std::string& name, size_t count, cudaStream_t s, cudaError_t* err) {
        cudaError_t e = cudaSuccess;
        T* p = static_cast<T*>(get_bytes(name, count * sizeof(T), s, &e));
        if (e != cudaSuccess) *err = e;
        return p;
    }
    void release();
};

struct SolveStats {
    int64_t pcg_iters = 0;
    int64_t solves = 0;
    int64_t refinements = 0;
    int64_t fp64_fallbacks = 0;     // mixed-precision solves redone in FP64
    int64_t launches = 0;
    int64_t rhs_iters = 0;          // sum over PCG launches of iterations x right-hand sides of the launch
};

struct OpState {
    int kind = OP_K;
    const double* c1_64 = nullptr;  // kappa (OP_K) or kappa_tilde (OP_PRIOR), library order
    const double* c2_64 = nullptr;  // mu or mu_tilde
    float* c1_32 = nullptr;
    float* c2_32 = nullptr;
    double* inv64 = nullptr;        // inverse diagonal (N, or N x 2 for the prior)
    float* inv32 = nullptr;
    double inv_T2 = 0, scale1 = 1, delta = 0;
    int prior_kind = 0;             // r(t) of the prior (prior_weight in fem.cuh)
    double prior_q = 1;
    int nv = 1;                     // assembled value sets (1: K, 2: prior blocks)
    double* gbound = nullptr;       // Gershgorin bound of D^-1 A over the value sets (1 double)
    double* v64[2] = {nullptr, nullptr};  // assembled FP64 values (sliced ELLPACK)
    float* v32[2] = {nullptr, nullptr};   // FP32 copy (K only)
    uint64_t stamp = 0;             // new for every preparation (keys values derived from the operator)
};

struct SolveOpts {
    int precision = 0;        // 0 FP64 PCG, 1 FP32 PCG + FP64 refinement
    double rtol = 1e-13;
    int maxit = 20000;
    double inner_rtol = 1e-4;
    int max_sweeps = 30;
    int fp32_assembled = 0;   // FP32 inner operator: 0 matrix-free elements, 1 assembled values
    int pcg_variant = 0;      // assembled operators: 0 (= 1) two reductions, 2 one reduction, 3 bulk-copy ring
    int mixed_restart = 0;    // precision 1: 0 reliable updates (keep the direction), 1 restart every sweep
    int poly_k = 0;           // patch-local Chebyshev degree of the K preconditioner (0 Jacobi)
    int poly_prior = 0;       // the same for M_delta
    long long spin_limit = 0; // grid-barrier polls before a timeout (0 = default)
    int multigrid = 0;        // 1: CG with the smoothed-aggregation V-cycle (FP64); 2: its K cycle in FP32
    int mg_degree = 1;        // Chebyshev degree of each smoothing
    double mg_ratio = 30.0;   // smoothing interval [hi / mg_ratio, hi] of D^-1 A
};

struct DeviceGuard {
    int prev = 0;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != prev) cudaSetDevice(prev);
    }
};

struct AmgState;  // smoothed-aggregation hierarchy of a mesh (amg.cu)

}  // namespace qpat

struct qpat_mesh_s {
    qpat::HostMesh h;
    qpat::MeshDev d{};
    qpat::MeshDev dp{};  // d with the stiffness-only pattern of the prior operators (psell)
    std::vector<void*> dev_allocs;
    int device = 0;
    cudaStream_t stream = nullptr;   // used by the host-pointer entry points
    double* host_scratch = nullptr;  // pinned, 256 doubles
    qpat::Workspace ws;
    qpat::SolveStats stats;
    // optional CUDA-event timing of every PCG launch (on the launching stream)
    int timing = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double pcg_ms = 0.0;
    qpat::AmgState* amg = nullptr;   // built on the first multigrid solve
    double mg_fine_ms = 0.0;         // with timing on: fine-level smoothing launches of the multigrid cycle
    int64_t mg_fine_launches = 0;
};

namespace qpat {

extern thread_local std::string g_err;
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);
int round_rhs(int K);

int upload_mesh(qpat_mesh_s* M);
int prepare_K(qpat_mesh_s* M, const double* kap_l, const double* mu_l, OpState& st, cudaStream_t s,
              const char* tag = "opK");
int prepare_prior(qpat_mesh_s* M, const double* kt_l, const double* mt_l, double T, int kind, double q,
                  double b_over_a, double delta,
                  OpState& st, cudaStream_t s);
// X0 (optional): initial guess; the solve then stops at the same absolute
// residual |B - A X| <= rtol |B| as from zero.
int solve(qpat_mesh_s* M, const OpState& st, const SolveOpts& so, int R, const double* B, double* X,
          cudaStream_t s, const double* X0 = nullptr);
cudaError_t launch_add(int64_t n, const double* a, double* y, cudaStream_t s);  // y += a
uint64_t next_op_stamp();
// CG with one smoothed-aggregation V-cycle per iteration as the
// preconditioner (amg.cu); X0 as in solve().  The hierarchy's patterns are
// built on the first call per mesh and matrix pattern, its values once per
// prepared operator.
int amg_solve(qpat_mesh_s* M, const OpState& st, const SolveOpts& so, int R, const double* B, double* X,
              cudaStream_t s, const double* X0 = nullptr);
// rows of each level of the hierarchy of the K (prior = 0) or prior pattern; returns the level count
int amg_levels(qpat_mesh_s* M, int prior, int64_t* rows, int max_levels);
void amg_release(qpat_mesh_s* M);
SolveOpts solve_opts(const qpat_params* prm);

// node-major caller layout (x[c*R + r], r < R) <-> library N x Rp (zero padding)
cudaError_t launch_nodemajor_to_lib(const MeshDev& m, int R, int Rp, const double* in, double* out, cudaStream_t s);
cudaError_t launch_nodemajor_from_lib(const MeshDev& m, int R, int Rp, const double* in, double* out,
                                      cudaStream_t s);
cudaError_t launch_cast_f2d(int64_t n, const float* in, double* out, cudaStream_t s);

void k_mul_launch(int64_t n, const double* a, const double* b, double* out, cudaStream_t s);
void k_exp_scale_launch(int64_t n, double c0, const double* u, double* out, cudaStream_t s);
void k_rowscale_launch(int64_t N, int R, const double* d, const double* x, double* out, cudaStream_t s);
void k_jv_out_launch(int64_t N, int R, const double* mu, const double* b, const double* x, const double* phi,
                     const double* w, double* out, cudaStream_t s);
void k_jt_out_launch(int64_t N, int R, const double* kappa, const double* mu, const double* y, const double* phi,
                     const double* tw, double* ok, double* om, cudaStream_t s);

// Linearisation state on the device (library order): the coefficients,
// the forward solutions and the K operator (recon.cu and ops.cu).
struct LinState {
    int K = 0, R = 0;
    double* kap = nullptr;   // N
    double* mu = nullptr;    // N
    double* phi = nullptr;   // N x R
    double* w = nullptr;     // N x R whitening (nullptr = 1)
    OpState opK;
};

// J s and J^T t on library-order device data (ops.cu).
int jvp_lib(qpat_mesh_s* M, const SolveOpts& so, LinState& L, const double* s1, const double* s2, double* out,
            cudaStream_t s);
int vjp_lib(qpat_mesh_s* M, const SolveOpts& so, LinState& L, const double* t, double* o1, double* o2,
            cudaStream_t s);
int forward_lib(qpat_mesh_s* M, const SolveOpts& so, LinState& L, const double* flux_dev, cudaStream_t s,
                const double* x0 = nullptr);

}  // namespace qpat

extern "C" int qpat_mesh_stats(qpat_mesh_t M, int64_t* out4);
extern "C" int qpat_mesh_reset_stats(qpat_mesh_t M);
