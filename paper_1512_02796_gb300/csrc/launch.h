// Host-side launchers of the CUDA kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "fem.cuh"
#include "qpat_internal.h"

namespace qpat {

// ---------------------------------------------------------------- kernels.cu
// y = sign * (S(c1) + M(c2) + robin * B) x for R RHS, library order, N x R node-major.
template <typename T>
cudaError_t launch_apply_K(const MeshDev& m, int R, const T* c1, const T* c2, int robin, T sign,
                           const T* x, T* y, cudaStream_t s);
// y = (blkdiag(M(u1), scale1 M(u2)) + delta I) x, x and y N x 2 node-major;
// kind, q select the prior's r(t) (prior_weight in fem.cuh).
template <typename T>
cudaError_t launch_apply_prior(const MeshDev& m, const T* u1, const T* u2, T inv_T2, int kind, T q, T scale1,
                               T delta, const T* x, T* y, cudaStream_t s);
// inverse diagonal of K(kappa, mu) (N) and of M_delta (N x 2), computed in FP64.
cudaError_t launch_invdiag_K(const MeshDev& m, const double* kappa, const double* mu, double* inv64,
                             float* inv32, cudaStream_t s);
cudaError_t launch_invdiag_prior(const MeshDev& m, const double* u1, const double* u2, double inv_T2, int kind,
                                 double q, double scale1, double delta, double* inv64, float* inv32,
                                 cudaStream_t s);
// Assembly of K (FP64 values in the sliced-ELLPACK pattern; val must hold
// m.sell_entries) and of the two prior blocks with delta on the diagonal;
// both also write the inverse diagonal (FP64 and, if not null, FP32).
// gbound (optional, one double): receives max over rows and value sets of
// sum_j |a_ij| / a_ii, a Gershgorin bound of the spectrum of D^-1 A (and of
// D^-1 A_pp for every principal block A_pp).
cudaError_t launch_assemble_K(const MeshDev& m, const double* kappa, const double* mu, double* val, double* inv64,
                              float* inv32, cudaStream_t s, double* gbound = nullptr);
cudaError_t launch_assemble_prior(const MeshDev& m, const double* u1, const double* u2, double inv_T2, int kind,
                                  double q, double scale1, double delta, double* val0, double* val1, double* inv64,
                                  float* inv32, cudaStream_t s, double* gbound = nullptr);
cudaError_t launch_cast_vals(int64_t n, const double* in, float* out, cudaStream_t s);
// y = A x with an assembled operator (NV = 1: one value set for R RHS; NV = 2: the prior, R = 2)
template <typename T>
cudaError_t launch_apply_csr(const MeshDev& m, int NV, int R, const T* v0, const T* v1, const T* x, T* y,
                             cudaStream_t s);
// y (N x 2) = [ -sum_k G1-transpose-type term ; -sum_k M(phi_k) z_k ] (see kernels.cu)
template <typename T>
cudaError_t launch_vjp_accum(const MeshDev& m, int K, const T* phi, const T* z, T* y, cudaStream_t s);
// f (N x R node-major, library order, column k < K) += 2 Phi_F |F| / 3 at the
// vertices of every face (flux: K x F canonical order); f must be zeroed.
cudaError_t launch_load(const MeshDev& m, int K, int R, const double* flux, double* f, cudaStream_t s);

// layout helpers: caller K x N rows  <->  library N x R node-major
template <typename Tin, typename Tout>
cudaError_t launch_to_lib(const MeshDev& m, int K, int R, const Tin* in, Tout* out, cudaStream_t s);
template <typename Tin, typename Tout>
cudaError_t launch_from_lib(const MeshDev& m, int K, int R, const Tin* in, Tout* out, cudaStream_t s);

// per-RHS dot products of N x R node-major arrays, out[r] (double, device)
template <typename T>
cudaError_t launch_dots(int64_t n, int R, const T* a, const T* b, double* partial, double* out, cudaStream_t s);

// elementwise helpers (see kernels.cu for the formulas)
cudaError_t launch_cast_d2f_scaled(int64_t n, int R, const double* in, const double* scale, float* out,
                                   cudaStream_t s);
cudaError_t launch_axpy_f2d_scaled(int64_t n, int R, const float* d, const double* scale, double* x,
                                   cudaStream_t s);
cudaError_t launch_sub(int64_t n, const double* a, const double* b, double* out, cudaStream_t s);
cudaError_t launch_cast_d2f(int64_t n, const double* in, float* out, cudaStream_t s);

// ---------------------------------------------------------------- pcg.cu
// largest degree of the patch-local Chebyshev preconditioner (see pcg.cu)
constexpr int kMaxPolyDegree = 8;

// Bounds of the persistent PCG kernels' grid reductions: at most kMaxGrid
// CTAs, each contributing kMaxNS doubles (3 quantities x 16 RHS).  The
// partials buffer holds 2 x kMaxGrid x kMaxNS + 2 x kMaxNS doubles
// (pcg_partials_doubles).
constexpr int kMaxGrid = 152 * 8;
constexpr int kMaxNS = 48;
// Default bound of a grid-barrier wait: polls of ~32 ns sleep (about 2 s).
constexpr long long kDefaultSpinLimit = 40000000LL;

struct PcgWork {
    void* b;  // N x R (T)
    void* x;
    void* r;
    void* p0;
    void* p1;
    void* q;
    void* z = nullptr;  // optional N x R: D^-1 r kept by the owner (saves a multiply per halo node)
    // optional resume state of the two-reduction kernel (reliable updates):
    // resume_gamma (R, NULL = fresh start), rz_state (R), pbuf (1); see pcg.cu
    const double* resume_gamma = nullptr;
    double* rz_state = nullptr;
    int* pbuf = nullptr;
    // extra vectors of the single-reduction variant (see pcg.cu)
    void* r1 = nullptr;
    void* s0 = nullptr;
    void* s1 = nullptr;
    void* w1 = nullptr;
    // patch-local Chebyshev preconditioner (two-reduction kernel on assembled
    // operators, needs z): degree 0 = Jacobi; poly_hi = device pointer to an
    // upper bound of the spectrum of D^-1 A
    int poly_deg = 0;
    const double* poly_hi = nullptr;
    double* partials;   // 2 x max_grid x 3R
    unsigned* bar;      // 2
    int* status;        // 1
    int* iters;         // 1
    double* stats;      // 2R: final r.r, b.b
    long long spin_limit = 0;  // grid-barrier polls before QPAT_ETIMEOUT (0 = default, about 2 s)
    int force_narrow = 0;      // 1: the plain two-reduction kernel only (no wide or occupancy-bounded form)
};

// Persistent fused Jacobi-PCG on R right-hand sides (see pcg.cu).  b is
// read from w.b; the solution is left in w.x.  Asynchronous.
template <typename T>
cudaError_t launch_pcg(const MeshDev& m, int OP, int R, const OpParams<T>& op, const T* invdiag,
                       const PcgWork& w, double rtol, int maxit, cudaStream_t s, int* grid_used);
// Single-reduction (Chronopoulos-Gear) PCG for the assembled operators
// (OP_CSR1 / OP_CSR2): one grid barrier per iteration; needs w.r1, s0, s1, w1.
template <typename T>
cudaError_t launch_pcg1(const MeshDev& m, int OP, int R, const OpParams<T>& op, const T* invdiag,
                        const PcgWork& w, double rtol, int maxit, cudaStream_t s, int* grid_used);

// Two-reduction PCG on the assembled operators with the operator streamed
// through a shared-memory ring by bulk copies (see pcg.cu).  Returns
// cudaErrorNotSupported, launching nothing, when no ring of >= 2 slots fits
// beside the staged vector at the wanted occupancy.
template <typename T>
cudaError_t launch_pcg_ring(const MeshDev& m, int OP, int R, const OpParams<T>& op, const T* invdiag,
                            const PcgWork& w, double rtol, int maxit, cudaStream_t s, int* grid_used);

// Many independent FP64 assembled-K solves (different meshes) in one
// cooperative launch; see k_pcg_batch in pcg.cu.
struct PcgBatchProblem {
    MeshDev m;
    const double* vals;     // assembled K values
    const double* invdiag;  // N
    PcgWork w;              // b, x, r, p0, p1, q, partials, bar, status, iters, stats
    double rtol;
    int maxit;
};
struct PcgBatchPlan {
    void* dev_args = nullptr;
    int* dev_cta_begin = nullptr;
    int R = 0, nprob = 0, grid = 0;
    size_t smem = 0;
    bool poly = false;  // patch-local Chebyshev preconditioner (every problem has z, poly_deg, poly_hi)
    std::vector<int> cta_count;
};
cudaError_t pcg_batch_prepare(int R, const std::vector<PcgBatchProblem>& probs, PcgBatchPlan& plan);
cudaError_t pcg_batch_launch(const PcgBatchPlan& plan, cudaStream_t s);
void pcg_batch_release(PcgBatchPlan& plan);

// Shared-memory fit of the PCG kernel (launch_pcg) and of k_apply_csr for R
// right-hand sides on this mesh's patches (false: split the RHS).
template <typename T>
bool pcg_fits(const MeshDev& m, int OP, int R, int deg);
template <typename T>
bool apply_csr_fits(const MeshDev& m, int R);
int pcg_max_grid();            // upper bound of the cooperative grid
size_t pcg_partials_doubles();  // size of PcgWork::partials (per-CTA partials + totals)

}  // namespace qpat
