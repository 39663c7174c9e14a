// Algorithm 1 on the device: background fit, mu_tilde initialisation,
// step 0 (kappa-only sweep, Sec. 5), then linearisation + lagged
// diffusivity + priorconditioned LSQR (Eqs. (21)-(22)) + acceptance.
//
// LSQR runs in beta-space with only M_delta^-1 applied, once per round:
//   beta u = A v - alpha u,  p = A^T u - beta q,  z = M_delta^-1 p,
//   alpha = sqrt(p . z),  v = z / alpha,  q = p / alpha,
// followed by the plane rotation of the bidiagonal QR factor.  All vectors
// and the recurrence scalars stay in device memory in FP64; the host reads
// only the residual estimate phibar once per round for the stopping rule.
// beta-space vectors are stored node-interleaved (N x 2: kappa_tilde,
// mu_tilde), the layout of the two-block prior solve.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <stdexcept>
#include <string>
#include <vector>

#include "abi_internal.h"

namespace qpat {

namespace {

int gridn(int64_t n) {
    int64_t g = (n + 255) / 256;
    return int(std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16)));
}

#define GS(n) gridn(n), 256, 0, s
#define FOR_I(n) for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < (n); i += int64_t(gridDim.x) * blockDim.x)

enum { S_ALPHA = 0, S_BETA, S_RHOBAR, S_PHIBAR, S_RHO, S_C, S_S, S_THETA, S_PHI, S_T0, S_T1, S_T2, S_T3,
       S_COUNT = 16 };

// A Golub-Kahan direction whose norm falls below this fraction of the norm of
// the product that made it counts as zero: the bidiagonalisation has
// exhausted the Krylov space, the last rotation completes the exact
// least-squares solution and LSQR stops (the oracle uses the same rule).
constexpr double kBreakdown = 1e-12;

// Full reorthogonalisation (qpat_params.lsqr_reorth): projections against
// the stored bases, two passes of classical Gram-Schmidt.  Partial dot
// products over kChunks slices of each stored vector, then a fixed-order sum
// per vector, so the coefficients are the same from run to run.
constexpr int kChunks = 64;

// part[j * kChunks + c] = sum over slice c of B_j . x   (B_j = B + j * n)
__global__ void k_mdot_partial(int64_t n, const double* __restrict__ B, const double* __restrict__ x,
                               double* __restrict__ part) {
    const int c = blockIdx.x, j = blockIdx.y;
    const int64_t len = (n + kChunks - 1) / kChunks;
    const int64_t b = int64_t(c) * len, e = b + len < n ? b + len : n;
    const double* Bj = B + int64_t(j) * n;
    double a = 0.0;
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) a += Bj[i] * x[i];
    __shared__ double sh[256 / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += sh[w];
        part[j * kChunks + c] = t;
    }
}

// coef[j] = sum_c part[j * kChunks + c], one warp per stored vector
__global__ void k_mdot_final(int m, const double* __restrict__ part, double* __restrict__ coef) {
    const int j = blockIdx.x;
    if (j >= m) return;
    double a = 0.0;
    for (int c = threadIdx.x; c < kChunks; c += 32) a += part[j * kChunks + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (threadIdx.x == 0) coef[j] = a;
}

// y -= sum_j coef[j] C_j   (C_j = C + j * n), j = 0 .. m-1 in order
__global__ void k_msub(int64_t n, int m, const double* __restrict__ C, const double* __restrict__ coef,
                       double* __restrict__ y) {
    FOR_I(n) {
        double a = y[i];
        for (int j = 0; j < m; ++j) a -= coef[j] * C[int64_t(j) * n + i];
        y[i] = a;
    }
}

__global__ void k_set_scalar(double* S, int idx, double v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) S[idx] = v;
}

__global__ void k_fill(int64_t n, double v, double* out) { FOR_I(n) out[i] = v; }

// out = c0 exp(u[2l + blk])  (coefficient from a beta block)
__global__ void k_coef_from_beta(int64_t N, int blk, double c0, const double* beta, double* out) {
    FOR_I(N) out[i] = c0 * exp(beta[2 * i + blk]);
}

// mu_tilde_init = log(mu_init / mu0), mu_init = mean_k chi/phi0 (Algorithm 1 with
// Sec. 4's average); where that mean is not positive (phi0 may undershoot to
// <= 0 far from the sources) mu_init = mu0, then mu_init is clipped to
// [mu0 / 10, 10 mu0].
__global__ void k_mu_init(int64_t N, int K, int R, const double* chi, const double* phi0, double mu0, double* beta) {
    FOR_I(N) {
        double a = 0.0;
        for (int r = 0; r < K; ++r) a += chi[i * R + r] / phi0[i * R + r];
        a /= K;
        if (!(a > 0.0)) a = mu0;
        a = fmin(fmax(a, 0.1 * mu0), 10.0 * mu0);
        beta[2 * i] = 0.0;
        beta[2 * i + 1] = log(a / mu0);
    }
}

// out = w o (chi - mu o phi [+ jb])   (whitened data residual / y-tilde)
__global__ void k_wresid(int64_t N, int R, const double* w, const double* chi, const double* mu, const double* phi,
                         const double* jb, double* out) {
    FOR_I(N * R) {
        const int64_t l = i / R;
        double v = chi[i] - mu[l] * phi[i];
        if (jb) v += jb[i];
        out[i] = w[i] * v;
    }
}

__global__ void k_unpack_beta(int64_t N, const double* v, int kappa_only, double* s1, double* s2) {
    FOR_I(N) {
        s1[i] = v[2 * i];
        s2[i] = kappa_only ? 0.0 : v[2 * i + 1];
    }
}

__global__ void k_scal_set(double* S, int dst, int src, int op) {
    // op 0: S[dst] = sqrt(max(S[src], 0))
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (op == 0) S[dst] = sqrt(fmax(S[src], 0.0));
    }
}

// u = (Av - alpha u) / beta  in two passes: first uh = Av - alpha u
__global__ void k_uh(int64_t n, const double* Av, const double* S, double* u, int first) {
    const double a = first ? 0.0 : S[S_ALPHA];
    FOR_I(n) u[i] = Av[i] - a * u[i];
}

__global__ void k_scale_inv(int64_t n, const double* S, int idx, double* x) {
    const double b = S[idx];
    const double inv = b > 0.0 ? 1.0 / b : 0.0;
    FOR_I(n) x[i] *= inv;
}

// p = [o1, o2] - beta q (packed), the mu block zeroed in the kappa-only sweep
__global__ void k_p_update(int64_t N, const double* o1, const double* o2, const double* q, const double* S,
                           int first, int kappa_only, double* p) {
    const double b = first ? 0.0 : S[S_BETA];
    FOR_I(N) {
        p[2 * i] = o1[i] - b * q[2 * i];
        p[2 * i + 1] = kappa_only ? 0.0 : o2[i] - b * q[2 * i + 1];
    }
}

// v = z / alpha, q = p / alpha ; on the first round also w_d = v, x = 0.
// alpha = 0 (breakdown) leaves v and q as they are.
__global__ void k_vq(int64_t n, const double* z, const double* p, const double* S, double* v, double* q, int first,
                     double* wd, double* x) {
    const double a = S[S_ALPHA];
    if (!(a > 0.0)) return;
    const double inv = 1.0 / a;
    FOR_I(n) {
        const double vi = z[i] * inv;
        v[i] = vi;
        q[i] = p[i] * inv;
        if (first) {
            wd[i] = vi;
            x[i] = 0.0;
        }
    }
}

__global__ void k_lsqr_init_scalars(double* S, double* hist) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        S[S_PHIBAR] = S[S_BETA];
        S[S_RHOBAR] = S[S_ALPHA];
        hist[0] = S[S_PHIBAR];
    }
}

// plane rotation of LSQR (Paige-Saunders), FP64 on the device
__global__ void k_givens(double* S, double* hist, int m) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double rhobar = S[S_RHOBAR], beta = S[S_BETA], alpha = S[S_ALPHA], phibar = S[S_PHIBAR];
        const double rho = hypot(rhobar, beta);
        const double c = rho > 0 ? rhobar / rho : 1.0;
        const double sn = rho > 0 ? beta / rho : 0.0;
        S[S_RHO] = rho;
        S[S_C] = c;
        S[S_S] = sn;
        S[S_THETA] = sn * alpha;
        S[S_RHOBAR] = -c * alpha;
        S[S_PHI] = c * phibar;
        S[S_PHIBAR] = sn * phibar;
        hist[m] = sn * phibar;
    }
}

// x += (phi/rho) w_d ; w_d = v - (theta/rho) w_d
__global__ void k_xw(int64_t n, const double* S, const double* v, double* x, double* wd) {
    const double rho = S[S_RHO];
    const double a = rho > 0 ? S[S_PHI] / rho : 0.0, b = rho > 0 ? S[S_THETA] / rho : 0.0;
    FOR_I(n) {
        const double w = wd[i];
        x[i] += a * w;
        wd[i] = v[i] - b * w;
    }
}

// beta_new = beta_old + x (kappa block only when kappa_only)
__global__ void k_halve(int64_t n, double* x) { FOR_I(n) x[i] *= 0.5; }

// out = beta + t (beta_new - beta) over the 2N entries (shortened step)
__global__ void k_beta_step(int64_t n, double t, const double* beta, const double* beta_new, double* out) {
    FOR_I(n) out[i] = beta[i] + (beta_new[i] - beta[i]) * t;
}

// beta (interleaved per node) from its two blocks
__global__ void k_pack_beta(int64_t N, const double* s1, const double* s2, double* beta) {
    FOR_I(N) {
        beta[2 * i] = s1[i];
        beta[2 * i + 1] = s2[i];
    }
}

__global__ void k_add_beta(int64_t N, const double* x, int kappa_only, double* beta) {
    FOR_I(N) {
        beta[2 * i] += x[2 * i];
        if (!kappa_only) beta[2 * i + 1] += x[2 * i + 1];
    }
}

__global__ void k_ratio_rows(int64_t N, int R, const double* w, double* out) { FOR_I(N * R) out[i] = w[i]; }

__global__ void k_inv_sigma(int64_t N, int K, int R, const double* sig_lib, double* w) {
    FOR_I(N * R) {
        const int r = int(i % R);
        w[i] = r < K ? 1.0 / sig_lib[i] : 0.0;
    }
}

struct Recon {
    qpat_mesh_s* M;
    cudaStream_t s;
    SolveOpts so;
    int K, R;
    int64_t N;
    double* chi;    // N x R
    double* w;      // N x R (0 on padded columns)
    double* flux;   // K x F
    double* S;      // scalars
    double* hist;   // phibar history (max_lsqr + 1)
    double* dpart;
    double* tmpR;   // N x R
    std::string err;

    double* buf(const char* name, size_t n) {
        cudaError_t e = cudaSuccess;
        double* p = M->ws.get<double>(std::string("rc.") + name, n, s, &e);
        if (e != cudaSuccess) throw std::runtime_error(std::string("workspace ") + name);
        return p;
    }
    void ck(cudaError_t e, const char* where) {
        if (e != cudaSuccess) throw std::runtime_error(std::string(where) + ": " + cudaGetErrorString(e));
    }
    void ckq(int rc) {
        if (rc != QPAT_OK) throw rc;
    }
    double dot(int64_t n, const double* a, const double* b) {
        ck(launch_dots<double>(n, 1, a, b, dpart, S + S_T0, s), "dot");
        double h = 0;
        ck(cudaMemcpyAsync(M->host_scratch, S + S_T0, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
        ck(cudaStreamSynchronize(s), "sync");
        h = M->host_scratch[0];
        return h;
    }
    // linearisation state at coefficients kap, mu (device, library order)
    void lin(LinState& L, double* kap, double* mu, double* phi, const char* tag) {
        L.K = K;
        L.R = R;
        L.kap = kap;
        L.mu = mu;
        L.phi = phi;
        L.w = w;
        ckq(prepare_K(M, kap, mu, L.opK, s, tag));
    }
    double residual(LinState& L) {
        qpat::note_launch(1);
        k_wresid<<<GS(N * R)>>>(N, R, w, chi, L.mu, L.phi, nullptr, tmpR);
        return std::sqrt(dot(N * R, tmpR, tmpR));
    }
};

// One priorconditioned LSQR sweep (oracle: lsqr_prior).  b: N x R data
// vector; x: N x 2 result.  Returns rounds run.  With prm.lsqr_reorth the
// u's (N x R) and the v's and q = M_delta v (N x 2) are kept and every new
// u-hat and p is projected off them (two classical Gram-Schmidt passes).
// A direction that vanishes against the product that made it (kBreakdown)
// ends the sweep after its last rotation, as in the oracle.
int lsqr(Recon& rc, LinState& L, const OpState& P, const double* b, int kappa_only, const qpat_params& prm,
         double* x, std::vector<double>& hist_out) {
    const int64_t N = rc.N, R = rc.R;
    cudaStream_t s = rc.s;
    double* u = rc.buf("u", N * R);
    double* Av = rc.buf("Av", N * R);
    double* v = rc.buf("v", 2 * N);
    double* q = rc.buf("q", 2 * N);
    double* p = rc.buf("p", 2 * N);
    double* z = rc.buf("z", 2 * N);
    double* wd = rc.buf("wd", 2 * N);
    double* s1 = rc.buf("s1", N);
    double* s2 = rc.buf("s2", N);
    double* o1 = rc.buf("o1", N);
    double* o2 = rc.buf("o2", N);
    double* S = rc.S;
    double* hs = rc.M->host_scratch;
    const int maxit = std::max(0, prm.max_lsqr);
    const bool reorth = prm.lsqr_reorth != 0;
    const int64_t nu = N * R, nv = 2 * N;
    double *Ub = nullptr, *Vb = nullptr, *Qb = nullptr, *cf = nullptr, *cpart = nullptr;
    if (reorth) {
        Ub = rc.buf("Ub", size_t(nu) * (maxit + 1));
        Vb = rc.buf("Vb", size_t(nv) * (maxit + 1));
        Qb = rc.buf("Qb", size_t(nv) * (maxit + 1));
        cf = rc.buf("cf", maxit + 1);
        cpart = rc.buf("cpart", size_t(maxit + 1) * kChunks);
    }
    // y -= Bsub (Bdot^T y) over the first m stored vectors, twice
    auto project = [&](double* y, const double* Bdot, const double* Bsub, int64_t n, int m) {
        for (int pass = 0; pass < 2; ++pass) {
            qpat::note_launch(3);
            k_mdot_partial<<<dim3(kChunks, m), 256, 0, s>>>(n, Bdot, y, cpart);
            k_mdot_final<<<m, 32, 0, s>>>(m, cpart, cf);
            k_msub<<<GS(n)>>>(n, m, Bsub, cf, y);
        }
    };
    auto store = [&](int j) {
        rc.ck(cudaMemcpyAsync(Ub + j * nu, u, nu * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
        rc.ck(cudaMemcpyAsync(Vb + j * nv, v, nv * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
        rc.ck(cudaMemcpyAsync(Qb + j * nv, q, nv * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    };
    // S[idx[k]] -> hs[k] (scalars the host needs for a decision)
    auto readS = [&](std::initializer_list<int> idx) {
        int k = 0;
        for (int i : idx) rc.ck(cudaMemcpyAsync(hs + k++, S + i, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
        rc.ck(cudaStreamSynchronize(s), "sync");
    };
    hist_out.assign(1, 0.0);
    // beta u = b
    rc.ck(cudaMemcpyAsync(u, b, N * R * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    const double bb = rc.dot(N * R, u, u);
    if (!(bb > 0.0)) {
        rc.ck(cudaMemsetAsync(x, 0, 2 * N * sizeof(double), s), "memset");
        return 0;
    }
    qpat::note_launch(1);
    k_scal_set<<<1, 32, 0, s>>>(S, S_BETA, S_T0, 0);
    qpat::note_launch(1);
    k_scale_inv<<<GS(N * R)>>>(N * R, S, S_BETA, u);
    // p = A^T u ; z = P^-1 p ; alpha ; v, q ; w_d = v ; x = 0
    rc.ckq(vjp_lib(rc.M, rc.so, L, u, o1, o2, s));
    qpat::note_launch(1);
    k_p_update<<<GS(N)>>>(N, o1, o2, q, S, 1, kappa_only, p);
    rc.ckq(solve(rc.M, P, rc.so, 2, p, z, s));
    rc.ck(launch_dots<double>(2 * N, 1, p, z, rc.dpart, S + S_T1, s), "dot");
    readS({S_T1});
    hist_out[0] = std::sqrt(bb);
    if (!(hs[0] > 0.0)) {
        rc.ck(cudaMemsetAsync(x, 0, 2 * N * sizeof(double), s), "memset");
        return 0;
    }
    qpat::note_launch(1);
    k_scal_set<<<1, 32, 0, s>>>(S, S_ALPHA, S_T1, 0);
    qpat::note_launch(1);
    k_vq<<<GS(2 * N)>>>(2 * N, z, p, S, v, q, 1, wd, x);
    qpat::note_launch(1);
    k_lsqr_init_scalars<<<1, 32, 0, s>>>(S, rc.hist);
    if (reorth) store(0);
    int m = 0;
    while (m < maxit) {
        ++m;
        bool done = false;
        // u = (A v - alpha u) / beta
        qpat::note_launch(1);
        k_unpack_beta<<<GS(N)>>>(N, v, kappa_only, s1, s2);
        rc.ckq(jvp_lib(rc.M, rc.so, L, s1, s2, Av, s));
        qpat::note_launch(1);
        k_uh<<<GS(N * R)>>>(N * R, Av, S, u, 0);
        if (reorth) project(u, Ub, Ub, nu, m);
        rc.ck(launch_dots<double>(N * R, 1, u, u, rc.dpart, S + S_T0, s), "dot");
        rc.ck(launch_dots<double>(N * R, 1, Av, Av, rc.dpart, S + S_T2, s), "dot");
        readS({S_T0, S_T2});
        if (hs[0] <= kBreakdown * kBreakdown * hs[1]) {
            done = true;
            qpat::note_launch(2);
            k_set_scalar<<<1, 32, 0, s>>>(S, S_BETA, 0.0);
            k_set_scalar<<<1, 32, 0, s>>>(S, S_ALPHA, 0.0);
        } else {
            qpat::note_launch(1);
            k_scal_set<<<1, 32, 0, s>>>(S, S_BETA, S_T0, 0);
            qpat::note_launch(1);
            k_scale_inv<<<GS(N * R)>>>(N * R, S, S_BETA, u);
            // p = A^T u - beta q ; z = P^-1 p ; alpha = sqrt(p.z) ; v = z/alpha ; q = p/alpha
            rc.ckq(vjp_lib(rc.M, rc.so, L, u, o1, o2, s));
            rc.ck(launch_dots<double>(N, 1, o1, o1, rc.dpart, S + S_T2, s), "dot");
            if (!kappa_only) rc.ck(launch_dots<double>(N, 1, o2, o2, rc.dpart, S + S_T3, s), "dot");
            qpat::note_launch(1);
            k_p_update<<<GS(N)>>>(N, o1, o2, q, S, 0, kappa_only, p);
            if (reorth) project(p, Vb, Qb, nv, m);
            rc.ck(launch_dots<double>(2 * N, 1, p, p, rc.dpart, S + S_T0, s), "dot");
            readS({S_T0, S_T2, S_T3});
            const double atu2 = hs[1] + (kappa_only ? 0.0 : hs[2]);   // |A^T u|^2
            if (hs[0] <= kBreakdown * kBreakdown * atu2) {
                done = true;
                qpat::note_launch(1);
                k_set_scalar<<<1, 32, 0, s>>>(S, S_ALPHA, 0.0);
            } else {
                rc.ckq(solve(rc.M, P, rc.so, 2, p, z, s));
                rc.ck(launch_dots<double>(2 * N, 1, p, z, rc.dpart, S + S_T1, s), "dot");
                qpat::note_launch(1);
                k_scal_set<<<1, 32, 0, s>>>(S, S_ALPHA, S_T1, 0);
                qpat::note_launch(1);
                k_vq<<<GS(2 * N)>>>(2 * N, z, p, S, v, q, 0, wd, x);
            }
        }
        if (reorth && !done) store(m);
        // rotation, then x and w_d
        qpat::note_launch(1);
        k_givens<<<1, 32, 0, s>>>(S, rc.hist, m);
        qpat::note_launch(1);
        k_xw<<<GS(2 * N)>>>(2 * N, S, v, x, wd);
        rc.ck(cudaMemcpyAsync(hs, S + S_PHIBAR, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
        rc.ck(cudaMemcpyAsync(hs + 1, S + S_ALPHA, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
        rc.ck(cudaStreamSynchronize(s), "sync");
        hist_out.push_back(hs[0]);
        if (done || !(hs[1] > 0.0)) break;
        if (!prm.fixed_counts && m > prm.m0) {
            const double r_m = 1.0 - hist_out[m] / hist_out[m - prm.m0];
            if (r_m <= prm.tau) break;
        }
    }
    return m;
}

}  // namespace

}  // namespace qpat

using namespace qpat;

// Algorithm 1.  beta_in (2N, caller order: kappa_tilde then mu_tilde) resumes
// a stopped run at step 1 with beta^(l) = beta_in after lin_done
// linearisations (the background constants must then be given); beta_out
// (optional) receives the final beta^(l).
static int reconstruct_impl(qpat_mesh_t M, const qpat_params* prm_in, int K, const double* flux_face,
                            const double* chi, const double* sigma, const double* kappa0_mu0, const double* beta_in,
                            int lin_done, double* kappa, double* mu, double* beta_out, qpat_report* rep) {
    if (!M || !flux_face || !chi || !sigma || !kappa || !mu) return fail(QPAT_EINVAL, "qpat_reconstruct: NULL argument");
    if (beta_in && (!kappa0_mu0 || lin_done < 1))
        return fail(QPAT_EINVAL, "qpat_reconstruct_ex: resuming needs kappa0_mu0 and lin_done >= 1");
    if (K < 1 || round_rhs(K) < 0) return fail(QPAT_EINVAL, "qpat_reconstruct: K must be in [1, 16]");
    qpat_params prm;
    qpat_default_params(&prm);
    if (prm_in) prm = *prm_in;
    if (prm.precision != 0 && prm.precision != 1) return fail(QPAT_EINVAL, "qpat_reconstruct: bad precision");
    if (prm.prior != 0 && prm.prior != 1) return fail(QPAT_EINVAL, "qpat_reconstruct: prior must be 0 or 1");
    if (prm.prior == 1 && !(prm.prior_q > 0.0 && prm.prior_q <= 2.0))
        return fail(QPAT_EINVAL, "qpat_reconstruct: prior_q must lie in (0, 2]");
    if (prm.max_lin < 1 || prm.max_lin > 32 || prm.max_lsqr < 0 || prm.m0 < 1)
        return fail(QPAT_EINVAL, "qpat_reconstruct: max_lin must be in [1, 32], max_lsqr >= 0, m0 >= 1");
    if (!(prm.T > 0) || !(prm.delta > 0) || !(prm.b_over_a > 0))
        return fail(QPAT_EINVAL, "qpat_reconstruct: T, delta, b/a must be positive");
    if (prm.step_halvings < 0 || prm.step_halvings > 16)
        return fail(QPAT_EINVAL, "qpat_reconstruct: step_halvings must lie in [0, 16]");
    if (prm.lsqr_reorth != 0 && prm.lsqr_reorth != 1)
        return fail(QPAT_EINVAL, "qpat_reconstruct: lsqr_reorth must be 0 or 1");
    if (prm.barrier_spin_limit < 0) return fail(QPAT_EINVAL, "qpat_reconstruct: barrier_spin_limit must be >= 0");
    {
        // the data model of Eq. (8): finite data, Gamma = diag(sigma^2) positive definite
        const int64_t n = int64_t(K) * M->h.N;
        for (int64_t i = 0; i < n; ++i) {
            if (!std::isfinite(chi[i])) return fail(QPAT_EINVAL, "qpat_reconstruct: chi must be finite");
            if (!(sigma[i] > 0.0) || !std::isfinite(sigma[i]))
                return fail(QPAT_EINVAL, "qpat_reconstruct: sigma must be positive and finite");
        }
        for (int64_t i = 0; i < int64_t(K) * M->h.F; ++i)
            if (!std::isfinite(flux_face[i])) return fail(QPAT_EINVAL, "qpat_reconstruct: flux must be finite");
    }
    DeviceGuard dg(M->device);
    const auto t0 = std::chrono::steady_clock::now();
    Recon rc{};
    rc.M = M;
    rc.s = M->stream;
    rc.so = solve_opts(&prm);
    rc.K = K;
    rc.R = round_rhs(K);
    rc.N = M->h.N;
    const int64_t N = rc.N, R = rc.R, F = M->h.F;
    cudaStream_t s = rc.s;
    const SolveStats st0 = M->stats;
    qpat_report report;
    std::memset(&report, 0, sizeof(report));
    try {
        rc.chi = rc.buf("chi", N * R);
        rc.w = rc.buf("w", N * R);
        rc.flux = rc.buf("flux", size_t(K) * F);
        rc.S = rc.buf("S", S_COUNT);
        rc.hist = rc.buf("hist", prm.max_lsqr + 2);
        rc.dpart = rc.buf("dpart", 608 * 16);
        rc.tmpR = rc.buf("tmpR", N * R);
        double* hchi = rc.buf("hchi", size_t(K) * N);
        double* hsig = rc.buf("hsig", size_t(K) * N);
        double* sig_l = rc.buf("sigl", N * R);
        rc.ck(cudaMemcpyAsync(rc.flux, flux_face, sizeof(double) * K * F, cudaMemcpyHostToDevice, s), "H2D");
        rc.ck(cudaMemcpyAsync(hchi, chi, sizeof(double) * K * N, cudaMemcpyHostToDevice, s), "H2D");
        rc.ck(cudaMemcpyAsync(hsig, sigma, sizeof(double) * K * N, cudaMemcpyHostToDevice, s), "H2D");
        rc.ck(launch_to_lib<double, double>(M->d, K, R, hchi, rc.chi, s), "to_lib");
        rc.ck(launch_to_lib<double, double>(M->d, K, R, hsig, sig_l, s), "to_lib");
        qpat::note_launch(1);
        k_inv_sigma<<<GS(N * R)>>>(N, K, R, sig_l, rc.w);

        double* kapA = rc.buf("kapA", N);
        double* muA = rc.buf("muA", N);
        double* phiA = rc.buf("phiA", N * R);
        double* kapB = rc.buf("kapB", N);
        double* muB = rc.buf("muB", N);
        double* phiB = rc.buf("phiB", N * R);
        double* beta = rc.buf("beta", 2 * N);
        double* betaN = rc.buf("betaN", 2 * N);
        double* xls = rc.buf("xls", 2 * N);
        double* jb = rc.buf("jb", N * R);
        double* ytil = rc.buf("ytil", N * R);
        double* s1 = rc.buf("bs1", N);
        double* s2 = rc.buf("bs2", N);
        LinState LA, LB;

        auto forward_const = [&](double k, double m, LinState& L, double* kp, double* mp, double* ph) {
            qpat::note_launch(1);
            k_fill<<<GS(N)>>>(N, k, kp);
            qpat::note_launch(1);
            k_fill<<<GS(N)>>>(N, m, mp);
            rc.lin(L, kp, mp, ph, "rKA");
            rc.ckq(forward_lib(M, rc.so, L, rc.flux, s));
            return rc.residual(L);
        };

        double* ktmp = rc.buf("ktv", N);
        double* mtmp = rc.buf("mtv", N);
        OpState P;
        std::vector<double> hist;
        // ---- (kappa_0, mu_0): given, or the reading of Algorithm 1's preamble
        double k0, m0;
        if (kappa0_mu0) {
            k0 = kappa0_mu0[0];
            m0 = kappa0_mu0[1];
            if (!(k0 > 0) || !(m0 > 0)) throw std::runtime_error("kappa0_mu0 must be positive");
        } else {
            const int G = std::max(2, prm.fit_grid);
            double best = INFINITY, ba = 0, bb = 0;
            for (int i = 0; i < G; ++i)
                for (int j = 0; j < G; ++j) {
                    const double a = std::log(0.05) + (std::log(2.0) - std::log(0.05)) * i / (G - 1);
                    const double b = std::log(1e-3) + (std::log(0.1) - std::log(1e-3)) * j / (G - 1);
                    const double r = forward_const(std::exp(a), std::exp(b), LA, kapA, muA, phiA);
                    if (r < best) {
                        best = r;
                        ba = a;
                        bb = b;
                    }
                }
            double* ja = rc.buf("ja", N * R);
            double* jbv = rc.buf("jbv", N * R);
            double* one = rc.buf("one", N);
            double* zero = rc.buf("zero", N);
            qpat::note_launch(1);
            k_fill<<<GS(N)>>>(N, 1.0, one);
            qpat::note_launch(1);
            k_fill<<<GS(N)>>>(N, 0.0, zero);
            for (int it = 0; it < prm.fit_gn_steps; ++it) {
                const double r0 = forward_const(std::exp(ba), std::exp(bb), LA, kapA, muA, phiA);
                rc.ckq(jvp_lib(M, rc.so, LA, one, zero, ja, s));
                rc.ckq(jvp_lib(M, rc.so, LA, zero, one, jbv, s));
                qpat::note_launch(1);
                k_wresid<<<GS(N * R)>>>(N, R, rc.w, rc.chi, LA.mu, LA.phi, nullptr, rc.tmpR);
                const double aa = rc.dot(N * R, ja, ja), ab = rc.dot(N * R, ja, jbv), bbv = rc.dot(N * R, jbv, jbv);
                const double ra = rc.dot(N * R, ja, rc.tmpR), rb = rc.dot(N * R, jbv, rc.tmpR);
                const double det = aa * bbv - ab * ab;
                if (!(std::fabs(det) > 0)) break;
                const double da = (bbv * ra - ab * rb) / det, db = (aa * rb - ab * ra) / det;
                double step = 1.0;
                bool acc = false;
                for (int hh = 0; hh < 6; ++hh) {
                    const double r1 =
                        forward_const(std::exp(ba + step * da), std::exp(bb + step * db), LA, kapA, muA, phiA);
                    if (r1 < r0) {
                        ba += step * da;
                        bb += step * db;
                        acc = true;
                        break;
                    }
                    step *= 0.5;
                }
                if (!acc) break;
            }
            k0 = std::exp(ba);
            m0 = std::exp(bb);
        }
        report.kappa0 = k0;
        report.mu0 = m0;

        if (beta_in) {
        // ---- resume: beta^(l) given, continue at step 1
        double* hb = rc.buf("hbeta", 2 * N);
        rc.ck(cudaMemcpyAsync(hb, beta_in, 2 * N * sizeof(double), cudaMemcpyHostToDevice, s), "H2D");
        rc.ck(launch_to_lib<double, double>(M->d, 1, 1, hb, ktmp, s), "to_lib");
        rc.ck(launch_to_lib<double, double>(M->d, 1, 1, hb + N, mtmp, s), "to_lib");
        qpat::note_launch(1);
        k_pack_beta<<<GS(N)>>>(N, ktmp, mtmp, beta);
        report.linearisations = lin_done;
        } else {
        // ---- initialisation: phi0 at the constants, mu_tilde_init, kappa_tilde_init = 0
        forward_const(k0, m0, LA, kapA, muA, phiA);
        qpat::note_launch(1);
        k_mu_init<<<GS(N)>>>(N, K, R, rc.chi, LA.phi, m0, beta);

        // ---- step 0: kappa-only LSQR with M_delta(kappa_tilde_init)
        qpat::note_launch(1);
        k_coef_from_beta<<<GS(N)>>>(N, 0, k0, beta, kapA);
        qpat::note_launch(1);
        k_coef_from_beta<<<GS(N)>>>(N, 1, m0, beta, muA);
        rc.lin(LA, kapA, muA, phiA, "rKA");
        rc.ckq(forward_lib(M, rc.so, LA, rc.flux, s));
        qpat::note_launch(1);
        k_wresid<<<GS(N * R)>>>(N, R, rc.w, rc.chi, LA.mu, LA.phi, nullptr, ytil);
        qpat::note_launch(1);
        k_unpack_beta<<<GS(N)>>>(N, beta, 0, ktmp, mtmp);
        rc.ckq(prepare_prior(M, ktmp, mtmp, prm.T, prm.prior, prm.prior_q, prm.b_over_a, prm.delta, P, s));
        int it0 = lsqr(rc, LA, P, ytil, 1, prm, xls, hist);
        if (prm.step_halvings > 0) {
            // option: keep the first of x, x/2, ... that lowers the residual at beta_init
            const double r_init = rc.residual(LA);
            double* binit = rc.buf("binit", 2 * N);
            double* bcand = rc.buf("bcand", 2 * N);
            rc.ck(cudaMemcpyAsync(binit, beta, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
            bool kept = false;
            for (int j = 0; j <= prm.step_halvings && !kept; ++j) {
                rc.ck(cudaMemcpyAsync(bcand, binit, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
                if (j > 0) {
                    qpat::note_launch(1);
                    k_halve<<<GS(2 * N)>>>(2 * N, xls);  // x / 2^j (exact: powers of two)
                }
                qpat::note_launch(1);
                k_add_beta<<<GS(N)>>>(N, xls, 1, bcand);
                qpat::note_launch(1);
                k_coef_from_beta<<<GS(N)>>>(N, 0, k0, bcand, kapB);
                qpat::note_launch(1);
                k_coef_from_beta<<<GS(N)>>>(N, 1, m0, bcand, muB);
                rc.lin(LB, kapB, muB, phiB, "rKB");
                rc.ckq(forward_lib(M, rc.so, LB, rc.flux, s));
                if (rc.residual(LB) < r_init) {
                    rc.ck(cudaMemcpyAsync(beta, bcand, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
                    kept = true;
                }
            }
        } else {
            qpat::note_launch(1);
            k_add_beta<<<GS(N)>>>(N, xls, 1, beta);
        }
        report.lsqr_iters[0] = it0;
        report.linearisations = 1;
        }

        // ---- h(beta^(0))
        qpat::note_launch(1);
        k_coef_from_beta<<<GS(N)>>>(N, 0, k0, beta, kapA);
        qpat::note_launch(1);
        k_coef_from_beta<<<GS(N)>>>(N, 1, m0, beta, muA);
        rc.lin(LA, kapA, muA, phiA, "rKA");
        rc.ckq(forward_lib(M, rc.so, LA, rc.flux, s));
        double r_cur = rc.residual(LA);
        report.residuals[0] = r_cur;
        int nres = 1;
        report.accepted_last = 1;
        LinState* cur = &LA;
        LinState* nxt = &LB;
        double *kapC = kapA, *muC = muA, *phiC = phiA, *kapN = kapB, *muN = muB, *phiN = phiB;
        const char* tagC = "rKA";
        const char* tagN = "rKB";

        while (report.linearisations < prm.max_lin) {
            // step 1: y-tilde = w o (chi - h + J beta)   (J unweighted here)
            qpat::note_launch(1);
            k_unpack_beta<<<GS(N)>>>(N, beta, 0, s1, s2);
            double* wsave = cur->w;
            cur->w = nullptr;
            rc.ckq(jvp_lib(M, rc.so, *cur, s1, s2, jb, s));
            cur->w = wsave;
            qpat::note_launch(1);
            k_wresid<<<GS(N * R)>>>(N, R, rc.w, rc.chi, cur->mu, cur->phi, jb, ytil);
            // step 2: M_delta from the current iterate
            qpat::note_launch(1);
            k_unpack_beta<<<GS(N)>>>(N, beta, 0, ktmp, mtmp);
            rc.ckq(prepare_prior(M, ktmp, mtmp, prm.T, prm.prior, prm.prior_q, prm.b_over_a, prm.delta, P, s));
            // step 3: LSQR from zero
            const int it = lsqr(rc, *cur, P, ytil, 0, prm, betaN, hist);
            report.lsqr_iters[report.linearisations] = it;
            report.linearisations += 1;
            // step 4: accept only if the nonlinear residual decreased (option:
            // first try the shorter steps beta + 2^-j (beta_new - beta))
            double r_new = INFINITY;
            for (int j = 0; j <= prm.step_halvings; ++j) {
                const double* cand = betaN;
                if (j > 0) {
                    double* bc = rc.buf("bstep", 2 * N);
                    qpat::note_launch(1);
                    k_beta_step<<<GS(2 * N)>>>(2 * N, std::ldexp(1.0, -j), beta, betaN, bc);
                    cand = bc;
                }
                qpat::note_launch(1);
                k_coef_from_beta<<<GS(N)>>>(N, 0, k0, cand, kapN);
                qpat::note_launch(1);
                k_coef_from_beta<<<GS(N)>>>(N, 1, m0, cand, muN);
                rc.lin(*nxt, kapN, muN, phiN, tagN);
                rc.ckq(forward_lib(M, rc.so, *nxt, rc.flux, s));
                r_new = rc.residual(*nxt);
                if (r_new < r_cur) {
                    if (j > 0)
                        rc.ck(cudaMemcpyAsync(betaN, cand, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, s),
                              "copy");
                    break;
                }
            }
            if (!(r_new < r_cur)) {
                report.accepted_last = 0;
                break;
            }
            rc.ck(cudaMemcpyAsync(beta, betaN, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
            std::swap(cur, nxt);
            std::swap(kapC, kapN);
            std::swap(muC, muN);
            std::swap(phiC, phiN);
            std::swap(tagC, tagN);
            r_cur = r_new;
            if (nres < 33) report.residuals[nres++] = r_cur;
        }
        // ---- output kappa = k0 exp(kt), mu = m0 exp(mt) in caller order
        qpat::note_launch(1);
        k_coef_from_beta<<<GS(N)>>>(N, 0, k0, beta, s1);
        qpat::note_launch(1);
        k_coef_from_beta<<<GS(N)>>>(N, 1, m0, beta, s2);
        double* outk = rc.buf("outk", N);
        double* outm = rc.buf("outm", N);
        rc.ck(launch_from_lib<double, double>(M->d, 1, 1, s1, outk, s), "from_lib");
        rc.ck(launch_from_lib<double, double>(M->d, 1, 1, s2, outm, s), "from_lib");
        rc.ck(cudaMemcpyAsync(kappa, outk, N * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
        rc.ck(cudaMemcpyAsync(mu, outm, N * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
        if (beta_out) {
            double* ob = rc.buf("outb", 2 * N);
            qpat::note_launch(1);
            k_unpack_beta<<<GS(N)>>>(N, beta, 0, s1, s2);
            rc.ck(launch_from_lib<double, double>(M->d, 1, 1, s1, ob, s), "from_lib");
            rc.ck(launch_from_lib<double, double>(M->d, 1, 1, s2, ob + N, s), "from_lib");
            rc.ck(cudaMemcpyAsync(beta_out, ob, 2 * N * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
        }
        rc.ck(cudaStreamSynchronize(s), "sync");
        (void)kapC;
        (void)muC;
        (void)phiC;
        (void)tagC;
    } catch (int code) {
        return code;
    } catch (const std::exception& ex) {
        return fail(QPAT_ECUDA, std::string("qpat_reconstruct: ") + ex.what());
    }
    report.pcg_iters = M->stats.pcg_iters - st0.pcg_iters;
    report.solves = M->stats.solves - st0.solves;
    report.refinements = M->stats.refinements - st0.refinements;
    report.ms_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = report;
    return QPAT_OK;
}

extern "C" int qpat_reconstruct(qpat_mesh_t M, const qpat_params* prm, int K, const double* flux_face,
                                const double* chi, const double* sigma, const double* kappa0_mu0, double* kappa,
                                double* mu, qpat_report* rep) {
    return reconstruct_impl(M, prm, K, flux_face, chi, sigma, kappa0_mu0, nullptr, 0, kappa, mu, nullptr, rep);
}

extern "C" int qpat_reconstruct_ex(qpat_mesh_t M, const qpat_params* prm, int K, const double* flux_face,
                                   const double* chi, const double* sigma, const double* kappa0_mu0,
                                   const double* beta_in, int lin_done, double* kappa, double* mu, double* beta_out,
                                   qpat_report* rep) {
    return reconstruct_impl(M, prm, K, flux_face, chi, sigma, kappa0_mu0, beta_in, lin_done, kappa, mu, beta_out,
                            rep);
}
