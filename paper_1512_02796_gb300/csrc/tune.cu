// Autotuner: picks the owned nodes per CTA patch (which sets the elements
// per CTA) and the FP32 inner operator form (matrix-free element apply or
// assembled values) for a mesh and an illumination count, by timing a fixed
// number of FP32 PCG iterations of each candidate on the GPU.
#include <cmath>
#include <vector>

#include "abi_internal.h"

using namespace qpat;

namespace {

// timing of `iters` FP32 PCG iterations with R right-hand sides (CUDA events)
int time_candidate(qpat_mesh_s* M, const double* kap_h, const double* mu_h, int R, int fp32_op, int iters,
                   double* us_per_iter) {
    const int64_t N = M->h.N;
    cudaStream_t s = M->stream;
    cudaError_t e = cudaSuccess;
    double* kl = M->ws.get<double>("tune.k", N, s, &e);
    double* ml = M->ws.get<double>("tune.m", N, s, &e);
    float* b32 = M->ws.get<float>("tune.b", N * R, s, &e);
    float* x32 = M->ws.get<float>("tune.x", N * R, s, &e);
    float* r32 = M->ws.get<float>("tune.r", N * R, s, &e);
    float* p0 = M->ws.get<float>("tune.p0", N * R, s, &e);
    float* p1 = M->ws.get<float>("tune.p1", N * R, s, &e);
    float* q = M->ws.get<float>("tune.q", N * R, s, &e);
    double* part = M->ws.get<double>("tune.part", pcg_partials_doubles(), s, &e);
    double* ctl = M->ws.get<double>("tune.ctl", 64, s, &e);
    if (e != cudaSuccess) return cuda_fail(e, "qpat_autotune: workspace");
    // coefficients in library order, and a smooth deterministic right-hand side
    std::vector<double> kh(N), mh(N);
    std::vector<float> bh(N * R);
    for (int64_t l = 0; l < N; ++l) {
        kh[l] = kap_h[M->h.perm[l]];
        mh[l] = mu_h[M->h.perm[l]];
        for (int r = 0; r < R; ++r) bh[l * R + r] = float(1.0 + 0.5 * std::sin(0.001 * double(l) + r));
    }
    if ((e = cudaMemcpyAsync(kl, kh.data(), N * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(ml, mh.data(), N * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b32, bh.data(), N * R * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "qpat_autotune: upload");
    OpState st;
    int rc = prepare_K(M, kl, ml, st, s, "tuneK");
    if (rc) return rc;
    PcgWork w{};
    w.b = b32;
    w.x = x32;
    w.r = r32;
    w.p0 = p0;
    w.p1 = p1;
    w.q = q;
    w.partials = part;
    w.bar = reinterpret_cast<unsigned*>(ctl);
    w.status = reinterpret_cast<int*>(ctl + 1);
    w.iters = reinterpret_cast<int*>(ctl + 2);
    w.stats = ctl + 8;
    OpParams<float> op{st.c1_32, st.c2_32, 0.f, 0.f, 0.f, 1, st.v32[0], nullptr};
    const int OP = fp32_op ? OP_CSR1 : OP_K;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    // warm-up, then the timed run; rtol 0 makes the run last exactly `iters`
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) cudaEventRecord(a, s);
        if ((e = launch_pcg<float>(M->d, OP, R, op, st.inv32, w, 0.0, iters, s, nullptr)) != cudaSuccess) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return cuda_fail(e, "qpat_autotune: pcg");
        }
        if (pass == 1) cudaEventRecord(b, s);
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "qpat_autotune: sync");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *us_per_iter = 1e3 * ms / iters;
    return QPAT_OK;
}

}  // namespace

extern "C" int qpat_autotune(const double* xyz, int64_t N, const int32_t* tets, int64_t E, const double* kappa,
                             const double* mu, int K, int iters, int* best_patch_nodes, int* best_fp32_operator,
                             double* us_per_iter, int* ncand) {
    if (!xyz || !tets || !kappa || !mu || !best_patch_nodes || !best_fp32_operator)
        return fail(QPAT_EINVAL, "qpat_autotune: NULL argument");
    const int R = round_rhs(K);
    if (K < 1 || R < 0) return fail(QPAT_EINVAL, "qpat_autotune: K must be in [1, 16]");
    if (iters < 1) iters = 30;
    // candidate patch sizes: 0 = the library default (balanced over 4 CTAs per SM)
    static const int cands[] = {0, 128, 256, 512, 1024};
    double best = INFINITY;
    int n = 0;
    for (int pn : cands) {
        qpat_mesh_t M = nullptr;
        int rc = pn == 0 ? qpat_mesh(xyz, N, tets, E, &M) : qpat_mesh_ex(xyz, N, tets, E, pn, &M);
        if (rc) return rc;
        for (int op = 0; op < 2; ++op) {
            double us = INFINITY;
            rc = time_candidate(M, kappa, mu, R, op, iters, &us);
            if (rc) {
                // a candidate whose staging does not fit is skipped
                (void)cudaGetLastError();
                us = INFINITY;
            }
            if (us_per_iter) us_per_iter[n] = us;
            ++n;
            if (us < best) {
                best = us;
                *best_patch_nodes = pn;
                *best_fp32_operator = op;
            }
        }
        qpat_mesh_free(M);
    }
    if (ncand) *ncand = n;
    if (!std::isfinite(best)) return fail(QPAT_ECUDA, "qpat_autotune: no candidate ran");
    return QPAT_OK;
}
