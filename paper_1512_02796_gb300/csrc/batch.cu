// Uneven batches: forward solves of many meshes of different sizes run as
// one cooperative launch (k_pcg_batch) and replayed as one CUDA graph.
//
// A batch owns, per problem, the caller-visible device buffers (kappa, mu,
// fluxes, phi) and the solver's work vectors.  The first qpat_batch_forward
// records the whole sequence -- per problem the layout change, the assembly
// of K, the load vector; then the single batched PCG launch; then the output
// layout change -- into a CUDA graph on the caller's stream; every later call
// replays that graph.  Illuminations per problem are padded to a common R.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "abi_internal.h"

struct qpat_batch_s {
    struct Prob {
        qpat_mesh_s* mesh = nullptr;
        int K = 0;
        double *kappa = nullptr, *mu = nullptr, *flux = nullptr, *phi = nullptr;   // caller layout
        double *kl = nullptr, *ml = nullptr, *vals = nullptr, *inv = nullptr;     // library layout
        double *f = nullptr, *x = nullptr, *r = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr;
        double *partials = nullptr, *ctl = nullptr;
        double *z = nullptr, *gb = nullptr;  // patch-local Chebyshev preconditioner
    };
    int device = 0;
    int R = 0;
    double rtol = 1e-13;
    int maxit = 20000;
    int poly_deg = 0;
    std::vector<Prob> probs;
    std::vector<void*> allocs;
    qpat::PcgBatchPlan plan;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

using namespace qpat;

namespace {

int batch_alloc(qpat_batch_s* B, double** p, size_t n) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(n, 1) * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e, "qpat_batch_create: cudaMalloc");
    B->allocs.push_back(v);
    *p = static_cast<double*>(v);
    return cudaMemset(v, 0, std::max<size_t>(n, 1) * sizeof(double)) == cudaSuccess
               ? QPAT_OK
               : cuda_fail(cudaGetLastError(), "qpat_batch_create: memset");
}

void batch_release(qpat_batch_s* B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    pcg_batch_release(B->plan);
    for (void* p : B->allocs) cudaFree(p);
    B->allocs.clear();
}

// the recorded sequence (also valid eagerly)
int batch_sequence(qpat_batch_s* B, cudaStream_t s) {
    cudaError_t e;
    for (auto& P : B->probs) {
        const MeshDev& m = P.mesh->d;
        const int64_t N = m.N;
        if ((e = launch_to_lib<double, double>(m, 1, 1, P.kappa, P.kl, s)) != cudaSuccess ||
            (e = launch_to_lib<double, double>(m, 1, 1, P.mu, P.ml, s)) != cudaSuccess)
            return cuda_fail(e, "qpat_batch_forward: to_lib");
        if ((e = launch_assemble_K(m, P.kl, P.ml, P.vals, P.inv, nullptr, s, B->poly_deg > 0 ? P.gb : nullptr)) !=
            cudaSuccess)
            return cuda_fail(e, "qpat_batch_forward: assemble");
        if ((e = cudaMemsetAsync(P.f, 0, sizeof(double) * N * B->R, s)) != cudaSuccess)
            return cuda_fail(e, "qpat_batch_forward: memset");
        if ((e = launch_load(m, P.K, B->R, P.flux, P.f, s)) != cudaSuccess)
            return cuda_fail(e, "qpat_batch_forward: load");
        if ((e = cudaMemsetAsync(P.ctl, 0, sizeof(double) * 8, s)) != cudaSuccess)  // barrier, status, iterations
            return cuda_fail(e, "qpat_batch_forward: memset");
    }
    if ((e = pcg_batch_launch(B->plan, s)) != cudaSuccess) return cuda_fail(e, "qpat_batch_forward: batched pcg");
    for (auto& P : B->probs)
        if ((e = launch_from_lib<double, double>(P.mesh->d, P.K, B->R, P.x, P.phi, s)) != cudaSuccess)
            return cuda_fail(e, "qpat_batch_forward: from_lib");
    return QPAT_OK;
}

}  // namespace

extern "C" {

int qpat_batch_create(int nprob, const qpat_mesh_t* meshes, const int* K, const qpat_params* prm,
                      qpat_batch_t* out) {
    if (!out || !meshes || !K || nprob < 1) return fail(QPAT_EINVAL, "qpat_batch_create: bad arguments");
    *out = nullptr;
    int Kmax = 0;
    for (int j = 0; j < nprob; ++j) {
        if (!meshes[j]) return fail(QPAT_EINVAL, "qpat_batch_create: NULL mesh");
        if (K[j] < 1 || K[j] > 8) return fail(QPAT_EINVAL, "qpat_batch_create: K must be in [1, 8]");
        if (meshes[j]->device != meshes[0]->device) return fail(QPAT_EINVAL, "qpat_batch_create: meshes on two devices");
        Kmax = std::max(Kmax, K[j]);
    }
    auto* B = new qpat_batch_s();
    B->device = meshes[0]->device;
    B->R = round_rhs(Kmax);
    const SolveOpts so = solve_opts(prm);
    B->rtol = so.rtol;
    B->maxit = so.maxit;
    B->poly_deg = so.poly_k;
    DeviceGuard dg(B->device);
    std::vector<PcgBatchProblem> pp;
    int rc = QPAT_OK;
    for (int j = 0; j < nprob && rc == QPAT_OK; ++j) {
        qpat_batch_s::Prob P;
        P.mesh = meshes[j];
        P.K = K[j];
        const size_t N = P.mesh->h.N, F = P.mesh->h.F, R = B->R;
        if ((rc = batch_alloc(B, &P.kappa, N)) || (rc = batch_alloc(B, &P.mu, N)) ||
            (rc = batch_alloc(B, &P.flux, size_t(P.K) * F)) || (rc = batch_alloc(B, &P.phi, size_t(P.K) * N)) ||
            (rc = batch_alloc(B, &P.kl, N)) || (rc = batch_alloc(B, &P.ml, N)) ||
            (rc = batch_alloc(B, &P.vals, size_t(P.mesh->d.sell_entries))) || (rc = batch_alloc(B, &P.inv, N)) ||
            (rc = batch_alloc(B, &P.f, N * R)) || (rc = batch_alloc(B, &P.x, N * R)) ||
            (rc = batch_alloc(B, &P.r, N * R)) || (rc = batch_alloc(B, &P.p0, N * R)) ||
            (rc = batch_alloc(B, &P.p1, N * R)) || (rc = batch_alloc(B, &P.q, N * R)) ||
            (rc = batch_alloc(B, &P.partials, pcg_partials_doubles())) || (rc = batch_alloc(B, &P.ctl, 64)))
            break;
        if (B->poly_deg > 0 && ((rc = batch_alloc(B, &P.z, N * R)) || (rc = batch_alloc(B, &P.gb, 1)))) break;
        PcgBatchProblem q;
        q.m = P.mesh->d;
        q.vals = P.vals;
        q.invdiag = P.inv;
        q.w.b = P.f;
        q.w.x = P.x;
        q.w.r = P.r;
        q.w.p0 = P.p0;
        q.w.p1 = P.p1;
        q.w.q = P.q;
        q.w.partials = P.partials;
        q.w.bar = reinterpret_cast<unsigned*>(P.ctl);
        q.w.status = reinterpret_cast<int*>(P.ctl + 1);
        q.w.iters = reinterpret_cast<int*>(P.ctl + 2);
        q.w.stats = P.ctl + 8;
        q.w.z = P.z;
        q.w.poly_deg = B->poly_deg;
        q.w.poly_hi = P.gb;
        q.rtol = B->rtol;
        q.maxit = B->maxit;
        pp.push_back(q);
        B->probs.push_back(P);
    }
    if (rc == QPAT_OK) {
        cudaError_t e = pcg_batch_prepare(B->R, pp, B->plan);
        if (e != cudaSuccess) rc = cuda_fail(e, "qpat_batch_create: too many problems or patches too large");
    }
    if (rc != QPAT_OK) {
        batch_release(B);
        delete B;
        return rc;
    }
    *out = B;
    return QPAT_OK;
}

int qpat_batch_buffers(qpat_batch_t B, int j, double** kappa, double** mu, double** flux, double** phi) {
    if (!B || j < 0 || j >= int(B->probs.size())) return fail(QPAT_EINVAL, "qpat_batch_buffers: bad index");
    if (kappa) *kappa = B->probs[j].kappa;
    if (mu) *mu = B->probs[j].mu;
    if (flux) *flux = B->probs[j].flux;
    if (phi) *phi = B->probs[j].phi;
    return QPAT_OK;
}

int qpat_batch_forward(qpat_batch_t B, void* stream) {
    if (!B) return fail(QPAT_EINVAL, "qpat_batch_forward: NULL batch");
    DeviceGuard dg(B->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (!B->exec) {
        // recorded on a private stream (the legacy default stream cannot be
        // captured); the graph is then launched on the caller's stream
        cudaStream_t cs = nullptr;
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "qpat_batch_forward: stream");
        if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
            cudaStreamDestroy(cs);
            return cuda_fail(e, "qpat_batch_forward: begin capture");
        }
        const int rc = batch_sequence(B, cs);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (rc != QPAT_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "qpat_batch_forward: end capture");
        B->graph = g;
        if ((e = cudaGraphInstantiate(&B->exec, g, 0)) != cudaSuccess)
            return cuda_fail(e, "qpat_batch_forward: instantiate");
    }
    qpat::note_launch(1);  // the graph holds one cooperative kernel
    if ((e = cudaGraphLaunch(B->exec, s)) != cudaSuccess) return cuda_fail(e, "qpat_batch_forward: graph launch");
    return QPAT_OK;
}

int qpat_batch_status(qpat_batch_t B, int* status, int* iters, int* ctas) {
    if (!B) return fail(QPAT_EINVAL, "qpat_batch_status: NULL batch");
    DeviceGuard dg(B->device);
    for (size_t j = 0; j < B->probs.size(); ++j) {
        int h[2] = {0, 0};
        cudaError_t e1 = cudaMemcpy(&h[0], B->probs[j].ctl + 1, sizeof(int), cudaMemcpyDeviceToHost);
        cudaError_t e2 = cudaMemcpy(&h[1], B->probs[j].ctl + 2, sizeof(int), cudaMemcpyDeviceToHost);
        if (e1 != cudaSuccess || e2 != cudaSuccess) return cuda_fail(e1 != cudaSuccess ? e1 : e2, "qpat_batch_status");
        if (status) status[j] = h[0];
        if (iters) iters[j] = h[1];
        if (ctas) ctas[j] = B->plan.cta_count[j];
    }
    return QPAT_OK;
}

void qpat_batch_free(qpat_batch_t B) {
    if (!B) return;
    DeviceGuard dg(B->device);
    cudaDeviceSynchronize();
    batch_release(B);
    delete B;
}

}  // extern "C"
