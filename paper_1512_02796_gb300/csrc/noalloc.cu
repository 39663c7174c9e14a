// Allocation-free forward solve.
//
// Some callers cannot allocate device memory at the time they need a solve:
// real-time or embedded pipelines that forbid allocator calls after start-up
// (a cudaMalloc can block on the driver and stall the pipeline), and hosts
// that budget every byte of GPU memory themselves (an allocation inside a
// library call would break their budget).  For them,
// qpat_forward_noalloc_dev runs the forward solve phi = K^-1 f (FP64
// matrix-free PCG, the same kernel as the FP64 path) with all its scratch in
// one file-scope device array of fixed size, so that the call itself never
// allocates.  The caller still owns and passes every input and output; the
// mesh handle must have been built earlier (qpat_mesh allocates).
#include <mutex>

#include "abi_internal.h"

namespace qpat {

namespace {

// Node count times padded right-hand sides that the scratch can hold.
constexpr int64_t kNoallocMaxNR = int64_t(1) << 19;
// Scratch layout in doubles: kappa, mu, inverse diagonal (N each, N <= max),
// then six N x R vectors (f, x, r, p0, p1, q), two reduction buffers and a
// small control block (barrier, status, iteration count, statistics).
constexpr int64_t kPartials = int64_t(2) * kMaxGrid * kMaxNS + 2 * kMaxNS;  // = pcg_partials_doubles()
constexpr int64_t kCtl = 64;
// control block: barrier and status words in ctl[0..2], then 2 x 16 doubles
// of solver statistics from ctl[8]
static_assert(8 + 2 * 16 <= kCtl, "control block too small for the solver statistics");
constexpr int64_t kNoallocDoubles = 3 * kNoallocMaxNR + 6 * kNoallocMaxNR + kPartials + kCtl;

__device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {nullptr};

// Device address of the scratch on the current device, looked up once per
// device (cudaGetSymbolAddress, which allocates nothing).
int noalloc_base(int dev, double** out) {
    if (dev < 0 || dev >= 64) return fail(QPAT_EINVAL, "qpat_forward_noalloc_dev: device id out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "qpat_forward_noalloc_dev: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return QPAT_OK;
}

}  // namespace

}  // namespace qpat

using namespace qpat;

extern "C" int qpat_forward_noalloc_dev(qpat_mesh_t M, const double* kappa, const double* mu, int K,
                                        const double* flux_face, double rtol, int max_iter, double* phi,
                                        double* h, void* stream) {
    if (!M || !kappa || !mu || !flux_face) return fail(QPAT_EINVAL, "qpat_forward_noalloc_dev: NULL argument");
    const int R = round_rhs(K);
    if (K < 1 || R < 0) return fail(QPAT_EINVAL, "qpat_forward_noalloc_dev: K must be in [1, 16]");
    const int64_t N = M->h.N;
    if (N * R > kNoallocMaxNR)
        return fail(QPAT_EINVAL, "qpat_forward_noalloc_dev: nodes x padded illuminations = " +
                                     std::to_string(N * R) + " exceeds the fixed scratch limit " +
                                     std::to_string(kNoallocMaxNR));
    if (!(rtol > 0) || max_iter < 1) return fail(QPAT_EINVAL, "qpat_forward_noalloc_dev: rtol > 0, max_iter >= 1");
    DeviceGuard dg(M->device);
    double* base = nullptr;
    int rc = noalloc_base(M->device, &base);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = N * R;
    double* kl = base;
    double* ml = kl + kNoallocMaxNR;
    double* inv = ml + kNoallocMaxNR;
    double* f = inv + kNoallocMaxNR;
    double* x = f + kNoallocMaxNR;
    double* r = x + kNoallocMaxNR;
    double* p0 = r + kNoallocMaxNR;
    double* p1 = p0 + kNoallocMaxNR;
    double* q = p1 + kNoallocMaxNR;
    double* partials = q + kNoallocMaxNR;
    double* ctl = partials + kPartials;
    PcgWork w{};
    w.b = f;
    w.x = x;
    w.r = r;
    w.p0 = p0;
    w.p1 = p1;
    w.q = q;
    w.partials = partials;
    w.bar = reinterpret_cast<unsigned*>(ctl);        // 2 x unsigned in ctl[0]
    w.status = reinterpret_cast<int*>(ctl + 1);
    w.iters = reinterpret_cast<int*>(ctl + 2);
    w.stats = ctl + 8;                               // 32 doubles
    cudaError_t e;
    if ((e = launch_to_lib<double, double>(M->d, 1, 1, kappa, kl, s)) != cudaSuccess ||
        (e = launch_to_lib<double, double>(M->d, 1, 1, mu, ml, s)) != cudaSuccess)
        return cuda_fail(e, "qpat_forward_noalloc_dev: to_lib");
    // launch_load adds each node's face sums into f and leaves the padded
    // columns (K <= r < R) untouched: f must start at zero
    if ((e = cudaMemsetAsync(f, 0, sizeof(double) * n, s)) != cudaSuccess)
        return cuda_fail(e, "qpat_forward_noalloc_dev: memset");
    if ((e = launch_load(M->d, K, R, flux_face, f, s)) != cudaSuccess)
        return cuda_fail(e, "qpat_forward_noalloc_dev: load");
    if ((e = launch_invdiag_K(M->d, kl, ml, inv, nullptr, s)) != cudaSuccess)
        return cuda_fail(e, "qpat_forward_noalloc_dev: diagonal");
    OpParams<double> op{kl, ml, 0.0, 0.0, 0.0, 1, nullptr, nullptr};
    if ((e = launch_pcg<double>(M->d, OP_K, R, op, inv, w, rtol, max_iter, s, nullptr)) != cudaSuccess)
        return cuda_fail(e, "qpat_forward_noalloc_dev: pcg launch");
    if (phi && (e = launch_from_lib<double, double>(M->d, K, R, x, phi, s)) != cudaSuccess)
        return cuda_fail(e, "qpat_forward_noalloc_dev: from_lib");
    if (h) {
        k_rowscale_launch(N, R, ml, x, r, s);  // r is free once the solve is done
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "qpat_forward_noalloc_dev: rowscale");
        if ((e = launch_from_lib<double, double>(M->d, K, R, r, h, s)) != cudaSuccess)
            return cuda_fail(e, "qpat_forward_noalloc_dev: from_lib");
    }
    // solver status through the mesh's pinned host word (no allocation)
    int* hst = reinterpret_cast<int*>(M->host_scratch + 200);
    if ((e = cudaMemcpyAsync(hst, w.status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "qpat_forward_noalloc_dev: status");
    if (hst[0] == QPAT_ENOCONV) return fail(QPAT_ENOCONV, "qpat_forward_noalloc_dev: PCG iteration cap reached");
    if (hst[0] == QPAT_EBREAKDOWN) return fail(QPAT_EBREAKDOWN, "qpat_forward_noalloc_dev: PCG breakdown");
    if (hst[0] == QPAT_ETIMEOUT) return fail(QPAT_ETIMEOUT, "qpat_forward_noalloc_dev: grid barrier timed out");
    return QPAT_OK;
}
