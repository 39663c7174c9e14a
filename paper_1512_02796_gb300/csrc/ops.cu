// Mesh upload and the forward / Jacobian / prior entry points (Appendix;
// Eqs. (14), (16), (19)).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "abi_internal.h"

namespace qpat {

namespace {

int grid_n(int64_t n) {
    int64_t g = (n + 255) / 256;
    return int(std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16)));
}

__global__ void k_nm_to_lib(int N, int R, int Rp, const int* perm, const double* in, double* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < int64_t(N) * Rp;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int l = int(i / Rp), r = int(i % Rp);
        out[i] = r < R ? in[int64_t(perm[l]) * R + r] : 0.0;
    }
}

__global__ void k_nm_from_lib(int N, int R, int Rp, const int* perm, const double* in, double* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < int64_t(N) * R;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int l = int(i / R), r = int(i % R);
        out[int64_t(perm[l]) * R + r] = in[int64_t(l) * Rp + r];
    }
}

__global__ void k_cast_f2d(int64_t n, const float* in, double* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = double(in[i]);
}

// pack two N x R arrays into one N x 2R array, and back
__global__ void k_pack2(int64_t N, int R, const double* a, const double* b, double* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N * 2 * R;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t l = i / (2 * R);
        const int r = int(i % (2 * R));
        out[i] = r < R ? a[l * R + r] : b[l * R + r - R];
    }
}

__global__ void k_unpack2(int64_t N, int R, const double* in, double* a, double* b) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N * 2 * R;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t l = i / (2 * R);
        const int r = int(i % (2 * R));
        if (r < R)
            a[l * R + r] = in[i];
        else
            b[l * R + r - R] = in[i];
    }
}

template <typename T>
int up(qpat_mesh_s* M, const std::vector<T>& v, const T** dst) {
    void* p = nullptr;
    size_t bytes = std::max<size_t>(v.size() * sizeof(T), 16);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "qpat_mesh: cudaMalloc");
    M->dev_allocs.push_back(p);
    if (!v.empty()) {
        e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "qpat_mesh: cudaMemcpy");
    }
    *dst = static_cast<const T*>(p);
    return QPAT_OK;
}

}  // namespace

cudaError_t launch_nodemajor_to_lib(const MeshDev& m, int R, int Rp, const double* in, double* out, cudaStream_t s) {
    qpat::note_launch(1);
    k_nm_to_lib<<<grid_n(int64_t(m.N) * Rp), 256, 0, s>>>(m.N, R, Rp, m.perm, in, out);
    return cudaGetLastError();
}
cudaError_t launch_nodemajor_from_lib(const MeshDev& m, int R, int Rp, const double* in, double* out,
                                      cudaStream_t s) {
    qpat::note_launch(1);
    k_nm_from_lib<<<grid_n(int64_t(m.N) * R), 256, 0, s>>>(m.N, R, Rp, m.perm, in, out);
    return cudaGetLastError();
}
cudaError_t launch_cast_f2d(int64_t n, const float* in, double* out, cudaStream_t s) {
    qpat::note_launch(1);
    k_cast_f2d<<<grid_n(n), 256, 0, s>>>(n, in, out);
    return cudaGetLastError();
}

int upload_mesh(qpat_mesh_s* M) {
    cudaError_t e = cudaGetDevice(&M->device);
    if (e != cudaSuccess) return cuda_fail(e, "qpat_mesh: no CUDA device");
    const HostMesh& h = M->h;
    MeshDev& d = M->d;
    d.N = int(h.N);
    d.E = int(h.E);
    d.F = int(h.F);
    d.P = h.P;
    d.max_touched = h.max_touched;
    d.max_own = h.max_own;
    d.max_ptets = h.max_ptets;
    d.max_pfaces = h.max_pfaces;
    std::vector<float> xyz32(h.xyz.begin(), h.xyz.end());
    std::vector<float> pa32(h.pface_area.begin(), h.pface_area.end());
    int rc = QPAT_OK;
    if ((rc = up(M, h.xyz, &d.xyz64)) || (rc = up(M, xyz32, &d.xyz32)) || (rc = up(M, h.own_begin, &d.own_begin)) ||
        (rc = up(M, h.node_ptr, &d.node_ptr)) || (rc = up(M, h.nodes, &d.nodes)) ||
        (rc = up(M, h.tet_ptr, &d.tet_ptr)) || (rc = up(M, h.face_ptr, &d.face_ptr)) ||
        (rc = up(M, h.pface_area, &d.pface_area64)) || (rc = up(M, pa32, &d.pface_area32)) ||
        (rc = up(M, h.faces_lib, &d.faces_lib)) || (rc = up(M, h.farea, &d.farea)) ||
        (rc = up(M, h.perm, &d.perm)) || (rc = up(M, h.iperm, &d.iperm)) ||
        (rc = up(M, h.tcol_beg, &d.tcol_beg)) || (rc = up(M, h.tcol_off, &d.tcol_off)) ||
        (rc = up(M, h.fcol_beg, &d.fcol_beg)) || (rc = up(M, h.fcol_off, &d.fcol_off)) ||
        (rc = up(M, h.nface_ptr, &d.nface_ptr)) || (rc = up(M, h.nface, &d.nface)))
        return rc;
    if ((rc = up(M, h.sell_ptr, &d.sell_ptr)) || (rc = up(M, h.sell_col, &d.sell_col)) ||
        (rc = up(M, h.sell_len, &d.sell_len)) || (rc = up(M, h.sell_diag, &d.sell_diag)))
        return rc;
    d.sell_entries = int64_t(h.sell_col.size());
    d.sell_wmax = h.sell_wmax;
    const uint16_t* tl = nullptr;
    if ((rc = up(M, h.tet_loc, &tl))) return rc;
    d.tet_loc = reinterpret_cast<const ushort4*>(tl);
    const uint16_t* fl = nullptr;
    if ((rc = up(M, h.face_loc, &fl))) return rc;
    d.face_loc = reinterpret_cast<const ushort4*>(fl);
    // the prior's view: everything as d, but the stiffness-only pattern
    MeshDev& dp = M->dp;
    dp = d;
    if ((rc = up(M, h.psell_ptr, &dp.sell_ptr)) || (rc = up(M, h.psell_col, &dp.sell_col)) ||
        (rc = up(M, h.psell_len, &dp.sell_len)) || (rc = up(M, h.psell_diag, &dp.sell_diag)))
        return rc;
    dp.sell_entries = int64_t(h.psell_col.size());
    dp.sell_wmax = h.psell_wmax;
    if ((e = cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "qpat_mesh: stream");
    if ((e = cudaMallocHost(&M->host_scratch, 256 * sizeof(double))) != cudaSuccess)
        return cuda_fail(e, "qpat_mesh: pinned scratch");
    return QPAT_OK;
}

SolveOpts solve_opts(const qpat_params* prm) {
    qpat_params d;
    qpat_default_params(&d);
    const qpat_params* p = prm ? prm : &d;
    SolveOpts so;
    so.precision = p->precision;
    so.rtol = p->pcg_rtol > 0 ? p->pcg_rtol : 1e-13;
    so.maxit = p->max_pcg_iter > 0 ? p->max_pcg_iter : 20000;
    so.fp32_assembled = p->fp32_operator == 1 ? 1 : 0;
    so.pcg_variant = p->pcg_variant;
    so.mixed_restart = p->mixed_restart ? 1 : 0;
    so.poly_k = p->poly_degree;
    so.poly_prior = p->prior_poly_degree;
    so.spin_limit = p->barrier_spin_limit > 0 ? p->barrier_spin_limit : 0;
    so.multigrid = p->multigrid;
    so.mg_degree = p->mg_degree > 0 ? p->mg_degree : 1;
    so.mg_ratio = p->mg_ratio > 0 ? p->mg_ratio : 30.0;
    return so;
}

static int check_params(const qpat_params* prm, const char* who) {
    if (!prm) return QPAT_OK;
    if (prm->precision != 0 && prm->precision != 1)
        return fail(QPAT_EINVAL, std::string(who) + ": precision must be 0 or 1");
    if (prm->pcg_variant < 0 || prm->pcg_variant > 3)
        return fail(QPAT_EINVAL, std::string(who) + ": pcg_variant must be 0, 1, 2 or 3");
    if (prm->prior != 0 && prm->prior != 1) return fail(QPAT_EINVAL, std::string(who) + ": prior must be 0 or 1");
    if (prm->poly_degree < 0 || prm->poly_degree > kMaxPolyDegree || prm->prior_poly_degree < 0 ||
        prm->prior_poly_degree > kMaxPolyDegree)
        return fail(QPAT_EINVAL, std::string(who) + ": poly_degree and prior_poly_degree must lie in [0, 8]");
    if (prm->prior == 1 && !(prm->prior_q > 0.0 && prm->prior_q <= 2.0))
        return fail(QPAT_EINVAL, std::string(who) + ": prior_q must lie in (0, 2]");
    if (prm->barrier_spin_limit < 0) return fail(QPAT_EINVAL, std::string(who) + ": barrier_spin_limit must be >= 0");
    if (prm->lsqr_reorth != 0 && prm->lsqr_reorth != 1)
        return fail(QPAT_EINVAL, std::string(who) + ": lsqr_reorth must be 0 or 1");
    if (prm->multigrid < 0 || prm->multigrid > 2)
        return fail(QPAT_EINVAL, std::string(who) + ": multigrid must be 0, 1 or 2");
    if (prm->mg_degree < 0 || prm->mg_degree > 8 || prm->mg_ratio < 0 || (prm->mg_ratio > 0 && prm->mg_ratio <= 1))
        return fail(QPAT_EINVAL, std::string(who) + ": mg_degree must lie in [0, 8] and mg_ratio be 0 or above 1");
    return QPAT_OK;
}

int forward_lib(qpat_mesh_s* M, const SolveOpts& so, LinState& L, const double* flux_dev, cudaStream_t s,
                const double* x0) {
    const int64_t N = M->h.N;
    cudaError_t e = cudaSuccess;
    double* f = M->ws.get<double>("fw.f", N * L.R, s, &e);
    if (e != cudaSuccess) return cuda_fail(e, "workspace");
    if ((e = cudaMemsetAsync(f, 0, N * L.R * sizeof(double), s)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = launch_load(M->d, L.K, L.R, flux_dev, f, s)) != cudaSuccess) return cuda_fail(e, "load");
    return solve(M, L.opK, so, L.R, f, L.phi, s, x0);
}

int jvp_lib(qpat_mesh_s* M, const SolveOpts& so, LinState& L, const double* s1, const double* s2, double* out,
            cudaStream_t s) {
    const int64_t N = M->h.N;
    const int R = L.R;
    cudaError_t e = cudaSuccess;
    double* a = M->ws.get<double>("jv.a", N, s, &e);
    double* b = M->ws.get<double>("jv.b", N, s, &e);
    double* rhs = M->ws.get<double>("jv.rhs", N * R, s, &e);
    double* x = M->ws.get<double>("jv.x", N * R, s, &e);
    if (e != cudaSuccess) return cuda_fail(e, "workspace");
    k_mul_launch(N, L.kap, s1, a, s);
    k_mul_launch(N, L.mu, s2, b, s);
    // rhs = G1 diag(kappa) s1 + G2 diag(mu) s2 = -(S(kappa o s1) + M(mu o s2)) phi
    if ((e = launch_apply_K<double>(M->d, R, a, b, 0, -1.0, L.phi, rhs, s)) != cudaSuccess)
        return cuda_fail(e, "jv rhs");
    int rc = solve(M, L.opK, so, R, rhs, x, s);
    if (rc != QPAT_OK) return rc;
    k_jv_out_launch(N, R, L.mu, b, x, L.phi, L.w, out, s);
    return QPAT_OK;
}

int vjp_lib(qpat_mesh_s* M, const SolveOpts& so, LinState& L, const double* t, double* o1, double* o2,
            cudaStream_t s) {
    const int64_t N = M->h.N;
    const int R = L.R;
    cudaError_t e = cudaSuccess;
    double* tw = M->ws.get<double>("jt.tw", N * R, s, &e);
    double* rhs = M->ws.get<double>("jt.rhs", N * R, s, &e);
    double* z = M->ws.get<double>("jt.z", N * R, s, &e);
    double* y = M->ws.get<double>("jt.y", N * 2, s, &e);
    if (e != cudaSuccess) return cuda_fail(e, "workspace");
    if (L.w)
        k_mul_launch(N * R, L.w, t, tw, s);
    else if ((e = cudaMemcpyAsync(tw, t, N * R * sizeof(double), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "copy");
    k_rowscale_launch(N, R, L.mu, tw, rhs, s);
    int rc = solve(M, L.opK, so, R, rhs, z, s);
    if (rc != QPAT_OK) return rc;
    if ((e = launch_vjp_accum<double>(M->d, R, L.phi, z, y, s)) != cudaSuccess) return cuda_fail(e, "vjp accum");
    k_jt_out_launch(N, R, L.kap, L.mu, y, L.phi, tw, o1, o2, s);
    return QPAT_OK;
}

namespace {
// flag = 1 if some a[i] (or b[i]) is not finite, or (positive) not > 0
__global__ void k_check_coeffs(int64_t n, const double* a, const double* b, int positive, int* flag) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double x = a[i], y = b ? b[i] : 1.0;
        const bool bad = positive ? !(x > 0.0 && isfinite(x) && y > 0.0 && isfinite(y)) : !(isfinite(x) && isfinite(y));
        if (bad) *flag = 1;
    }
}
}  // namespace

// Rejects coefficient inputs the operators are not defined for (Eq. (1) needs
// kappa, mu in L^inf_+: positive and finite; log parameters must be finite)
// before any assembly: QPAT_EINVAL with `what` in the message.  Reads one
// flag back (synchronises the stream).
int check_coeffs(qpat_mesh_s* M, int64_t n, const double* a, const double* b, int positive, const char* what,
                 cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    int* flag = M->ws.get<int>("chk.flag", 1, s, &e);
    if (e != cudaSuccess) return cuda_fail(e, "workspace");
    if ((e = cudaMemsetAsync(flag, 0, sizeof(int), s)) != cudaSuccess) return cuda_fail(e, "memset");
    const int64_t g = std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
    qpat::note_launch(1);
    k_check_coeffs<<<int(g), 256, 0, s>>>(n, a, b, positive, flag);
    int* hf = reinterpret_cast<int*>(M->host_scratch + 210);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(hf, flag, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "coefficient check");
    if (*hf) return fail(QPAT_EINVAL, std::string(what) + (positive ? " must be positive and finite" : " must be finite"));
    return QPAT_OK;
}

// Upload caller-order device inputs into a LinState (library order).
static int lin_from_caller(qpat_mesh_s* M, const double* kappa, const double* mu, int K, const double* phi,
                           const double* w, LinState& L, cudaStream_t s) {
    const int64_t N = M->h.N;
    cudaError_t e = cudaSuccess;
    L.K = K;
    L.R = round_rhs(K);
    L.kap = M->ws.get<double>("lin.kap", N, s, &e);
    L.mu = M->ws.get<double>("lin.mu", N, s, &e);
    L.phi = M->ws.get<double>("lin.phi", N * L.R, s, &e);
    L.w = w ? M->ws.get<double>("lin.w", N * L.R, s, &e) : nullptr;
    if (e != cudaSuccess) return cuda_fail(e, "workspace");
    if ((e = launch_to_lib<double, double>(M->d, 1, 1, kappa, L.kap, s)) != cudaSuccess ||
        (e = launch_to_lib<double, double>(M->d, 1, 1, mu, L.mu, s)) != cudaSuccess)
        return cuda_fail(e, "to_lib");
    int rc = check_coeffs(M, N, L.kap, L.mu, 1, "kappa and mu", s);
    if (rc != QPAT_OK) return rc;
    if (phi && (e = launch_to_lib<double, double>(M->d, K, L.R, phi, L.phi, s)) != cudaSuccess)
        return cuda_fail(e, "to_lib");
    if (w && (e = launch_to_lib<double, double>(M->d, K, L.R, w, L.w, s)) != cudaSuccess)
        return cuda_fail(e, "to_lib");
    return prepare_K(M, L.kap, L.mu, L.opK, s);
}

}  // namespace qpat

using namespace qpat;

namespace {

struct HostCall {
    // stages host arrays in the mesh workspace (slots hc0, hc1, ...) on the
    // mesh's own stream; no allocation after the first call of a given size
    qpat_mesh_s* M;
    int slot = 0;
    explicit HostCall(qpat_mesh_s* m) : M(m) {}
    double* out(size_t n, int* rc) {
        cudaError_t e = cudaSuccess;
        double* p = M->ws.get<double>("hc" + std::to_string(slot++), std::max<size_t>(n, 1), M->stream, &e);
        if (e != cudaSuccess) *rc = cuda_fail(e, "host call: workspace");
        return p;
    }
    double* in(const double* h, size_t n, int* rc) {
        if (!h) return nullptr;
        double* p = out(n, rc);
        if (!p) return nullptr;
        cudaError_t e = cudaMemcpyAsync(p, h, n * sizeof(double), cudaMemcpyHostToDevice, M->stream);
        if (e != cudaSuccess) *rc = cuda_fail(e, "host call: H2D");
        return p;
    }
    int back(double* h, const double* d, size_t n) {
        if (!h || !d) return QPAT_OK;
        cudaError_t e = cudaMemcpyAsync(h, d, n * sizeof(double), cudaMemcpyDeviceToHost, M->stream);
        if (e != cudaSuccess) return cuda_fail(e, "host call: D2H");
        return QPAT_OK;
    }
    int sync() {
        cudaError_t e = cudaStreamSynchronize(M->stream);
        return e == cudaSuccess ? QPAT_OK : cuda_fail(e, "host call: sync");
    }
};

}  // namespace

extern "C" {

int qpat_forward_dev(qpat_mesh_t M, const qpat_params* prm, const double* kappa, const double* mu, int K,
                     const double* flux_face, double* phi, double* h, void* stream) {
    return qpat_forward_guess_dev(M, prm, kappa, mu, K, flux_face, nullptr, phi, h, stream);
}

int qpat_forward_guess_dev(qpat_mesh_t M, const qpat_params* prm, const double* kappa, const double* mu, int K,
                           const double* flux_face, const double* phi0, double* phi, double* h, void* stream) {
    if (!M || !kappa || !mu || !flux_face) return fail(QPAT_EINVAL, "qpat_forward: NULL argument");
    if (K < 1 || round_rhs(K) < 0) return fail(QPAT_EINVAL, "qpat_forward: K must be in [1, 16]");
    int rc = check_params(prm, "qpat_forward");
    if (rc) return rc;
    DeviceGuard dg(M->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LinState L;
    if ((rc = lin_from_caller(M, kappa, mu, K, nullptr, nullptr, L, s))) return rc;
    SolveOpts so = solve_opts(prm);
    double* x0 = nullptr;
    if (phi0) {
        cudaError_t e0 = cudaSuccess;
        x0 = M->ws.get<double>("fw.x0", M->h.N * L.R, s, &e0);
        if (e0 != cudaSuccess) return cuda_fail(e0, "workspace");
        if ((e0 = launch_to_lib<double, double>(M->d, K, L.R, phi0, x0, s)) != cudaSuccess)
            return cuda_fail(e0, "to_lib");
    }
    if ((rc = forward_lib(M, so, L, flux_face, s, x0))) return rc;
    cudaError_t e = cudaSuccess;
    if (phi && (e = launch_from_lib<double, double>(M->d, K, L.R, L.phi, phi, s)) != cudaSuccess)
        return cuda_fail(e, "from_lib");
    if (h) {
        const int64_t N = M->h.N;
        double* hl = M->ws.get<double>("fw.h", N * L.R, s, &e);
        if (e != cudaSuccess) return cuda_fail(e, "workspace");
        k_rowscale_launch(N, L.R, L.mu, L.phi, hl, s);
        if ((e = launch_from_lib<double, double>(M->d, K, L.R, hl, h, s)) != cudaSuccess)
            return cuda_fail(e, "from_lib");
    }
    return QPAT_OK;
}

int qpat_forward(qpat_mesh_t M, const qpat_params* prm, const double* kappa, const double* mu, int K,
                 const double* flux_face, double* phi, double* h) {
    if (!M) return fail(QPAT_EINVAL, "qpat_forward: NULL mesh");
    DeviceGuard dg(M->device);
    const size_t N = M->h.N, F = M->h.F;
    int rc = QPAT_OK;
    HostCall hc(M);
    double* dk = hc.in(kappa, N, &rc);
    double* dm = hc.in(mu, N, &rc);
    double* df = hc.in(flux_face, size_t(K > 0 ? K : 0) * F, &rc);
    double* dp = phi ? hc.out(size_t(K) * N, &rc) : nullptr;
    double* dh = h ? hc.out(size_t(K) * N, &rc) : nullptr;
    if (rc) return rc;
    if ((rc = qpat_forward_dev(M, prm, dk, dm, K, df, dp, dh, M->stream))) return rc;
    if ((rc = hc.back(phi, dp, size_t(K) * N)) || (rc = hc.back(h, dh, size_t(K) * N))) return rc;
    return hc.sync();
}

int qpat_jvp_dev(qpat_mesh_t M, const qpat_params* prm, const double* kappa, const double* mu, int K,
                 const double* phi, const double* w, const double* sv, double* out, void* stream) {
    if (!M || !kappa || !mu || !phi || !sv || !out) return fail(QPAT_EINVAL, "qpat_jvp: NULL argument");
    if (K < 1 || round_rhs(K) < 0) return fail(QPAT_EINVAL, "qpat_jvp: K must be in [1, 16]");
    int rc = check_params(prm, "qpat_jvp");
    if (rc) return rc;
    DeviceGuard dg(M->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t N = M->h.N;
    LinState L;
    if ((rc = lin_from_caller(M, kappa, mu, K, phi, w, L, s))) return rc;
    cudaError_t e = cudaSuccess;
    double* s1 = M->ws.get<double>("jvp.s1", N, s, &e);
    double* s2 = M->ws.get<double>("jvp.s2", N, s, &e);
    double* o = M->ws.get<double>("jvp.out", N * L.R, s, &e);
    if (e != cudaSuccess) return cuda_fail(e, "workspace");
    if ((e = launch_to_lib<double, double>(M->d, 1, 1, sv, s1, s)) != cudaSuccess ||
        (e = launch_to_lib<double, double>(M->d, 1, 1, sv + N, s2, s)) != cudaSuccess)
        return cuda_fail(e, "to_lib");
    if ((rc = jvp_lib(M, solve_opts(prm), L, s1, s2, o, s))) return rc;
    if ((e = launch_from_lib<double, double>(M->d, K, L.R, o, out, s)) != cudaSuccess)
        return cuda_fail(e, "from_lib");
    return QPAT_OK;
}

int qpat_jvp(qpat_mesh_t M, const qpat_params* prm, const double* kappa, const double* mu, int K, const double* phi,
             const double* w, const double* sv, double* out) {
    if (!M) return fail(QPAT_EINVAL, "qpat_jvp: NULL mesh");
    DeviceGuard dg(M->device);
    const size_t N = M->h.N;
    int rc = QPAT_OK;
    HostCall hc(M);
    double* dk = hc.in(kappa, N, &rc);
    double* dm = hc.in(mu, N, &rc);
    double* dp = hc.in(phi, size_t(K) * N, &rc);
    double* dw = hc.in(w, size_t(K) * N, &rc);
    double* ds = hc.in(sv, 2 * N, &rc);
    double* dout = hc.out(size_t(K) * N, &rc);
    if (rc) return rc;
    if ((rc = qpat_jvp_dev(M, prm, dk, dm, K, dp, dw, ds, dout, M->stream))) return rc;
    if ((rc = hc.back(out, dout, size_t(K) * N))) return rc;
    return hc.sync();
}

int qpat_vjp_dev(qpat_mesh_t M, const qpat_params* prm, const double* kappa, const double* mu, int K,
                 const double* phi, const double* w, const double* t, double* out, void* stream) {
    if (!M || !kappa || !mu || !phi || !t || !out) return fail(QPAT_EINVAL, "qpat_vjp: NULL argument");
    if (K < 1 || round_rhs(K) < 0) return fail(QPAT_EINVAL, "qpat_vjp: K must be in [1, 16]");
    int rc = check_params(prm, "qpat_vjp");
    if (rc) return rc;
    DeviceGuard dg(M->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t N = M->h.N;
    LinState L;
    if ((rc = lin_from_caller(M, kappa, mu, K, phi, w, L, s))) return rc;
    cudaError_t e = cudaSuccess;
    double* tl = M->ws.get<double>("vjp.t", N * L.R, s, &e);
    double* o1 = M->ws.get<double>("vjp.o1", N, s, &e);
    double* o2 = M->ws.get<double>("vjp.o2", N, s, &e);
    if (e != cudaSuccess) return cuda_fail(e, "workspace");
    if ((e = launch_to_lib<double, double>(M->d, K, L.R, t, tl, s)) != cudaSuccess) return cuda_fail(e, "to_lib");
    if ((rc = vjp_lib(M, solve_opts(prm), L, tl, o1, o2, s))) return rc;
    if ((e = launch_from_lib<double, double>(M->d, 1, 1, o1, out, s)) != cudaSuccess ||
        (e = launch_from_lib<double, double>(M->d, 1, 1, o2, out + N, s)) != cudaSuccess)
        return cuda_fail(e, "from_lib");
    return QPAT_OK;
}

int qpat_vjp(qpat_mesh_t M, const qpat_params* prm, const double* kappa, const double* mu, int K, const double* phi,
             const double* w, const double* t, double* out) {
    if (!M) return fail(QPAT_EINVAL, "qpat_vjp: NULL mesh");
    DeviceGuard dg(M->device);
    const size_t N = M->h.N;
    int rc = QPAT_OK;
    HostCall hc(M);
    double* dk = hc.in(kappa, N, &rc);
    double* dm = hc.in(mu, N, &rc);
    double* dp = hc.in(phi, size_t(K) * N, &rc);
    double* dw = hc.in(w, size_t(K) * N, &rc);
    double* dt = hc.in(t, size_t(K) * N, &rc);
    double* dout = hc.out(2 * N, &rc);
    if (rc) return rc;
    if ((rc = qpat_vjp_dev(M, prm, dk, dm, K, dp, dw, dt, dout, M->stream))) return rc;
    if ((rc = hc.back(out, dout, 2 * N))) return rc;
    return hc.sync();
}

int qpat_jvp_vjp_pair_dev(qpat_mesh_t M, const qpat_params* prm, const double* kappa, const double* mu, int K,
                          const double* phi, const double* w, const double* sv, const double* t, double* out_jv,
                          double* out_vjp, void* stream) {
    if (!M || !kappa || !mu || !phi || !sv || !t || !out_jv || !out_vjp)
        return fail(QPAT_EINVAL, "qpat_jvp_vjp_pair: NULL argument");
    if (K < 1 || round_rhs(K) < 0 || 2 * round_rhs(K) > 16)
        return fail(QPAT_EINVAL, "qpat_jvp_vjp_pair: K must be in [1, 8]");
    int rc = check_params(prm, "qpat_jvp_vjp_pair");
    if (rc) return rc;
    DeviceGuard dg(M->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t N = M->h.N;
    LinState L;
    if ((rc = lin_from_caller(M, kappa, mu, K, phi, w, L, s))) return rc;
    const int R = L.R;
    cudaError_t e = cudaSuccess;
    double* s1 = M->ws.get<double>("pair.s1", N, s, &e);
    double* s2 = M->ws.get<double>("pair.s2", N, s, &e);
    double* a = M->ws.get<double>("pair.a", N, s, &e);
    double* b = M->ws.get<double>("pair.b", N, s, &e);
    double* tl = M->ws.get<double>("pair.t", N * R, s, &e);
    double* tw = M->ws.get<double>("pair.tw", N * R, s, &e);
    double* rj = M->ws.get<double>("pair.rj", N * R, s, &e);
    double* rt = M->ws.get<double>("pair.rt", N * R, s, &e);
    double* rhs2 = M->ws.get<double>("pair.rhs2", N * 2 * R, s, &e);
    double* x2 = M->ws.get<double>("pair.x2", N * 2 * R, s, &e);
    double* xj = M->ws.get<double>("pair.xj", N * R, s, &e);
    double* z = M->ws.get<double>("pair.z", N * R, s, &e);
    double* y = M->ws.get<double>("pair.y", N * 2, s, &e);
    double* oj = M->ws.get<double>("pair.oj", N * R, s, &e);
    double* o1 = M->ws.get<double>("pair.o1", N, s, &e);
    double* o2 = M->ws.get<double>("pair.o2", N, s, &e);
    if (e != cudaSuccess) return cuda_fail(e, "workspace");
    if ((e = launch_to_lib<double, double>(M->d, 1, 1, sv, s1, s)) != cudaSuccess ||
        (e = launch_to_lib<double, double>(M->d, 1, 1, sv + N, s2, s)) != cudaSuccess ||
        (e = launch_to_lib<double, double>(M->d, K, R, t, tl, s)) != cudaSuccess)
        return cuda_fail(e, "to_lib");
    // J s right-hand sides
    k_mul_launch(N, L.kap, s1, a, s);
    k_mul_launch(N, L.mu, s2, b, s);
    if ((e = launch_apply_K<double>(M->d, R, a, b, 0, -1.0, L.phi, rj, s)) != cudaSuccess)
        return cuda_fail(e, "jv rhs");
    // J^T w right-hand sides
    if (L.w)
        k_mul_launch(N * R, L.w, tl, tw, s);
    else if ((e = cudaMemcpyAsync(tw, tl, N * R * sizeof(double), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "copy");
    k_rowscale_launch(N, R, L.mu, tw, rt, s);
    // one 2R-RHS block solve
    qpat::note_launch(1);
    k_pack2<<<grid_n(N * 2 * R), 256, 0, s>>>(N, R, rj, rt, rhs2);
    if ((rc = solve(M, L.opK, solve_opts(prm), 2 * R, rhs2, x2, s))) return rc;
    qpat::note_launch(1);
    k_unpack2<<<grid_n(N * 2 * R), 256, 0, s>>>(N, R, x2, xj, z);
    k_jv_out_launch(N, R, L.mu, b, xj, L.phi, L.w, oj, s);
    if ((e = launch_vjp_accum<double>(M->d, R, L.phi, z, y, s)) != cudaSuccess) return cuda_fail(e, "vjp accum");
    k_jt_out_launch(N, R, L.kap, L.mu, y, L.phi, tw, o1, o2, s);
    if ((e = launch_from_lib<double, double>(M->d, K, R, oj, out_jv, s)) != cudaSuccess ||
        (e = launch_from_lib<double, double>(M->d, 1, 1, o1, out_vjp, s)) != cudaSuccess ||
        (e = launch_from_lib<double, double>(M->d, 1, 1, o2, out_vjp + N, s)) != cudaSuccess)
        return cuda_fail(e, "from_lib");
    return QPAT_OK;
}

int qpat_jvp_vjp_pair(qpat_mesh_t M, const qpat_params* prm, const double* kappa, const double* mu, int K,
                      const double* phi, const double* w, const double* sv, const double* t, double* out_jv,
                      double* out_vjp) {
    if (!M) return fail(QPAT_EINVAL, "qpat_jvp_vjp_pair: NULL mesh");
    DeviceGuard dg(M->device);
    const size_t N = M->h.N;
    int rc = QPAT_OK;
    HostCall hc(M);
    double* dk = hc.in(kappa, N, &rc);
    double* dm = hc.in(mu, N, &rc);
    double* dp = hc.in(phi, size_t(K) * N, &rc);
    double* dw = hc.in(w, size_t(K) * N, &rc);
    double* ds = hc.in(sv, 2 * N, &rc);
    double* dt = hc.in(t, size_t(K) * N, &rc);
    double* dj = hc.out(size_t(K) * N, &rc);
    double* dv = hc.out(2 * N, &rc);
    if (rc) return rc;
    if ((rc = qpat_jvp_vjp_pair_dev(M, prm, dk, dm, K, dp, dw, ds, dt, dj, dv, M->stream))) return rc;
    if ((rc = hc.back(out_jv, dj, size_t(K) * N)) || (rc = hc.back(out_vjp, dv, 2 * N))) return rc;
    return hc.sync();
}

int qpat_prior_solve_dev(qpat_mesh_t M, const qpat_params* prm, const double* kt, const double* mt,
                         const double* rhs, double* out, void* stream) {
    if (!M || !kt || !mt || !rhs || !out) return fail(QPAT_EINVAL, "qpat_prior_solve: NULL argument");
    int rc = check_params(prm, "qpat_prior_solve");
    if (rc) return rc;
    qpat_params d;
    qpat_default_params(&d);
    const qpat_params* p = prm ? prm : &d;
    if (!(p->T > 0) || !(p->delta > 0) || !(p->b_over_a > 0))
        return fail(QPAT_EINVAL, "qpat_prior_solve: T, delta and b/a must be positive");
    DeviceGuard dg(M->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t N = M->h.N;
    cudaError_t e = cudaSuccess;
    double* ktl = M->ws.get<double>("pr.kt", N, s, &e);
    double* mtl = M->ws.get<double>("pr.mt", N, s, &e);
    double* bl = M->ws.get<double>("pr.b", 2 * N, s, &e);
    double* xl = M->ws.get<double>("pr.x", 2 * N, s, &e);
    if (e != cudaSuccess) return cuda_fail(e, "workspace");
    if ((e = launch_to_lib<double, double>(M->d, 1, 1, kt, ktl, s)) != cudaSuccess ||
        (e = launch_to_lib<double, double>(M->d, 1, 1, mt, mtl, s)) != cudaSuccess ||
        (e = launch_to_lib<double, double>(M->d, 2, 2, rhs, bl, s)) != cudaSuccess)
        return cuda_fail(e, "to_lib");
    if ((rc = check_coeffs(M, N, ktl, mtl, 0, "qpat_prior_solve: kt and mt", s))) return rc;
    OpState st;
    if ((rc = prepare_prior(M, ktl, mtl, p->T, p->prior, p->prior_q, p->b_over_a, p->delta, st, s))) return rc;
    if ((rc = solve(M, st, solve_opts(prm), 2, bl, xl, s))) return rc;
    if ((e = launch_from_lib<double, double>(M->d, 2, 2, xl, out, s)) != cudaSuccess)
        return cuda_fail(e, "from_lib");
    return QPAT_OK;
}

int qpat_prior_solve(qpat_mesh_t M, const qpat_params* prm, const double* kt, const double* mt, const double* rhs,
                     double* out) {
    if (!M) return fail(QPAT_EINVAL, "qpat_prior_solve: NULL mesh");
    DeviceGuard dg(M->device);
    const size_t N = M->h.N;
    int rc = QPAT_OK;
    HostCall hc(M);
    double* dk = hc.in(kt, N, &rc);
    double* dm = hc.in(mt, N, &rc);
    double* db = hc.in(rhs, 2 * N, &rc);
    double* dout = hc.out(2 * N, &rc);
    if (rc) return rc;
    if ((rc = qpat_prior_solve_dev(M, prm, dk, dm, db, dout, M->stream))) return rc;
    if ((rc = hc.back(out, dout, 2 * N))) return rc;
    return hc.sync();
}

}  // extern "C"
