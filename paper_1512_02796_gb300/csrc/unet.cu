// 3D U-Net runtime: a learned initial guess for the forward solves (not in
// the paper).  Four levels (16, 32, 64, 128 channels), two 3x3x3 ReLU convs
// per level, 2x2x2 average pooling down, nearest upsampling + skip
// concatenation up, and a final linear 3x3x3 conv whose channel 0 is the
// predicted fluence.  Weights are fp32 masters with bf16 copies; every conv
// runs on the bf16 tensor-core kernels of unet_kernels.cu, forward and
// backward, and Adam updates the masters.
//
// Input features on a Kuhn grid (node index = voxel index, n a multiple of
// 8): log(mu / 0.01), log(kappa / 0.33) and the load vector of the
// illumination (2 integral Phi lambda_i, Appendix) divided by h^2; target:
// the fluence phi of that illumination.
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "abi_internal.h"
#include "unet_kernels.cuh"

using bf16 = __nv_bfloat16;
using namespace qpat;

namespace {

struct Conv {
    int cin = 0, cout = 0, lvl = 0, relu = 1;
    float *w32 = nullptr, *b32 = nullptr;      // masters
    bf16 *w = nullptr, *wt = nullptr;           // bf16 copy and its flipped transpose
    float *gw = nullptr, *gb = nullptr;         // gradient of the last sample
    float *aw = nullptr, *ab = nullptr;         // accumulated gradient
    float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
    int64_t nw() const { return int64_t(27) * cin * cout; }
};

__global__ void k_features(int64_t nvox, const double* mu, const double* kappa, const double* f, double inv_h2,
                           float* x) {
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < nvox; v += int64_t(gridDim.x) * blockDim.x) {
        x[v * 3 + 0] = float(log(mu[v] / 0.01));
        x[v * 3 + 1] = float(log(kappa[v] / 0.33));
        x[v * 3 + 2] = float(f[v] * inv_h2);
    }
}

// network input (channels-last, 16 channels, 3 used) from fp32 features
__global__ void k_pack_input(int64_t nvox, const float* x, bf16* xin) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nvox * 16; i += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(i % 16);
        xin[i] = __float2bfloat16(c < 3 ? x[(i / 16) * 3 + c] : 0.f);
    }
}

// channel 0 of the output; in log mode (log_floor > 0) the network's output
// is log(phi) and the prediction is its exponential
__global__ void k_take_channel0(int64_t nvox, const float* y32, float* y, float log_floor) {
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < nvox; v += int64_t(gridDim.x) * blockDim.x)
        y[v] = log_floor > 0.f ? expf(y32[v * 16]) : y32[v * 16];
}

// mean-squared error of channel 0 and its gradient (bf16, 16 channels); in
// log mode against log(max(t, log_floor))
__global__ void k_mse(int64_t nvox, const float* y32, const float* t, float scale, bf16* dy, float* loss,
                      float log_floor) {
    __shared__ float red[256];
    float s = 0.f;
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < nvox; v += int64_t(gridDim.x) * blockDim.x) {
        const float tv = log_floor > 0.f ? logf(fmaxf(t[v], log_floor)) : t[v];
        const float d = y32[v * 16] - tv;
        s += d * d;
        dy[v * 16] = __float2bfloat16(2.f * d * scale);
        for (int c = 1; c < 16; ++c) dy[v * 16 + c] = __float2bfloat16(0.f);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] * scale);
}

__global__ void k_axpy32(int64_t n, float a, const float* x, float* y, int overwrite) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = overwrite ? a * x[i] : y[i] + a * x[i];
}

__global__ void k_f32_to_f64(int64_t n, const float* in, double* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = double(in[i]);
}

int g1(int64_t n) { return int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16))); }

}  // namespace

struct qpat_unet_s {
    int n = 0;
    int device = 0;
    int step = 0;
    std::vector<Conv> conv;
    std::vector<void*> allocs;
    int lv[4] = {0, 0, 0, 0};  // grid side per level
    // activations (bf16 channels-last) and their gradients
    bf16 *xin, *a0, *s0, *p0, *a1, *s1, *p1, *a2, *s2, *p2, *a3, *bt, *cat2, *a4, *d2, *cat1, *a5, *d1, *cat0, *a6,
        *d0, *yb;
    bf16 *g_y, *g_d0, *g_a6, *g_cat0, *g_d1, *g_s0, *g_a5, *g_cat1, *g_d2, *g_s1, *g_a4, *g_cat2, *g_bt, *g_s2, *g_a3,
        *g_p2, *g_a2, *g_p1, *g_a1, *g_p0, *g_a0;
    float* y32 = nullptr;
    float log_floor = 0.f;  // > 0: the network learns log(max(phi, log_floor)) (qpat_unet_set_log_output)
    float* partial = nullptr;
    float* loss = nullptr;
    float* hloss = nullptr;
};

namespace {

template <typename T>
int ualloc(qpat_unet_s* U, T** p, size_t count) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, "qpat_unet: cudaMalloc");
    U->allocs.push_back(v);
    *p = static_cast<T*>(v);
    e = cudaMemset(v, 0, std::max<size_t>(count, 1) * sizeof(T));
    return e == cudaSuccess ? QPAT_OK : cuda_fail(e, "qpat_unet: memset");
}

#define UCK(x)                                           \
    do {                                                 \
        cudaError_t e_ = (x);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
    } while (0)

int conv_fwd(const Conv& c, const bf16* in, bf16* out, float* out32, int n, cudaStream_t s) {
    UCK(unet::conv3d_fwd(in, c.cin, c.w, c.b32, c.cout, c.relu, out, out32, n, s));
    return QPAT_OK;
}

// backward of one conv: gout (gradient of its output, masked here by the
// ReLU through `out`) -> weight/bias gradient, and gin if not null
int conv_bwd(qpat_unet_s* U, Conv& c, const bf16* in, const bf16* out, bf16* gout, bf16* gin, int n,
             cudaStream_t s) {
    const int64_t nv = int64_t(n) * n * n;
    if (c.relu) UCK(unet::relu_mask(gout, out, nv * c.cout, s));
    UCK(unet::conv3d_wgrad(in, c.cin, gout, c.cout, c.gw, c.gb, U->partial, n, s));
    if (gin) UCK(unet::conv3d_fwd(gout, c.cout, c.wt, nullptr, c.cin, 0, gin, nullptr, n, s));
    return QPAT_OK;
}

int unet_forward(qpat_unet_s* U, cudaStream_t s) {
    auto& C = U->conv;
    const int n0 = U->lv[0], n1 = U->lv[1], n2 = U->lv[2], n3 = U->lv[3];
    int rc;
    if ((rc = conv_fwd(C[0], U->xin, U->a0, nullptr, n0, s)) || (rc = conv_fwd(C[1], U->a0, U->s0, nullptr, n0, s)))
        return rc;
    UCK(unet::avgpool(U->s0, 16, n0, U->p0, s));
    if ((rc = conv_fwd(C[2], U->p0, U->a1, nullptr, n1, s)) || (rc = conv_fwd(C[3], U->a1, U->s1, nullptr, n1, s)))
        return rc;
    UCK(unet::avgpool(U->s1, 32, n1, U->p1, s));
    if ((rc = conv_fwd(C[4], U->p1, U->a2, nullptr, n2, s)) || (rc = conv_fwd(C[5], U->a2, U->s2, nullptr, n2, s)))
        return rc;
    UCK(unet::avgpool(U->s2, 64, n2, U->p2, s));
    if ((rc = conv_fwd(C[6], U->p2, U->a3, nullptr, n3, s)) || (rc = conv_fwd(C[7], U->a3, U->bt, nullptr, n3, s)))
        return rc;
    UCK(unet::upcat(U->bt, 128, U->s2, 64, n2, U->cat2, s));
    if ((rc = conv_fwd(C[8], U->cat2, U->a4, nullptr, n2, s)) || (rc = conv_fwd(C[9], U->a4, U->d2, nullptr, n2, s)))
        return rc;
    UCK(unet::upcat(U->d2, 64, U->s1, 32, n1, U->cat1, s));
    if ((rc = conv_fwd(C[10], U->cat1, U->a5, nullptr, n1, s)) ||
        (rc = conv_fwd(C[11], U->a5, U->d1, nullptr, n1, s)))
        return rc;
    UCK(unet::upcat(U->d1, 32, U->s0, 16, n0, U->cat0, s));
    if ((rc = conv_fwd(C[12], U->cat0, U->a6, nullptr, n0, s)) ||
        (rc = conv_fwd(C[13], U->a6, U->d0, nullptr, n0, s)) || (rc = conv_fwd(C[14], U->d0, U->yb, U->y32, n0, s)))
        return rc;
    return QPAT_OK;
}

int unet_backward(qpat_unet_s* U, cudaStream_t s) {
    auto& C = U->conv;
    const int n0 = U->lv[0], n1 = U->lv[1], n2 = U->lv[2], n3 = U->lv[3];
    int rc;
    if ((rc = conv_bwd(U, C[14], U->d0, U->yb, U->g_y, U->g_d0, n0, s)) ||
        (rc = conv_bwd(U, C[13], U->a6, U->d0, U->g_d0, U->g_a6, n0, s)) ||
        (rc = conv_bwd(U, C[12], U->cat0, U->a6, U->g_a6, U->g_cat0, n0, s)))
        return rc;
    UCK(unet::upcat_bwd(U->g_cat0, 32, 16, n0, U->g_d1, U->g_s0, 0, s));
    if ((rc = conv_bwd(U, C[11], U->a5, U->d1, U->g_d1, U->g_a5, n1, s)) ||
        (rc = conv_bwd(U, C[10], U->cat1, U->a5, U->g_a5, U->g_cat1, n1, s)))
        return rc;
    UCK(unet::upcat_bwd(U->g_cat1, 64, 32, n1, U->g_d2, U->g_s1, 0, s));
    if ((rc = conv_bwd(U, C[9], U->a4, U->d2, U->g_d2, U->g_a4, n2, s)) ||
        (rc = conv_bwd(U, C[8], U->cat2, U->a4, U->g_a4, U->g_cat2, n2, s)))
        return rc;
    UCK(unet::upcat_bwd(U->g_cat2, 128, 64, n2, U->g_bt, U->g_s2, 0, s));
    if ((rc = conv_bwd(U, C[7], U->a3, U->bt, U->g_bt, U->g_a3, n3, s)) ||
        (rc = conv_bwd(U, C[6], U->p2, U->a3, U->g_a3, U->g_p2, n3, s)))
        return rc;
    UCK(unet::avgpool_bwd(U->g_p2, 64, n2, U->g_s2, 1, s));
    if ((rc = conv_bwd(U, C[5], U->a2, U->s2, U->g_s2, U->g_a2, n2, s)) ||
        (rc = conv_bwd(U, C[4], U->p1, U->a2, U->g_a2, U->g_p1, n2, s)))
        return rc;
    UCK(unet::avgpool_bwd(U->g_p1, 32, n1, U->g_s1, 1, s));
    if ((rc = conv_bwd(U, C[3], U->a1, U->s1, U->g_s1, U->g_a1, n1, s)) ||
        (rc = conv_bwd(U, C[2], U->p0, U->a1, U->g_a1, U->g_p0, n1, s)))
        return rc;
    UCK(unet::avgpool_bwd(U->g_p0, 16, n0, U->g_s0, 1, s));
    if ((rc = conv_bwd(U, C[1], U->a0, U->s0, U->g_s0, U->g_a0, n0, s)) ||
        (rc = conv_bwd(U, C[0], U->xin, U->a0, U->g_a0, nullptr, n0, s)))
        return rc;
    return QPAT_OK;
}

int refresh_bf16(qpat_unet_s* U, cudaStream_t s) {
    for (auto& c : U->conv) {
        UCK(unet::f32_to_bf16(c.w32, c.w, c.nw(), s));
        UCK(unet::flip_weights(c.w, c.cin, c.cout, c.wt, s));
    }
    return QPAT_OK;
}

}  // namespace

extern "C" {

int qpat_unet_create(int n, uint64_t seed, qpat_unet_t* out) {
    if (!out) return fail(QPAT_EINVAL, "qpat_unet_create: out is NULL");
    *out = nullptr;
    if (n < 32 || n % 16 || n > 512)
        return fail(QPAT_EINVAL, "qpat_unet_create: n must be a multiple of 16 in [32, 512]");
    auto* U = new qpat_unet_s();
    cudaGetDevice(&U->device);
    U->n = n;
    for (int l = 0; l < 4; ++l) U->lv[l] = n >> l;
    // (cin, cout, level, relu) of the 15 convs
    const int spec[15][4] = {{16, 16, 0, 1},  {16, 16, 0, 1},  {16, 32, 1, 1},  {32, 32, 1, 1},  {32, 64, 2, 1},
                             {64, 64, 2, 1},  {64, 128, 3, 1}, {128, 128, 3, 1}, {192, 64, 2, 1}, {64, 64, 2, 1},
                             {96, 32, 1, 1},  {32, 32, 1, 1},  {48, 16, 0, 1},  {16, 16, 0, 1},  {16, 16, 0, 0}};
    std::mt19937_64 rng(seed);
    int rc = QPAT_OK;
    const int64_t v0 = int64_t(n) * n * n, v1 = v0 / 8, v2 = v1 / 8, v3 = v2 / 8;
    for (int i = 0; i < 15 && rc == QPAT_OK; ++i) {
        Conv c;
        c.cin = spec[i][0];
        c.cout = spec[i][1];
        c.lvl = spec[i][2];
        c.relu = spec[i][3];
        const int64_t nw = c.nw();
        if ((rc = ualloc(U, &c.w32, nw)) || (rc = ualloc(U, &c.b32, c.cout)) || (rc = ualloc(U, &c.w, nw)) ||
            (rc = ualloc(U, &c.wt, nw)) || (rc = ualloc(U, &c.gw, nw)) || (rc = ualloc(U, &c.gb, c.cout)) ||
            (rc = ualloc(U, &c.aw, nw)) || (rc = ualloc(U, &c.ab, c.cout)) || (rc = ualloc(U, &c.mw, nw)) ||
            (rc = ualloc(U, &c.vw, nw)) || (rc = ualloc(U, &c.mb, c.cout)) || (rc = ualloc(U, &c.vb, c.cout)))
            break;
        // He-normal initialisation over the real fan-in (the first conv sees 3 channels)
        const int fan = 27 * (i == 0 ? 3 : c.cin);
        std::normal_distribution<float> nd(0.f, std::sqrt(2.f / float(fan)) * (c.relu ? 1.f : 0.5f));
        std::vector<float> hw(nw);
        for (int64_t k = 0; k < nw; ++k) {
            const int ci = int(k % c.cin);
            hw[k] = (i == 0 && ci >= 3) ? 0.f : nd(rng);
        }
        if (cudaMemcpy(c.w32, hw.data(), nw * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            rc = cuda_fail(cudaGetLastError(), "qpat_unet_create: upload");
        U->conv.push_back(c);
    }
    auto A = [&](bf16** p, int64_t nv, int ch) { return rc ? rc : (rc = ualloc(U, p, size_t(nv) * ch)); };
    A(&U->xin, v0, 16); A(&U->a0, v0, 16); A(&U->s0, v0, 16); A(&U->p0, v1, 16); A(&U->a1, v1, 32);
    A(&U->s1, v1, 32); A(&U->p1, v2, 32); A(&U->a2, v2, 64); A(&U->s2, v2, 64); A(&U->p2, v3, 64);
    A(&U->a3, v3, 128); A(&U->bt, v3, 128); A(&U->cat2, v2, 192); A(&U->a4, v2, 64); A(&U->d2, v2, 64);
    A(&U->cat1, v1, 96); A(&U->a5, v1, 32); A(&U->d1, v1, 32); A(&U->cat0, v0, 48); A(&U->a6, v0, 16);
    A(&U->d0, v0, 16); A(&U->yb, v0, 16);
    A(&U->g_y, v0, 16); A(&U->g_d0, v0, 16); A(&U->g_a6, v0, 16); A(&U->g_cat0, v0, 48); A(&U->g_d1, v1, 32);
    A(&U->g_s0, v0, 16); A(&U->g_a5, v1, 32); A(&U->g_cat1, v1, 96); A(&U->g_d2, v2, 64); A(&U->g_s1, v1, 32);
    A(&U->g_a4, v2, 64); A(&U->g_cat2, v2, 192); A(&U->g_bt, v3, 128); A(&U->g_s2, v2, 64); A(&U->g_a3, v3, 128);
    A(&U->g_p2, v3, 64); A(&U->g_a2, v2, 64); A(&U->g_p1, v2, 32); A(&U->g_a1, v1, 32); A(&U->g_p0, v1, 16);
    A(&U->g_a0, v0, 16);
    if (!rc) rc = ualloc(U, &U->y32, size_t(v0) * 16);
    if (!rc) rc = ualloc(U, &U->partial, size_t(unet::wgrad_chunks(n)) * 27 * 192 * 128);
    if (!rc) rc = ualloc(U, &U->loss, 1);
    if (!rc && cudaMallocHost(&U->hloss, sizeof(float)) != cudaSuccess) rc = fail(QPAT_ECUDA, "qpat_unet: pinned");
    if (!rc) rc = refresh_bf16(U, nullptr);
    if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "qpat_unet_create");
    if (rc) {
        qpat_unet_free(U);
        return rc;
    }
    *out = U;
    return QPAT_OK;
}

void qpat_unet_free(qpat_unet_t U) {
    if (!U) return;
    DeviceGuard dg(U->device);
    cudaDeviceSynchronize();
    for (void* p : U->allocs) cudaFree(p);
    if (U->hloss) cudaFreeHost(U->hloss);
    delete U;
}

int64_t qpat_unet_num_params(qpat_unet_t U) {
    if (!U) return -1;
    int64_t n = 0;
    for (auto& c : U->conv) n += c.nw() + c.cout;
    return n;
}

int qpat_unet_get_params(qpat_unet_t U, float* host) {
    if (!U || !host) return fail(QPAT_EINVAL, "qpat_unet_get_params: NULL argument");
    DeviceGuard dg(U->device);
    for (auto& c : U->conv) {
        UCK(cudaMemcpy(host, c.w32, c.nw() * sizeof(float), cudaMemcpyDeviceToHost));
        host += c.nw();
        UCK(cudaMemcpy(host, c.b32, c.cout * sizeof(float), cudaMemcpyDeviceToHost));
        host += c.cout;
    }
    return QPAT_OK;
}

int qpat_unet_set_params(qpat_unet_t U, const float* host) {
    if (!U || !host) return fail(QPAT_EINVAL, "qpat_unet_set_params: NULL argument");
    DeviceGuard dg(U->device);
    for (auto& c : U->conv) {
        UCK(cudaMemcpy(c.w32, host, c.nw() * sizeof(float), cudaMemcpyHostToDevice));
        host += c.nw();
        UCK(cudaMemcpy(c.b32, host, c.cout * sizeof(float), cudaMemcpyHostToDevice));
        host += c.cout;
    }
    int rc = refresh_bf16(U, nullptr);
    if (rc) return rc;
    UCK(cudaDeviceSynchronize());
    return QPAT_OK;
}

int qpat_unet_predict_dev(qpat_unet_t U, const float* x, int B, float* y, void* stream) {
    if (!U || !x || !y || B < 1) return fail(QPAT_EINVAL, "qpat_unet_predict_dev: bad argument");
    DeviceGuard dg(U->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t nv = int64_t(U->n) * U->n * U->n;
    for (int b = 0; b < B; ++b) {
        qpat::note_launch(1);
        k_pack_input<<<g1(nv * 16), 256, 0, s>>>(nv, x + b * nv * 3, U->xin);
        int rc = unet_forward(U, s);
        if (rc) return rc;
        qpat::note_launch(1);
        k_take_channel0<<<g1(nv), 256, 0, s>>>(nv, U->y32, y + b * nv, U->log_floor);
    }
    UCK(cudaGetLastError());
    return QPAT_OK;
}

// Loss (mean squared error over the B samples' voxels) into U->loss and its
// gradient with respect to every weight and bias into the accumulators
// aw, ab (summed over the samples).
static int unet_loss_grad(qpat_unet_s* U, const float* x, const float* t, int B, cudaStream_t s) {
    const int64_t nv = int64_t(U->n) * U->n * U->n;
    UCK(cudaMemsetAsync(U->loss, 0, sizeof(float), s));
    for (int b = 0; b < B; ++b) {
        qpat::note_launch(1);
        k_pack_input<<<g1(nv * 16), 256, 0, s>>>(nv, x + b * nv * 3, U->xin);
        int rc = unet_forward(U, s);
        if (rc) return rc;
        qpat::note_launch(1);
        k_mse<<<g1(nv), 256, 0, s>>>(nv, U->y32, t + b * nv, 1.f / float(nv * B), U->g_y, U->loss, U->log_floor);
        if ((rc = unet_backward(U, s))) return rc;
        for (auto& c : U->conv) {
            qpat::note_launch(1);
            k_axpy32<<<g1(c.nw()), 256, 0, s>>>(c.nw(), 1.f, c.gw, c.aw, b == 0);
            qpat::note_launch(1);
            k_axpy32<<<1, 256, 0, s>>>(c.cout, 1.f, c.gb, c.ab, b == 0);
        }
    }
    UCK(cudaGetLastError());
    return QPAT_OK;
}

int qpat_unet_grad_dev(qpat_unet_t U, const float* x, const float* t, int B, float* grad, float* loss,
                       void* stream) {
    if (!U || !x || !t || !grad || B < 1) return fail(QPAT_EINVAL, "qpat_unet_grad_dev: bad argument");
    DeviceGuard dg(U->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = unet_loss_grad(U, x, t, B, s);
    if (rc) return rc;
    size_t o = 0;
    for (auto& c : U->conv) {
        UCK(cudaMemcpyAsync(grad + o, c.aw, sizeof(float) * c.nw(), cudaMemcpyDeviceToHost, s));
        o += c.nw();
        UCK(cudaMemcpyAsync(grad + o, c.ab, sizeof(float) * c.cout, cudaMemcpyDeviceToHost, s));
        o += c.cout;
    }
    UCK(cudaMemcpyAsync(U->hloss, U->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    UCK(cudaStreamSynchronize(s));
    if (loss) *loss = *U->hloss;
    return QPAT_OK;
}

int qpat_unet_set_log_output(qpat_unet_t U, double floor) {
    if (!U || !(floor >= 0.0) || !std::isfinite(floor))
        return fail(QPAT_EINVAL, "qpat_unet_set_log_output: NULL network or bad floor");
    U->log_floor = float(floor);
    return QPAT_OK;
}

int qpat_unet_train_dev(qpat_unet_t U, const float* x, const float* t, int B, float lr, float* loss, void* stream) {
    if (!U || !x || !t || B < 1) return fail(QPAT_EINVAL, "qpat_unet_train_dev: bad argument");
    DeviceGuard dg(U->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc0 = unet_loss_grad(U, x, t, B, s);
    if (rc0) return rc0;
    ++U->step;
    for (auto& c : U->conv) {
        UCK(unet::adam(c.w32, nullptr, c.aw, c.mw, c.vw, c.nw(), lr, 0.9f, 0.999f, 1e-8f, U->step, s));
        UCK(unet::adam(c.b32, nullptr, c.ab, c.mb, c.vb, c.cout, lr, 0.9f, 0.999f, 1e-8f, U->step, s));
    }
    int rc = refresh_bf16(U, s);
    if (rc) return rc;
    if (loss) {
        UCK(cudaMemcpyAsync(U->hloss, U->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        UCK(cudaStreamSynchronize(s));
        *loss = *U->hloss;
    }
    return QPAT_OK;
}

// Network input of illumination k for every illumination of a Kuhn-grid mesh
// (caller node index = voxel index): x is K x N x 3 float
int qpat_unet_features_dev(qpat_mesh_t M, const double* kappa, const double* mu, int K, const double* flux_face,
                           double h, float* x, void* stream) {
    if (!M || !kappa || !mu || !flux_face || !x || K < 1 || !(h > 0))
        return fail(QPAT_EINVAL, "qpat_unet_features_dev: bad argument");
    DeviceGuard dg(M->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t N = M->h.N;
    const int R = round_rhs(K);
    if (R < 0) return fail(QPAT_EINVAL, "qpat_unet_features_dev: K must be in [1, 16]");
    cudaError_t e = cudaSuccess;
    double* f = M->ws.get<double>("un.f", N * R, s, &e);
    double* fc = M->ws.get<double>("un.fc", N * K, s, &e);
    if (e != cudaSuccess) return cuda_fail(e, "workspace");
    UCK(cudaMemsetAsync(f, 0, N * R * sizeof(double), s));
    UCK(launch_load(M->d, K, R, flux_face, f, s));
    UCK((launch_from_lib<double, double>(M->d, K, R, f, fc, s)));
    qpat::note_launch(K);
    for (int k = 0; k < K; ++k) k_features<<<g1(N), 256, 0, s>>>(N, mu, kappa, fc + k * N, 1.0 / (h * h), x + k * N * 3);
    UCK(cudaGetLastError());
    return QPAT_OK;
}

// float predictions -> double initial guess
int qpat_unet_to_double_dev(const float* y, int64_t count, double* out, void* stream) {
    qpat::note_launch(1);
    k_f32_to_f64<<<g1(count), 256, 0, static_cast<cudaStream_t>(stream)>>>(count, y, out);
    UCK(cudaGetLastError());
    return QPAT_OK;
}

// low-level entry points of the bf16 tensor-core convolution (tests)
int qpat_conv3d_bf16_dev(const void* in, int Cin, const void* w, const float* bias, int Cout, int relu, int n,
                         void* out, float* out_f32, void* stream) {
    if (!in || !w || !out) return fail(QPAT_EINVAL, "qpat_conv3d_bf16_dev: NULL argument");
    UCK(unet::conv3d_fwd(static_cast<const bf16*>(in), Cin, static_cast<const bf16*>(w), bias, Cout, relu,
                         static_cast<bf16*>(out), out_f32, n, static_cast<cudaStream_t>(stream)));
    return QPAT_OK;
}

int qpat_conv3d_bf16_wgrad_dev(const void* in, int Cin, const void* dy, int Cout, int n, float* dw, float* db,
                               float* partial, void* stream) {
    if (!in || !dy || !dw || !partial) return fail(QPAT_EINVAL, "qpat_conv3d_bf16_wgrad_dev: NULL argument");
    UCK(unet::conv3d_wgrad(static_cast<const bf16*>(in), Cin, static_cast<const bf16*>(dy), Cout, dw, db, partial, n,
                           static_cast<cudaStream_t>(stream)));
    return QPAT_OK;
}

int qpat_conv3d_set_engine(int engine) {
    if (engine != 0 && engine != 1) return fail(QPAT_EINVAL, "qpat_conv3d_set_engine: engine must be 0 or 1");
    unet::set_conv_engine(engine);
    return QPAT_OK;
}

int qpat_conv3d_tc_timeouts(void) { return unet::tc_timeouts(); }

int64_t qpat_conv3d_bf16_wgrad_scratch(int n, int Cin, int Cout) {
    return int64_t(unet::wgrad_chunks(n)) * 27 * Cin * Cout;
}

}  // extern "C"
