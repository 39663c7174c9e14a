// BF16 tensor-core kernels of the 3D U-Net (see unet_kernels.cuh).
#include <algorithm>

#include "unet_kernels.cuh"

namespace qpat {
namespace unet {

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return uint32_t(__bfloat16_as_ushort(lo)) | (uint32_t(__bfloat16_as_ushort(hi)) << 16);
}

// neighbour of linear voxel v = (z, y, x) across tap, or -1 outside the grid
__device__ __forceinline__ int nbr(int z, int y, int x, int tap, int n) {
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const int zz = z + dz, yy = y + dy, xx = x + dx;
    if (zz < 0 || yy < 0 || xx < 0 || zz >= n || yy >= n || xx >= n) return -1;
    return (zz * n + yy) * n + xx;
}

constexpr int kConvWarps = 8;  // 128 voxels per CTA

// out[v][co] = act( bias[co] + sum_{tap, ci} in[nbr(v, tap)][ci] * w[tap][co][ci] )
template <int NT>
__global__ void __launch_bounds__(kConvWarps * 32) k_conv_fwd(const bf16* __restrict__ in, int Cin,
                                                              const bf16* __restrict__ w,
                                                              const float* __restrict__ bias, int Cout, int relu,
                                                              bf16* __restrict__ out, float* __restrict__ out32,
                                                              int n) {
    extern __shared__ uint32_t sw[];  // one tap: Cout rows of (Cin + 8) bf16
    const int nvox = n * n * n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int v0 = (blockIdx.x * kConvWarps + warp) * 16;
    const bool live = v0 < nvox;
    const int rA = v0 + g, rB = v0 + g + 8;
    const int zA = rA / (n * n), yA = (rA / n) % n, xA = rA % n;
    const int zB = rB / (n * n), yB = (rB / n) % n, xB = rB % n;
    const int ldw = (Cin + 8) / 2;
    const int cw = Cin / 2;
    float acc[NT][4];
#pragma unroll
    for (int i = 0; i < NT; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    for (int tap = 0; tap < 27; ++tap) {
        __syncthreads();
        const uint32_t* wt = reinterpret_cast<const uint32_t*>(w + size_t(tap) * Cout * Cin);
        for (int i = threadIdx.x; i < Cout * cw; i += blockDim.x) sw[(i / cw) * ldw + (i % cw)] = wt[i];
        __syncthreads();
        if (!live) continue;
        const int nA = rA < nvox ? nbr(zA, yA, xA, tap, n) : -1;
        const int nB = rB < nvox ? nbr(zB, yB, xB, tap, n) : -1;
        const bf16* pA = in + size_t(nA < 0 ? 0 : nA) * Cin + 2 * t;
        const bf16* pB = in + size_t(nB < 0 ? 0 : nB) * Cin + 2 * t;
        for (int c0 = 0; c0 < Cin; c0 += 16) {
            uint32_t a[4];
            a[0] = nA >= 0 ? ld32(pA + c0) : 0u;
            a[1] = nB >= 0 ? ld32(pB + c0) : 0u;
            a[2] = nA >= 0 ? ld32(pA + c0 + 8) : 0u;
            a[3] = nB >= 0 ? ld32(pB + c0 + 8) : 0u;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const uint32_t* row = sw + (nt * 8 + g) * ldw + c0 / 2 + t;
                const uint32_t b[2] = {row[0], row[4]};
                mma_bf16(acc[nt], a, b);
            }
        }
    }
    if (!live) return;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int co = nt * 8 + 2 * t;
        const float b0 = bias ? bias[co] : 0.f, b1 = bias ? bias[co + 1] : 0.f;
        float v[4] = {acc[nt][0] + b0, acc[nt][1] + b1, acc[nt][2] + b0, acc[nt][3] + b1};
        if (relu)
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = fmaxf(v[k], 0.f);
        if (rA < nvox) {
            *reinterpret_cast<uint32_t*>(out + size_t(rA) * Cout + co) =
                pack2(__float2bfloat16(v[0]), __float2bfloat16(v[1]));
            if (out32) {
                out32[size_t(rA) * Cout + co] = v[0];
                out32[size_t(rA) * Cout + co + 1] = v[1];
            }
        }
        if (rB < nvox) {
            *reinterpret_cast<uint32_t*>(out + size_t(rB) * Cout + co) =
                pack2(__float2bfloat16(v[2]), __float2bfloat16(v[3]));
            if (out32) {
                out32[size_t(rB) * Cout + co] = v[2];
                out32[size_t(rB) * Cout + co + 1] = v[3];
            }
        }
    }
}

template <int NT>
cudaError_t conv_fwd_t(const bf16* in, int Cin, const bf16* w, const float* bias, int Cout, int relu, bf16* out,
                       float* out32, int n, cudaStream_t s) {
    const size_t smem = sizeof(uint32_t) * size_t(Cout) * ((Cin + 8) / 2);
    cudaError_t e = qpat::allow_smem((const void*)k_conv_fwd<NT>, size_t(smem));
    if (e != cudaSuccess) return e;
    const int nvox = n * n * n;
    const int grid = (nvox + 16 * kConvWarps - 1) / (16 * kConvWarps);
    qpat::note_launch(1);
    k_conv_fwd<NT><<<grid, kConvWarps * 32, smem, s>>>(in, Cin, w, bias, Cout, relu, out, out32, n);
    return cudaGetLastError();
}

// partial[chunk][tap][co][ci] = sum_{v in chunk} dy[v][co] * in[nbr(v, tap)][ci]
constexpr int kWgradVox = 8192;  // voxels per chunk

template <int NCI>
__global__ void __launch_bounds__(128) k_conv_wgrad(const bf16* __restrict__ in, int Cin,
                                                    const bf16* __restrict__ dy, int Cout,
                                                    float* __restrict__ partial, int n) {
    __shared__ float red[16][NCI * 8 + 1];
    const int nvox = n * n * n;
    const int chunk = blockIdx.x, tap = blockIdx.y, co0 = blockIdx.z * 16;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int vbeg = chunk * kWgradVox, vend = min(nvox, vbeg + kWgradVox);
    float acc[NCI][4];
#pragma unroll
    for (int i = 0; i < NCI; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    for (int vb = vbeg + warp * 16; vb < vend; vb += 64) {
        // A (16 c_out x 16 voxels): A[co][v] = dy[v][co]
        const int va = vb + 2 * t, vc = vb + 2 * t + 8;
        uint32_t a[4];
        a[0] = pack2(dy[size_t(va) * Cout + co0 + g], dy[size_t(va + 1) * Cout + co0 + g]);
        a[1] = pack2(dy[size_t(va) * Cout + co0 + g + 8], dy[size_t(va + 1) * Cout + co0 + g + 8]);
        a[2] = pack2(dy[size_t(vc) * Cout + co0 + g], dy[size_t(vc + 1) * Cout + co0 + g]);
        a[3] = pack2(dy[size_t(vc) * Cout + co0 + g + 8], dy[size_t(vc + 1) * Cout + co0 + g + 8]);
        // B (16 voxels x 8 c_in): B[v][ci] = in[nbr(v, tap)][ci]
        int nb[4];
        const int vv[4] = {va, va + 1, vc, vc + 1};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int v = vv[k];
            nb[k] = nbr(v / (n * n), (v / n) % n, v % n, tap, n);
        }
        const bf16 zero = __float2bfloat16(0.f);
#pragma unroll
        for (int nc = 0; nc < NCI; ++nc) {
            const int ci = nc * 8 + g;
            const bf16 e0 = nb[0] >= 0 ? in[size_t(nb[0]) * Cin + ci] : zero;
            const bf16 e1 = nb[1] >= 0 ? in[size_t(nb[1]) * Cin + ci] : zero;
            const bf16 e2 = nb[2] >= 0 ? in[size_t(nb[2]) * Cin + ci] : zero;
            const bf16 e3 = nb[3] >= 0 ? in[size_t(nb[3]) * Cin + ci] : zero;
            const uint32_t b[2] = {pack2(e0, e1), pack2(e2, e3)};
            mma_bf16(acc[nc], a, b);
        }
    }
    // reduce the 4 warps in turn: C fragment rows co (g, g+8), columns ci (2t, 2t+1)
    for (int w = 0; w < 4; ++w) {
        if (warp == w) {
#pragma unroll
            for (int nc = 0; nc < NCI; ++nc) {
                const int c = nc * 8 + 2 * t;
                red[g][c] = (w ? red[g][c] : 0.f) + acc[nc][0];
                red[g][c + 1] = (w ? red[g][c + 1] : 0.f) + acc[nc][1];
                red[g + 8][c] = (w ? red[g + 8][c] : 0.f) + acc[nc][2];
                red[g + 8][c + 1] = (w ? red[g + 8][c + 1] : 0.f) + acc[nc][3];
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < 16 * Cin; i += blockDim.x) {
        const int r = i / Cin, c = i % Cin;
        partial[((size_t(chunk) * 27 + tap) * Cout + co0 + r) * Cin + c] = red[r][c];
    }
}

__global__ void k_sum_chunks(const float* partial, int chunks, int64_t count, float* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < chunks; ++c) s += partial[size_t(c) * count + i];
        out[i] = s;
    }
}

// db[co] = sum_v dy[v][co]
__global__ void k_bias_grad(const bf16* dy, int Cout, int nvox, float* db) {
    __shared__ float red[256];
    const int co = blockIdx.x;
    float s = 0.f;
    for (int v = threadIdx.x; v < nvox; v += blockDim.x) s += __bfloat162float(dy[size_t(v) * Cout + co]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[co] = red[0];
}

template <int NCI>
cudaError_t wgrad_t(const bf16* in, int Cin, const bf16* dy, int Cout, float* partial, int n, cudaStream_t s) {
    const int nvox = n * n * n;
    const int chunks = (nvox + kWgradVox - 1) / kWgradVox;
    dim3 grid(chunks, 27, Cout / 16);
    qpat::note_launch(1);
    k_conv_wgrad<NCI><<<grid, 128, 0, s>>>(in, Cin, dy, Cout, partial, n);
    return cudaGetLastError();
}

__global__ void k_flip(const bf16* w, int Cin, int Cout, bf16* wt) {
    const int64_t total = int64_t(27) * Cin * Cout;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        // wt[tap][ci][co] = w[26 - tap][co][ci]
        const int tap = int(i / (int64_t(Cin) * Cout));
        const int rem = int(i % (int64_t(Cin) * Cout));
        const int ci = rem / Cout, co = rem % Cout;
        wt[i] = w[(size_t(26 - tap) * Cout + co) * Cin + ci];
    }
}

__global__ void k_relu_mask(bf16* dy, const bf16* y, int64_t count) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
        if (!(__bfloat162float(y[i]) > 0.f)) dy[i] = __float2bfloat16(0.f);
}

__global__ void k_avgpool(const bf16* in, int C, int n, bf16* out) {
    const int m = n / 2;
    const int64_t total = int64_t(m) * m * m * C;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(i % C);
        const int64_t v = i / C;
        const int x = int(v % m), y = int((v / m) % m), z = int(v / (int64_t(m) * m));
        float s = 0.f;
        for (int d = 0; d < 8; ++d) {
            const int zz = 2 * z + (d >> 2), yy = 2 * y + ((d >> 1) & 1), xx = 2 * x + (d & 1);
            s += __bfloat162float(in[((size_t(zz) * n + yy) * n + xx) * C + c]);
        }
        out[i] = __float2bfloat16(0.125f * s);
    }
}

__global__ void k_avgpool_bwd(const bf16* dout, int C, int n, bf16* din, int accumulate) {
    const int m = n / 2;
    const int64_t total = int64_t(n) * n * n * C;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(i % C);
        const int64_t v = i / C;
        const int x = int(v % n), y = int((v / n) % n), z = int(v / (int64_t(n) * n));
        float g = 0.125f * __bfloat162float(dout[((size_t(z / 2) * m + y / 2) * m + x / 2) * C + c]);
        if (accumulate) g += __bfloat162float(din[i]);
        din[i] = __float2bfloat16(g);
    }
}

__global__ void k_upcat(const bf16* lo, int Clo, const bf16* skip, int Cs, int n, bf16* cat) {
    const int m = n / 2, C = Clo + Cs;
    const int64_t total = int64_t(n) * n * n * C;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(i % C);
        const int64_t v = i / C;
        if (c < Clo) {
            const int x = int(v % n), y = int((v / n) % n), z = int(v / (int64_t(n) * n));
            cat[i] = lo[((size_t(z / 2) * m + y / 2) * m + x / 2) * Clo + c];
        } else {
            cat[i] = skip[v * Cs + (c - Clo)];
        }
    }
}

__global__ void k_upcat_bwd_lo(const bf16* dcat, int Clo, int Cs, int n, bf16* dlo) {
    const int m = n / 2, C = Clo + Cs;
    const int64_t total = int64_t(m) * m * m * Clo;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(i % Clo);
        const int64_t v = i / Clo;
        const int x = int(v % m), y = int((v / m) % m), z = int(v / (int64_t(m) * m));
        float s = 0.f;
        for (int d = 0; d < 8; ++d) {
            const int zz = 2 * z + (d >> 2), yy = 2 * y + ((d >> 1) & 1), xx = 2 * x + (d & 1);
            s += __bfloat162float(dcat[((size_t(zz) * n + yy) * n + xx) * C + c]);
        }
        dlo[i] = __float2bfloat16(s);
    }
}

__global__ void k_upcat_bwd_skip(const bf16* dcat, int Clo, int Cs, int n, bf16* dskip, int accumulate) {
    const int C = Clo + Cs;
    const int64_t total = int64_t(n) * n * n * Cs;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(i % Cs);
        const int64_t v = i / Cs;
        float g = __bfloat162float(dcat[v * C + Clo + c]);
        if (accumulate) g += __bfloat162float(dskip[i]);
        dskip[i] = __float2bfloat16(g);
    }
}

__global__ void k_adam(float* w, bf16* wb, const float* g, float* m, float* v, int64_t count, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16(wi);
    }
}

__global__ void k_f2b(const float* in, bf16* out, int64_t count) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = __float2bfloat16(in[i]);
}

__global__ void k_b2f(const bf16* in, float* out, int64_t count) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = __bfloat162float(in[i]);
}

int grid1d(int64_t n) {
    return int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)));
}

}  // namespace

static int g_conv_engine = 0;
void set_conv_engine(int engine) { g_conv_engine = engine; }
int conv_engine() { return g_conv_engine; }

cudaError_t conv3d_fwd(const bf16* in, int Cin, const bf16* w, const float* bias, int Cout, int relu, bf16* out,
                       float* out32, int n, cudaStream_t s) {
    if (Cin % 16 || Cout % 8 || n % 2) return cudaErrorInvalidValue;
    if (g_conv_engine == 0 && conv3d_fwd_tc_supported(Cin, Cout))
        return conv3d_fwd_tc(in, Cin, w, bias, Cout, relu, out, out32, n, s);
    switch (Cout / 8) {
        case 1: return conv_fwd_t<1>(in, Cin, w, bias, Cout, relu, out, out32, n, s);
        case 2: return conv_fwd_t<2>(in, Cin, w, bias, Cout, relu, out, out32, n, s);
        case 4: return conv_fwd_t<4>(in, Cin, w, bias, Cout, relu, out, out32, n, s);
        case 6: return conv_fwd_t<6>(in, Cin, w, bias, Cout, relu, out, out32, n, s);
        case 8: return conv_fwd_t<8>(in, Cin, w, bias, Cout, relu, out, out32, n, s);
        case 12: return conv_fwd_t<12>(in, Cin, w, bias, Cout, relu, out, out32, n, s);
        case 16: return conv_fwd_t<16>(in, Cin, w, bias, Cout, relu, out, out32, n, s);
        case 24: return conv_fwd_t<24>(in, Cin, w, bias, Cout, relu, out, out32, n, s);
        default: return cudaErrorInvalidValue;
    }
}

int wgrad_chunks(int n) { return (n * n * n + kWgradVox - 1) / kWgradVox; }

cudaError_t conv3d_wgrad(const bf16* in, int Cin, const bf16* dy, int Cout, float* dw, float* db, float* partial,
                         int n, cudaStream_t s) {
    if (Cin % 8 || Cout % 16 || (n * n * n) % 16) return cudaErrorInvalidValue;
    cudaError_t e = cudaErrorInvalidValue;
    switch (Cin / 8) {
        case 2: e = wgrad_t<2>(in, Cin, dy, Cout, partial, n, s); break;
        case 4: e = wgrad_t<4>(in, Cin, dy, Cout, partial, n, s); break;
        case 6: e = wgrad_t<6>(in, Cin, dy, Cout, partial, n, s); break;
        case 8: e = wgrad_t<8>(in, Cin, dy, Cout, partial, n, s); break;
        case 12: e = wgrad_t<12>(in, Cin, dy, Cout, partial, n, s); break;
        case 16: e = wgrad_t<16>(in, Cin, dy, Cout, partial, n, s); break;
        case 24: e = wgrad_t<24>(in, Cin, dy, Cout, partial, n, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const int64_t count = int64_t(27) * Cout * Cin;
    qpat::note_launch(1);
    k_sum_chunks<<<grid1d(count), 256, 0, s>>>(partial, wgrad_chunks(n), count, dw);
    if (db) {
        qpat::note_launch(1);
        k_bias_grad<<<Cout, 256, 0, s>>>(dy, Cout, n * n * n, db);
    }
    return cudaGetLastError();
}

cudaError_t flip_weights(const bf16* w, int Cin, int Cout, bf16* w_t, cudaStream_t s) {
    qpat::note_launch(1);
    k_flip<<<grid1d(int64_t(27) * Cin * Cout), 256, 0, s>>>(w, Cin, Cout, w_t);
    return cudaGetLastError();
}

cudaError_t relu_mask(bf16* dy, const bf16* y, int64_t count, cudaStream_t s) {
    qpat::note_launch(1);
    k_relu_mask<<<grid1d(count), 256, 0, s>>>(dy, y, count);
    return cudaGetLastError();
}

cudaError_t avgpool(const bf16* in, int C, int n, bf16* out, cudaStream_t s) {
    qpat::note_launch(1);
    k_avgpool<<<grid1d(int64_t(n / 2) * (n / 2) * (n / 2) * C), 256, 0, s>>>(in, C, n, out);
    return cudaGetLastError();
}

cudaError_t avgpool_bwd(const bf16* dout, int C, int n, bf16* din, int accumulate, cudaStream_t s) {
    qpat::note_launch(1);
    k_avgpool_bwd<<<grid1d(int64_t(n) * n * n * C), 256, 0, s>>>(dout, C, n, din, accumulate);
    return cudaGetLastError();
}

cudaError_t upcat(const bf16* lo, int Clo, const bf16* skip, int Cs, int n, bf16* cat, cudaStream_t s) {
    qpat::note_launch(1);
    k_upcat<<<grid1d(int64_t(n) * n * n * (Clo + Cs)), 256, 0, s>>>(lo, Clo, skip, Cs, n, cat);
    return cudaGetLastError();
}

cudaError_t upcat_bwd(const bf16* dcat, int Clo, int Cs, int n, bf16* dlo, bf16* dskip, int accumulate_skip,
                      cudaStream_t s) {
    qpat::note_launch(1);
    k_upcat_bwd_lo<<<grid1d(int64_t(n / 2) * (n / 2) * (n / 2) * Clo), 256, 0, s>>>(dcat, Clo, Cs, n, dlo);
    qpat::note_launch(1);
    k_upcat_bwd_skip<<<grid1d(int64_t(n) * n * n * Cs), 256, 0, s>>>(dcat, Clo, Cs, n, dskip, accumulate_skip);
    return cudaGetLastError();
}

cudaError_t adam(float* w, bf16* wb, const float* g, float* m, float* v, int64_t count, float lr, float b1, float b2,
                 float eps, int step, cudaStream_t s) {
    const float c1 = 1.f - powf(b1, float(step)), c2 = 1.f - powf(b2, float(step));
    qpat::note_launch(1);
    k_adam<<<grid1d(count), 256, 0, s>>>(w, wb, g, m, v, count, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t f32_to_bf16(const float* in, bf16* out, int64_t count, cudaStream_t s) {
    qpat::note_launch(1);
    k_f2b<<<grid1d(count), 256, 0, s>>>(in, out, count);
    return cudaGetLastError();
}

cudaError_t bf16_to_f32(const bf16* in, float* out, int64_t count, cudaStream_t s) {
    qpat::note_launch(1);
    k_b2f<<<grid1d(count), 256, 0, s>>>(in, out, count);
    return cudaGetLastError();
}

}  // namespace unet
}  // namespace qpat
