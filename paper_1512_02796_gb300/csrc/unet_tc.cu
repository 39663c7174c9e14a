// 3x3x3 BF16 convolution of the U-Net on the 5th-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory), the forward kernel the
// U-Net's inference and data-gradient passes use on sm_100-class GPUs.
//
// Implicit GEMM: D[128 voxels][Cout] = sum over 27 taps of
// A_tap[128 voxels][Cin] x B_tap[Cin][Cout], with A_tap the input rows of the
// tap's neighbours (zero outside the grid) and B_tap = w[tap] stored
// [Cout][Cin] (Cin contiguous: a K-major B operand).  One CTA (4 warps)
// computes one 128-voxel tile for all output channels:
//   per tap: the 128 threads write A_tap and B_tap into shared memory in the
//   canonical no-swizzle K-major layout (8 x 16-byte core matrices, K-adjacent
//   core matrices 128 bytes apart, row-group stride = K/8 x 128 bytes), fence
//   the writes to the async proxy and synchronise; one thread issues Cin/16
//   tcgen05.mma (M = 128, N = Cout, K = 16, BF16 x BF16 -> FP32) and commits
//   them to an mbarrier that all threads wait on (bounded) before the tile
//   buffers are rewritten.
//   epilogue: each warp reads its 32 TMEM lanes (= 32 voxels) with
//   tcgen05.ld 32x32b, adds the bias, applies ReLU and stores BF16 / FP32.
// Tensor memory (Cout columns rounded up to a power of two >= 32) is
// allocated by warp 0 and freed on every exit path.  A wait that gives up
// writes NaN into the tile (the caller's parity checks see it) and counts
// the event in g_tc_timeouts.
#include <cstdint>

#include "unet_kernels.cuh"

namespace qpat {
namespace unet {

namespace {

using bf16 = __nv_bfloat16;

constexpr int kTcThreads = 128;
constexpr int kTcRows = 128;  // voxels per CTA = MMA M
constexpr long long kTcSpin = 1LL << 22;

__device__ int g_tc_timeouts;

__device__ __forceinline__ uint32_t s_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: no swizzle, K-major; lbo = byte distance
// of K-adjacent core matrices, sbo = byte distance of 8-row groups
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= uint64_t((addr & 0x3FFFF) >> 4);          // bits  0-13: start address / 16
    d |= uint64_t((lbo & 0x3FFFF) >> 4) << 16;     // bits 16-29: leading byte offset / 16
    d |= uint64_t((sbo & 0x3FFFF) >> 4) << 32;     // bits 32-45: stride byte offset / 16
    d |= uint64_t(1) << 46;                        // bits 46-47: descriptor version (sm_100)
    return d;                                      // base offset 0, no swizzle
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4)                      // D format: F32
           | (1u << 7)                    // A format: BF16
           | (1u << 10)                   // B format: BF16
           | (uint32_t(N >> 3) << 17)     // N / 8
           | (uint32_t(M >> 4) << 24);    // M / 16
}

__device__ __forceinline__ int tap_nbr(int v, int tap, int n) {
    const int z = v / (n * n), y = (v / n) % n, x = v % n;
    const int zz = z + tap / 9 - 1, yy = y + (tap / 3) % 3 - 1, xx = x + tap % 3 - 1;
    if (zz < 0 || yy < 0 || xx < 0 || zz >= n || yy >= n || xx >= n) return -1;
    return (zz * n + yy) * n + xx;
}

// byte offset of element (row, k) in a no-swizzle K-major tile with K columns
__device__ __forceinline__ uint32_t core_off(int row, int k, int K) {
    return uint32_t(((row >> 3) * (K >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ bool mbar_wait_parity(uint64_t* bar, uint32_t parity) {
    for (long long i = 0; i < kTcSpin; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(s_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

template <int NCOLS>
__global__ void __launch_bounds__(kTcThreads) k_conv_fwd_tc(const bf16* __restrict__ in, int Cin,
                                                            const bf16* __restrict__ w,
                                                            const float* __restrict__ bias, int Cout, int relu,
                                                            bf16* __restrict__ out, float* __restrict__ out32,
                                                            int n) {
    extern __shared__ __align__(128) unsigned char tc_smem[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_base_s;
    __shared__ int s_ok;
    // two stages (taps alternate): A 128 x Cin bf16, then B Cout x Cin bf16
    const size_t a_bytes = size_t(kTcRows) * Cin * 2, stage_bytes = a_bytes + size_t(Cout) * Cin * 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int v0 = blockIdx.x * kTcRows;
    const int nvox = n * n * n;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&tmem_base_s)),
                     "r"(NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_s;
    const uint32_t idesc = instr_desc(kTcRows, Cout);
    const int kc = Cin / 8;  // 16-byte chunks per row
    // completion of tap t's MMAs: phase (t / 2) of mbar[t % 2]
    auto wait_tap = [&](int t) { return mbar_wait_parity(&mbar[t & 1], uint32_t((t >> 1) & 1)); };

    int tap = 0;
    for (; tap < 27; ++tap) {
        unsigned char* sA = tc_smem + size_t(tap & 1) * stage_bytes;
        unsigned char* sB = sA + a_bytes;
        // the stage is rewritten only after the MMAs of tap - 2 have read it
        if (tap >= 2 && !wait_tap(tap - 2)) s_ok = 0;
        __syncthreads();
        if (!s_ok) break;
        // ---- stage A_tap (own row: one voxel's neighbour) and B_tap
        {
            const int v = v0 + threadIdx.x;
            const int nb = v < nvox ? tap_nbr(v, tap, n) : -1;
            const uint4* src = reinterpret_cast<const uint4*>(in + size_t(nb < 0 ? 0 : nb) * Cin);
            for (int c = 0; c < kc; ++c) {
                const uint4 val = nb >= 0 ? __ldg(src + c) : make_uint4(0, 0, 0, 0);
                *reinterpret_cast<uint4*>(sA + core_off(threadIdx.x, c * 8, Cin)) = val;
            }
            const uint4* wsrc = reinterpret_cast<const uint4*>(w + size_t(tap) * Cout * Cin);
            for (int i = threadIdx.x; i < Cout * kc; i += kTcThreads) {
                const int row = i / kc, c = i % kc;
                *reinterpret_cast<uint4*>(sB + core_off(row, c * 8, Cin)) = __ldg(wsrc + i);
            }
        }
        // generic-proxy writes of the tiles -> visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = s_addr(sA), b0 = s_addr(sB);
            const uint32_t sbo = uint32_t(Cin / 8) * 128u;
            for (int k = 0; k < Cin / 16; ++k) {
                const uint64_t da = smem_desc(a0 + uint32_t(k) * 256u, 128u, sbo);
                const uint64_t db = smem_desc(b0 + uint32_t(k) * 256u, 128u, sbo);
                const uint32_t acc = (tap > 0 || k > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             s_addr(&mbar[tap & 1]))
                         : "memory");
        }
    }
    // the last two taps' MMAs (or, after a give-up, those in flight) finish
    // before TMEM is read and freed; each wait is bounded
    {
        const int last = s_ok ? 26 : tap - 1;
        bool fin = true;
        if (last >= 1 && !wait_tap(last - 1)) fin = false;
        if (last >= 0 && !wait_tap(last)) fin = false;
        if (!fin) s_ok = 0;
        __syncthreads();
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // ---- epilogue: warp w owns TMEM lanes (voxels) 32w .. 32w + 31
    const int v = v0 + warp * 32 + lane;
    const bool ok = s_ok != 0;
    if (!ok && threadIdx.x == 0) atomicAdd(&g_tc_timeouts, 1);
    for (int c0 = 0; c0 < Cout; c0 += 16) {
        uint32_t r[16];
        const uint32_t taddr = tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (v >= nvox) continue;
        float f[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            float x = ok ? __uint_as_float(r[j]) : __int_as_float(0x7fc00000);
            if (bias) x += bias[c0 + j];
            if (relu) x = fmaxf(x, 0.f);
            f[j] = x;
        }
        uint32_t packed[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
            packed[j] = *reinterpret_cast<const uint32_t*>(&h);
        }
        uint4* o = reinterpret_cast<uint4*>(out + size_t(v) * Cout + c0);
        o[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        o[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        if (out32) {
            float4* o32 = reinterpret_cast<float4*>(out32 + size_t(v) * Cout + c0);
#pragma unroll
            for (int j = 0; j < 4; ++j) o32[j] = make_float4(f[4 * j], f[4 * j + 1], f[4 * j + 2], f[4 * j + 3]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
}

template <int NCOLS>
cudaError_t conv_fwd_tc_t(const bf16* in, int Cin, const bf16* w, const float* bias, int Cout, int relu, bf16* out,
                          float* out32, int n, cudaStream_t s) {
    const size_t smem = 2 * (size_t(kTcRows) * Cin * 2 + size_t(Cout) * Cin * 2);
    cudaError_t e = qpat::allow_smem((const void*)k_conv_fwd_tc<NCOLS>, size_t(smem));
    if (e != cudaSuccess) return e;
    const int nvox = n * n * n;
    qpat::note_launch(1);
    k_conv_fwd_tc<NCOLS><<<(nvox + kTcRows - 1) / kTcRows, kTcThreads, smem, s>>>(in, Cin, w, bias, Cout, relu, out,
                                                                                 out32, n);
    return cudaGetLastError();
}

}  // namespace

bool conv3d_fwd_tc_supported(int Cin, int Cout) {
    // M = 128 needs N = Cout a multiple of 16 in [16, 256]; K steps of 16
    return Cin % 16 == 0 && Cout % 16 == 0 && Cout >= 16 && Cout <= 256 &&
           2 * (size_t(kTcRows) * Cin * 2 + size_t(Cout) * Cin * 2) <= 200 * 1024;
}

cudaError_t conv3d_fwd_tc(const bf16* in, int Cin, const bf16* w, const float* bias, int Cout, int relu, bf16* out,
                          float* out32, int n, cudaStream_t s) {
    if (!conv3d_fwd_tc_supported(Cin, Cout)) return cudaErrorInvalidValue;
    if (Cout <= 32) return conv_fwd_tc_t<32>(in, Cin, w, bias, Cout, relu, out, out32, n, s);
    if (Cout <= 64) return conv_fwd_tc_t<64>(in, Cin, w, bias, Cout, relu, out, out32, n, s);
    if (Cout <= 128) return conv_fwd_tc_t<128>(in, Cin, w, bias, Cout, relu, out, out32, n, s);
    return conv_fwd_tc_t<256>(in, Cin, w, bias, Cout, relu, out, out32, n, s);
}

int tc_timeouts() {
    int h = 0;
    cudaMemcpyFromSymbol(&h, g_tc_timeouts, sizeof(int));
    return h;
}

}  // namespace unet
}  // namespace qpat
