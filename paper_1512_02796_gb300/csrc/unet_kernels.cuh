// BF16 tensor-core kernels of the 3D U-Net that supplies the initial guess
// of the forward solves (not part of the paper; the solve it feeds is the
// Appendix's K^-1 f).
//
// Activations are channels-last bf16 tensors [voxel][C] of one n^3 grid;
// convolutions are 3x3x3 with zero padding, written as implicit GEMMs
// (rows = voxels, columns = output channels, reduction = 27 taps x input
// channels): the forward convolution on tcgen05.mma with a tensor-memory
// accumulator (unet_tc.cu) where the shape allows, else mma.sync m16n8k16
// bf16 -> fp32; the weight gradient on mma.sync.  Weights are stored
// [tap][c_out][c_in] (c_in fastest), tap = (dz + 1) * 9 + (dy + 1) * 3 + dx + 1.
#pragma once

#include <cuda_bf16.h>

namespace qpat {
void note_launch(int n);  // launch counter (abi.cu)
cudaError_t allow_smem(const void* func, size_t smem);  // dynamic shared memory permission (abi.cu)
}
#include <cuda_runtime.h>

#include <cstdint>

namespace qpat {
namespace unet {

cudaError_t conv3d_fwd(const __nv_bfloat16* in, int Cin, const __nv_bfloat16* w, const float* bias, int Cout,
                       int relu, __nv_bfloat16* out, float* out_f32, int n, cudaStream_t s);
// the same convolution on tcgen05 tensor cores with a TMEM accumulator
// (unet_tc.cu); shapes: Cin % 16 == 0, Cout % 16 == 0, 16 <= Cout <= 256
bool conv3d_fwd_tc_supported(int Cin, int Cout);
cudaError_t conv3d_fwd_tc(const __nv_bfloat16* in, int Cin, const __nv_bfloat16* w, const float* bias, int Cout,
                          int relu, __nv_bfloat16* out, float* out_f32, int n, cudaStream_t s);
int tc_timeouts();  // bounded waits of the tcgen05 kernel that gave up (device counter)
// convolution engine: 0 = tcgen05 where the shape allows, else mma.sync; 1 = mma.sync only
void set_conv_engine(int engine);
int conv_engine();
// weight gradient (fp32, [tap][c_out][c_in]) of a conv whose input was `in`
// and whose output gradient (already masked by the ReLU) is `dy`; `partial`
// must hold chunks(n) * 27 * Cout * Cin floats
cudaError_t conv3d_wgrad(const __nv_bfloat16* in, int Cin, const __nv_bfloat16* dy, int Cout, float* dw,
                         float* db, float* partial, int n, cudaStream_t s);
int wgrad_chunks(int n);
// w_t[tap][c_in][c_out] = w[26 - tap][c_out][c_in]  (the data-gradient conv)
cudaError_t flip_weights(const __nv_bfloat16* w, int Cin, int Cout, __nv_bfloat16* w_t, cudaStream_t s);
// dy *= (y > 0)
cudaError_t relu_mask(__nv_bfloat16* dy, const __nv_bfloat16* y, int64_t count, cudaStream_t s);
// 2x2x2 average pooling n^3 -> (n/2)^3 and its gradient
cudaError_t avgpool(const __nv_bfloat16* in, int C, int n, __nv_bfloat16* out, cudaStream_t s);
cudaError_t avgpool_bwd(const __nv_bfloat16* dout, int C, int n, __nv_bfloat16* din, int accumulate,
                        cudaStream_t s);
// nearest upsampling (n/2)^3 -> n^3 of `lo` into channels [0, Clo) of `cat`,
// and `skip` into channels [Clo, Clo + Cs)
cudaError_t upcat(const __nv_bfloat16* lo, int Clo, const __nv_bfloat16* skip, int Cs, int n, __nv_bfloat16* cat,
                  cudaStream_t s);
// gradient of upcat: dlo (sum over the 8 children), dskip (+)= the skip channels
cudaError_t upcat_bwd(const __nv_bfloat16* dcat, int Clo, int Cs, int n, __nv_bfloat16* dlo, __nv_bfloat16* dskip,
                      int accumulate_skip, cudaStream_t s);
// Adam on fp32 master weights; refreshes the bf16 copy
cudaError_t adam(float* w, __nv_bfloat16* wb, const float* g, float* m, float* v, int64_t count, float lr,
                 float b1, float b2, float eps, int step, cudaStream_t s);
cudaError_t f32_to_bf16(const float* in, __nv_bfloat16* out, int64_t count, cudaStream_t s);
cudaError_t bf16_to_f32(const __nv_bfloat16* in, float* out, int64_t count, cudaStream_t s);

}  // namespace unet
}  // namespace qpat
