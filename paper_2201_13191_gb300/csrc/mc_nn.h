// Launch wrappers of the denoiser's element-wise kernels (k_nn.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

namespace mcx {
namespace nn {

cudaError_t image_mean(const float* img, int n, int hw, float* scale, cudaStream_t s);
cudaError_t pack_input(const float* img, const float* scale, int n, int hw, __nv_bfloat16* x, cudaStream_t s);
cudaError_t unpack_output(const float* img, const float* scale, const float* net, int n, int hw, float* out,
                          cudaStream_t s);
cudaError_t mse(const float* img, const float* tgt, const float* scale, const float* net, int n, int hw, float* g,
                double* loss, cudaStream_t s);
cudaError_t relu_mask(const float* g, const __nv_bfloat16* y, size_t n, __nv_bfloat16* gb, cudaStream_t s);
cudaError_t pool_fwd(const __nv_bfloat16* x, int n, int h, int w, int c, __nv_bfloat16* y, cudaStream_t s);
cudaError_t pool_bwd(const __nv_bfloat16* x, const float* gy, int n, int h, int w, int c, float* gx, cudaStream_t s);
cudaError_t up_fwd(const __nv_bfloat16* x, int n, int h, int w, int c, __nv_bfloat16* y, int ctot, int c_off,
                   cudaStream_t s);
cudaError_t up_bwd(const float* g, int n, int h, int w, int c, int ctot, int c_off, float* gx, cudaStream_t s);
cudaError_t copy_channels(const __nv_bfloat16* x, size_t npix, int c, __nv_bfloat16* y, int ctot, int c_off,
                          cudaStream_t s);
cudaError_t add_channels(const float* g, size_t npix, int ctot, int c_off, int c, float* gx, cudaStream_t s);
cudaError_t bias_grad(const __nv_bfloat16* gb, size_t npix, int c, float* db, cudaStream_t s);
cudaError_t adam(float* w, const float* g, float* m, float* v, size_t n, float lr, int step, __nv_bfloat16* wb,
                 cudaStream_t s);
// Tensor-core operand order of the convolution weights (forward wf and adjoint
// wa, either nullable): wf[ci/8][tap][co][ci%8], wa[co/8][8-tap][ci][co%8].
cudaError_t pack_weights(const float* w, int cout, int cin, __nv_bfloat16* wf, __nv_bfloat16* wa, cudaStream_t s);
cudaError_t pack_weights_bf16(const __nv_bfloat16* w, int cout, int cin, __nv_bfloat16* wf, cudaStream_t s);

}  // namespace nn
}  // namespace mcx
