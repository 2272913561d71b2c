// Element-wise, pooling, resampling, loss and optimiser kernels of the learned
// scatter denoiser (NHWC tensors; activations BF16, gradients FP32).
#include <cuda_bf16.h>
#include <stdint.h>

#include "mc_nn.h"

namespace mcx {
namespace nn {
namespace {

__device__ __forceinline__ size_t gtid() { return (size_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ size_t gstride() { return (size_t)gridDim.x * blockDim.x; }
__device__ __forceinline__ __nv_bfloat16 to_bf(float v) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ __nv_bfloat16 to_bf(__nv_bfloat16 v) { return v; }

int blocks_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

// Per-image scale: s[i] = mean of the image (floored at tiny > 0).
__global__ void k_image_mean(const float* __restrict__ img, int hw, float* __restrict__ s) {
  __shared__ float red[256];
  const float* im = img + (size_t)blockIdx.x * hw;
  float acc = 0.f;
  for (int i = threadIdx.x; i < hw; i += blockDim.x) acc += im[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) s[blockIdx.x] = fmaxf(red[0] / (float)hw, 1e-30f);
}

// x[n][y][x][0] = img / s, other 15 channels 0.
__global__ void k_pack_input(const float* __restrict__ img, const float* __restrict__ s, int n, int hw,
                             __nv_bfloat16* __restrict__ x) {
  for (size_t i = gtid(); i < (size_t)n * hw; i += gstride()) {
    const int b = (int)(i / hw);
    __align__(16) __nv_bfloat16 v[16];
    v[0] = __float2bfloat16_rn(img[i] / s[b]);
#pragma unroll
    for (int c = 1; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
    uint4* dst = reinterpret_cast<uint4*>(x + i * 16);
    dst[0] = reinterpret_cast<uint4*>(v)[0];
    dst[1] = reinterpret_cast<uint4*>(v)[1];
  }
}

// out = s * (img / s + net[...][0]) = img + s * net[...][0]   (residual output)
__global__ void k_unpack_output(const float* __restrict__ img, const float* __restrict__ s,
                                const float* __restrict__ net, int n, int hw, float* __restrict__ out) {
  for (size_t i = gtid(); i < (size_t)n * hw; i += gstride()) {
    const int b = (int)(i / hw);
    out[i] = img[i] + s[b] * net[i * 16];
  }
}

// Loss = mean over pixels of (x/s + net0 - y/s)^2; gradient into g[...][0].
__global__ void k_mse(const float* __restrict__ img, const float* __restrict__ tgt, const float* __restrict__ s,
                      const float* __restrict__ net, int n, int hw, float* __restrict__ g, double* __restrict__ loss) {
  __shared__ double red[256];
  const float inv = 1.f / (float)((size_t)n * hw);
  double acc = 0.0;
  for (size_t i = gtid(); i < (size_t)n * hw; i += gstride()) {
    const int b = (int)(i / hw);
    const float d = img[i] / s[b] + net[i * 16] - tgt[i] / s[b];
    acc += (double)d * d;
    float* gi = g + i * 16;
    gi[0] = 2.f * d * inv;
#pragma unroll
    for (int c = 1; c < 16; ++c) gi[c] = 0.f;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] * inv);
}

// gb = bf16(g * [y > 0]) (mask by the ReLU whose output is y), or plain conversion when y is null.
__global__ void k_relu_mask(const float* __restrict__ g, const __nv_bfloat16* __restrict__ y, size_t n,
                            __nv_bfloat16* __restrict__ gb) {
  for (size_t i = gtid(); i < n; i += gstride()) {
    const float v = (y == nullptr || __bfloat162float(y[i]) > 0.f) ? g[i] : 0.f;
    gb[i] = __float2bfloat16_rn(v);
  }
}

// 2x2 max pooling (h, w even).
__global__ void k_pool_fwd(const __nv_bfloat16* __restrict__ x, int n, int h, int w, int c,
                           __nv_bfloat16* __restrict__ y) {
  const int ho = h / 2, wo = w / 2;
  for (size_t i = gtid(); i < (size_t)n * ho * wo * c; i += gstride()) {
    const int ch = (int)(i % c);
    size_t t = i / c;
    const int xo = (int)(t % wo);
    t /= wo;
    const int yo = (int)(t % ho), b = (int)(t / ho);
    const __nv_bfloat16* base = x + (((size_t)b * h + 2 * yo) * w + 2 * xo) * c + ch;
    float m = __bfloat162float(base[0]);
    m = fmaxf(m, __bfloat162float(base[c]));
    m = fmaxf(m, __bfloat162float(base[(size_t)w * c]));
    m = fmaxf(m, __bfloat162float(base[(size_t)w * c + c]));
    y[i] = __float2bfloat16_rn(m);
  }
}

// Routes each pooled gradient to the first maximal input of its 2x2 window;
// adds into gx (which may already hold another contribution).
__global__ void k_pool_bwd(const __nv_bfloat16* __restrict__ x, const float* __restrict__ gy, int n, int h, int w,
                           int c, float* __restrict__ gx) {
  const int ho = h / 2, wo = w / 2;
  for (size_t i = gtid(); i < (size_t)n * ho * wo * c; i += gstride()) {
    const int ch = (int)(i % c);
    size_t t = i / c;
    const int xo = (int)(t % wo);
    t /= wo;
    const int yo = (int)(t % ho), b = (int)(t / ho);
    const size_t o0 = (((size_t)b * h + 2 * yo) * w + 2 * xo) * c + ch;
    const size_t idx[4] = {o0, o0 + c, o0 + (size_t)w * c, o0 + (size_t)w * c + c};
    int best = 0;
    float m = __bfloat162float(x[idx[0]]);
    for (int k = 1; k < 4; ++k) {
      const float v = __bfloat162float(x[idx[k]]);
      if (v > m) {
        m = v;
        best = k;
      }
    }
    gx[idx[best]] += gy[i];
  }
}

// Nearest 2x up-sampling into channels [c_off, c_off + c) of a tensor with ctot channels.
__global__ void k_up_fwd(const __nv_bfloat16* __restrict__ x, int n, int h, int w, int c,
                         __nv_bfloat16* __restrict__ y, int ctot, int c_off) {
  const int H = 2 * h, W = 2 * w;
  for (size_t i = gtid(); i < (size_t)n * H * W * c; i += gstride()) {
    const int ch = (int)(i % c);
    size_t t = i / c;
    const int X = (int)(t % W);
    t /= W;
    const int Y = (int)(t % H), b = (int)(t / H);
    y[(((size_t)b * H + Y) * W + X) * ctot + c_off + ch] = x[(((size_t)b * h + Y / 2) * w + X / 2) * c + ch];
  }
}

// Gradient of the up-sampling: sums 2x2 blocks of channels [c_off, c_off + c) of g (ctot channels).
__global__ void k_up_bwd(const float* __restrict__ g, int n, int h, int w, int c, int ctot, int c_off,
                         float* __restrict__ gx) {
  const int H = 2 * h, W = 2 * w;
  for (size_t i = gtid(); i < (size_t)n * h * w * c; i += gstride()) {
    const int ch = (int)(i % c);
    size_t t = i / c;
    const int xx = (int)(t % w);
    t /= w;
    const int yy = (int)(t % h), b = (int)(t / h);
    float acc = 0.f;
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) acc += g[(((size_t)b * H + 2 * yy + dy) * W + 2 * xx + dx) * ctot + c_off + ch];
    gx[i] = acc;
  }
}

// Copy x (c channels) into channels [c_off, c_off + c) of y (ctot channels).
__global__ void k_copy_channels(const __nv_bfloat16* __restrict__ x, size_t npix, int c,
                                __nv_bfloat16* __restrict__ y, int ctot, int c_off) {
  for (size_t i = gtid(); i < npix * c; i += gstride()) {
    const size_t p = i / c;
    y[p * ctot + c_off + (i % c)] = x[i];
  }
}

// gx (c channels) += channels [c_off, c_off + c) of g (ctot channels).
__global__ void k_add_channels(const float* __restrict__ g, size_t npix, int ctot, int c_off, int c,
                               float* __restrict__ gx) {
  for (size_t i = gtid(); i < npix * c; i += gstride()) {
    const size_t p = i / c;
    gx[i] += g[p * ctot + c_off + (i % c)];
  }
}

// db[c] += sum over pixels of gb[p][c] (BF16 gradient as fed to the weight gradient).
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ gb, size_t npix, int c, float* __restrict__ db) {
  const int ch = threadIdx.x % c;
  const int lanes = blockDim.x / c;
  float acc = 0.f;
  for (size_t p = (size_t)blockIdx.x * lanes + threadIdx.x / c; p < npix; p += (size_t)gridDim.x * lanes)
    acc += __bfloat162float(gb[p * c + ch]);
  if ((int)threadIdx.x < lanes * c) atomicAdd(db + ch, acc);
}

// Adam on FP32 master weights; also writes the BF16 forward copy.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16* __restrict__ wb) {
  for (size_t i = gtid(); i < n; i += gstride()) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
  }
}

// Weights in the operand order of the tensor-core convolution (k_conv.cu):
// wm[ci / 8][tap][co][ci % 8], i.e. for every 8-channel input group and tap a
// column of 16-byte rows, one per output channel.  wf: the forward operator
// from w[co][tap][ci].  wa: the adjoint (input gradient of a 3x3 'same'
// convolution), the operator with C_in' = cout, C_out' = cin and weights
// w'[ci][tap][co] = w[co][8 - tap][ci], in the same order:
// wa[co / 8][tap][ci][co % 8].  Either output may be null.
template <class T>
__global__ void k_pack_weights(const T* __restrict__ w, int cout, int cin, __nv_bfloat16* __restrict__ wf,
                               __nv_bfloat16* __restrict__ wa) {
  const size_t n = (size_t)cout * 9 * cin;
  for (size_t i = gtid(); i < n; i += gstride()) {
    const int ci = (int)(i % cin);
    const size_t t = i / cin;
    const int tap = (int)(t % 9), co = (int)(t / 9);
    const __nv_bfloat16 v = to_bf(w[i]);
    if (wf) wf[(((size_t)(ci >> 3) * 9 + tap) * cout + co) * 8 + (ci & 7)] = v;
    if (wa) wa[(((size_t)(co >> 3) * 9 + (8 - tap)) * cin + ci) * 8 + (co & 7)] = v;
  }
}

}  // namespace

#define NN_LAUNCH(kernel, n, ...)                                \
  do {                                                           \
    kernel<<<blocks_for(n), 256, 0, s>>>(__VA_ARGS__);           \
    return cudaGetLastError();                                   \
  } while (0)

cudaError_t image_mean(const float* img, int n, int hw, float* scale, cudaStream_t s) {
  k_image_mean<<<n, 256, 0, s>>>(img, hw, scale);
  return cudaGetLastError();
}
cudaError_t pack_input(const float* img, const float* scale, int n, int hw, __nv_bfloat16* x, cudaStream_t s) {
  NN_LAUNCH(k_pack_input, (size_t)n * hw, img, scale, n, hw, x);
}
cudaError_t unpack_output(const float* img, const float* scale, const float* net, int n, int hw, float* out,
                          cudaStream_t s) {
  NN_LAUNCH(k_unpack_output, (size_t)n * hw, img, scale, net, n, hw, out);
}
cudaError_t mse(const float* img, const float* tgt, const float* scale, const float* net, int n, int hw, float* g,
                double* loss, cudaStream_t s) {
  NN_LAUNCH(k_mse, (size_t)n * hw, img, tgt, scale, net, n, hw, g, loss);
}
cudaError_t relu_mask(const float* g, const __nv_bfloat16* y, size_t n, __nv_bfloat16* gb, cudaStream_t s) {
  NN_LAUNCH(k_relu_mask, n, g, y, n, gb);
}
cudaError_t pool_fwd(const __nv_bfloat16* x, int n, int h, int w, int c, __nv_bfloat16* y, cudaStream_t s) {
  NN_LAUNCH(k_pool_fwd, (size_t)n * (h / 2) * (w / 2) * c, x, n, h, w, c, y);
}
cudaError_t pool_bwd(const __nv_bfloat16* x, const float* gy, int n, int h, int w, int c, float* gx, cudaStream_t s) {
  NN_LAUNCH(k_pool_bwd, (size_t)n * (h / 2) * (w / 2) * c, x, gy, n, h, w, c, gx);
}
cudaError_t up_fwd(const __nv_bfloat16* x, int n, int h, int w, int c, __nv_bfloat16* y, int ctot, int c_off,
                   cudaStream_t s) {
  NN_LAUNCH(k_up_fwd, (size_t)n * 4 * h * w * c, x, n, h, w, c, y, ctot, c_off);
}
cudaError_t up_bwd(const float* g, int n, int h, int w, int c, int ctot, int c_off, float* gx, cudaStream_t s) {
  NN_LAUNCH(k_up_bwd, (size_t)n * h * w * c, g, n, h, w, c, ctot, c_off, gx);
}
cudaError_t copy_channels(const __nv_bfloat16* x, size_t npix, int c, __nv_bfloat16* y, int ctot, int c_off,
                          cudaStream_t s) {
  NN_LAUNCH(k_copy_channels, npix * c, x, npix, c, y, ctot, c_off);
}
cudaError_t add_channels(const float* g, size_t npix, int ctot, int c_off, int c, float* gx, cudaStream_t s) {
  NN_LAUNCH(k_add_channels, npix * c, g, npix, ctot, c_off, c, gx);
}
cudaError_t bias_grad(const __nv_bfloat16* gb, size_t npix, int c, float* db, cudaStream_t s) {
  const int threads = (256 / c) * c;
  k_bias_grad<<<304, threads, 0, s>>>(gb, npix, c, db);
  return cudaGetLastError();
}
cudaError_t adam(float* w, const float* g, float* m, float* v, size_t n, float lr, int step, __nv_bfloat16* wb,
                 cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  NN_LAUNCH(k_adam, n, w, g, m, v, n, lr, b1, b2, 1e-8f, c1, c2, wb);
}
cudaError_t pack_weights(const float* w, int cout, int cin, __nv_bfloat16* wf, __nv_bfloat16* wa, cudaStream_t s) {
  NN_LAUNCH(k_pack_weights<float>, (size_t)cout * 9 * cin, w, cout, cin, wf, wa);
}
cudaError_t pack_weights_bf16(const __nv_bfloat16* w, int cout, int cin, __nv_bfloat16* wf, cudaStream_t s) {
  NN_LAUNCH(k_pack_weights<__nv_bfloat16>, (size_t)cout * 9 * cin, w, cout, cin, wf, nullptr);
}

}  // namespace nn
}  // namespace mcx
