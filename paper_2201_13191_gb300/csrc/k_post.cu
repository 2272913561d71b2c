// Smoothing and dual interpolation of the simulated scatter (arXiv 2201.13191
// Sec. II-C.3 and II-C.4): separable Savitzky-Golay smoothing, then linear
// interpolation between simulated angles fused with separable Keys cubic
// up-sampling.  All passes are bandwidth bound: the smoothing keeps its small
// coefficient matrix in shared memory and each thread owns consecutive outputs
// along the fastest axis; the up-sampling runs separable and row-tiled (the
// low-resolution rows a block needs are interpolated along x into shared
// memory once), with a per-pixel fallback when those rows do not fit.
#include <stdint.h>

#include <cmath>

#include "mc_internal.h"

namespace mcx {
namespace {

constexpr int kMaxWin = 31;

// Rows: out[i][y][x] = sum_j H[p][j] in[i][y][s + j], s = clamp(x - m, 0, w - win), p = x - s.
// H is the win x win least-squares "hat" matrix of the polynomial fit: row m
// is the interior filter, rows < m / > m fit the first / last window (edges).
__global__ void k_sg_rows(const float* __restrict__ in, float* __restrict__ out, int n_img, int h, int w,
                          const float* __restrict__ coef, int win) {
  __shared__ float H[kMaxWin * kMaxWin];
  for (int q = threadIdx.x; q < win * win; q += blockDim.x) H[q] = coef[q];
  __syncthreads();
  const int m = win / 2;
  const size_t total = (size_t)n_img * h * w;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(idx % w);
    const float* row = in + (idx - x);
    const int s = min(max(x - m, 0), w - win);
    const float* hp = H + (x - s) * win;
    float acc = 0.f;
    for (int j = 0; j < win; ++j) acc = fmaf(hp[j], __ldg(row + s + j), acc);
    out[idx] = acc;
  }
}

// Columns: out[i][y][x] = sum_j H[p][j] in[i][s + j][x], s = clamp(y - m, 0, h - win).
__global__ void k_sg_cols(const float* __restrict__ in, float* __restrict__ out, int n_img, int h, int w,
                          const float* __restrict__ coef, int win) {
  __shared__ float H[kMaxWin * kMaxWin];
  for (int q = threadIdx.x; q < win * win; q += blockDim.x) H[q] = coef[q];
  __syncthreads();
  const int m = win / 2;
  const size_t total = (size_t)n_img * h * w;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(idx % w);
    const size_t iy = idx / w;
    const int y = (int)(iy % h);
    const float* img = in + (iy - y) * w;
    const int s = min(max(y - m, 0), h - win);
    const float* hp = H + (y - s) * win;
    float acc = 0.f;
    for (int j = 0; j < win; ++j) acc = fmaf(hp[j], __ldg(img + (size_t)(s + j) * w + x), acc);
    out[idx] = acc;
  }
}

// Keys cubic convolution weights for taps at offsets -1, 0, 1, 2 from floor(x).
__device__ __forceinline__ void keys_weights(float t, float a, float wt[4]) {
  const float d0 = 1.f + t, d1 = t, d2 = 1.f - t, d3 = 2.f - t;
  wt[0] = ((a * d0 - 5.f * a) * d0 + 8.f * a) * d0 - 4.f * a;
  wt[1] = ((a + 2.f) * d1 - (a + 3.f)) * d1 * d1 + 1.f;
  wt[2] = ((a + 2.f) * d2 - (a + 3.f)) * d2 * d2 + 1.f;
  wt[3] = ((a * d3 - 5.f * a) * d3 + 8.f * a) * d3 - 4.f * a;
}

// out[o][Y][X] = sum_ty sum_tx wy wx ((1-f) in[a0][y][x] + f in[a1][y][x]),
// source coordinate (X + 1/2) nu/NU - 1/2, taps clamped to the image.
// Each thread produces 4 consecutive X (one 16-byte store when aligned).
__global__ void k_lerp_upsample(const float* __restrict__ in, int nv, int nu, float* __restrict__ out, int n_out,
                                int NV, int NU, const int* __restrict__ a0s, const int* __restrict__ a1s,
                                const float* __restrict__ fas, float a) {
  const int qx = (NU + 3) / 4;
  const size_t total = (size_t)n_out * NV * qx;
  const float sx = (float)nu / (float)NU, sy = (float)nv / (float)NV;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int X0 = (int)(idx % qx) * 4;
    const size_t r = idx / qx;
    const int Y = (int)(r % NV);
    const int o = (int)(r / NV);
    const float* A = in + (size_t)__ldg(a0s + o) * nu * nv;
    const float* B = in + (size_t)__ldg(a1s + o) * nu * nv;
    const float f = __ldg(fas + o);
    const float yy = fmaf((float)Y + 0.5f, sy, -0.5f);
    const float yf = floorf(yy);
    float wy[4];
    keys_weights(yy - yf, a, wy);
    int ys[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) ys[k] = min(max((int)yf - 1 + k, 0), nv - 1);
    float res[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int X = X0 + e;
      const float xx = fmaf((float)min(X, NU - 1) + 0.5f, sx, -0.5f);
      const float xf = floorf(xx);
      float wx[4];
      keys_weights(xx - xf, a, wx);
      float acc = 0.f;
#pragma unroll
      for (int ky = 0; ky < 4; ++ky) {
        const size_t ro = (size_t)ys[ky] * nu;
        float racc = 0.f;
#pragma unroll
        for (int kx = 0; kx < 4; ++kx) {
          const int xi = min(max((int)xf - 1 + kx, 0), nu - 1);
          const float v = fmaf(f, __ldg(B + ro + xi) - __ldg(A + ro + xi), __ldg(A + ro + xi));
          racc = fmaf(wx[kx], v, racc);
        }
        acc = fmaf(wy[ky], racc, acc);
      }
      res[e] = acc;
    }
    float* dst = out + ((size_t)o * NV + Y) * NU + X0;
    if (X0 + 3 < NU && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
      *reinterpret_cast<float4*>(dst) = make_float4(res[0], res[1], res[2], res[3]);
    } else {
      for (int e = 0; e < 4 && X0 + e < NU; ++e) dst[e] = res[e];
    }
  }
}

// The same interpolation, separable and row-tiled: a block makes kUpRows
// output rows of one output angle.  It first interpolates between the two
// angles every low-resolution row those output rows touch (lr[j][x] for input
// row r0 + j, clamped: one read of each input value), then along x from there
// into shared memory (xr[j][X]), then each output pixel takes its four y taps
// from xr.  The sums run in the same order as in k_lerp_upsample (x taps
// inside, y taps outside, the angle lerp of each tap first), so the images
// agree bit for bit, with 4 instead of 16 taps per output pixel and the
// low-resolution reads shared by the block.
constexpr int kUpRows = 32;
__global__ void __launch_bounds__(256) k_lerp_upsample_rows(const float* __restrict__ in, int nv, int nu,
                                                            float* __restrict__ out, int NV, int NU,
                                                            const int* __restrict__ a0s, const int* __restrict__ a1s,
                                                            const float* __restrict__ fas, float a) {
  extern __shared__ __align__(16) float xr[];  // [rows][NU], then lr [rows][nu]
  const int o = blockIdx.y;
  const int Y0 = blockIdx.x * kUpRows, Y1 = min(Y0 + kUpRows, NV);
  const float sx = (float)nu / (float)NU, sy = (float)nv / (float)NV;
  const int r0 = (int)floorf(fmaf((float)Y0 + 0.5f, sy, -0.5f)) - 1;
  const int r1 = (int)floorf(fmaf((float)(Y1 - 1) + 0.5f, sy, -0.5f)) + 2;
  const int nrows = r1 - r0 + 1;
  const float* A = in + (size_t)__ldg(a0s + o) * nu * nv;
  const float* B = in + (size_t)__ldg(a1s + o) * nu * nv;
  const float f = __ldg(fas + o);
  // angle pass: the lerped low-resolution rows, each input value read once
  float* lr = xr + (size_t)nrows * NU;
  for (int q = threadIdx.x; q < nrows * nu; q += blockDim.x) {
    const int j = q / nu, x = q - j * nu;
    const size_t i = (size_t)min(max(r0 + j, 0), nv - 1) * nu + x;
    lr[q] = fmaf(f, __ldg(B + i) - __ldg(A + i), __ldg(A + i));
  }
  __syncthreads();
  // x pass: a column's taps and weights once, then every row
  for (int X = threadIdx.x; X < NU; X += blockDim.x) {
    const float xx = fmaf((float)X + 0.5f, sx, -0.5f);
    const float xf = floorf(xx);
    float wx[4];
    keys_weights(xx - xf, a, wx);
    int xi[4];
#pragma unroll
    for (int kx = 0; kx < 4; ++kx) xi[kx] = min(max((int)xf - 1 + kx, 0), nu - 1);
    for (int j = 0; j < nrows; ++j) {
      const float* row = lr + j * nu;
      float racc = 0.f;
#pragma unroll
      for (int kx = 0; kx < 4; ++kx) racc = fmaf(wx[kx], row[xi[kx]], racc);
      xr[j * NU + X] = racc;
    }
  }
  __syncthreads();
  // y pass: a row's weights once, then four consecutive outputs per thread (one 16-byte store)
  const bool vec = (NU & 3) == 0 && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
  for (int Y = Y0; Y < Y1; ++Y) {
    const float yy = fmaf((float)Y + 0.5f, sy, -0.5f);
    const float yf = floorf(yy);
    float wy[4];
    keys_weights(yy - yf, a, wy);
    const float* rows = xr + ((int)yf - 1 - r0) * NU;
    float* dst = out + ((size_t)o * NV + Y) * NU;
    if (vec) {
      for (int X = 4 * threadIdx.x; X < NU; X += 4 * blockDim.x) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ky = 0; ky < 4; ++ky) {
          const float4 v = *reinterpret_cast<const float4*>(rows + ky * NU + X);
          acc[0] = fmaf(wy[ky], v.x, acc[0]);
          acc[1] = fmaf(wy[ky], v.y, acc[1]);
          acc[2] = fmaf(wy[ky], v.z, acc[2]);
          acc[3] = fmaf(wy[ky], v.w, acc[3]);
        }
        *reinterpret_cast<float4*>(dst + X) = make_float4(acc[0], acc[1], acc[2], acc[3]);
      }
    } else {
      for (int X = threadIdx.x; X < NU; X += blockDim.x) {
        float acc = 0.f;
#pragma unroll
        for (int ky = 0; ky < 4; ++ky) acc = fmaf(wy[ky], rows[ky * NU + X], acc);
        dst[X] = acc;
      }
    }
  }
}

int grid_for(size_t n, int block) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = (n + block - 1) / block;
  const size_t cap = (size_t)sms * 8;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t launch_sg_rows(const float* in, float* out, int n_img, int h, int w, const float* coef, int win,
                           cudaStream_t s) {
  if (win > kMaxWin) return cudaErrorInvalidValue;
  k_sg_rows<<<grid_for((size_t)n_img * h * w, 256), 256, 0, s>>>(in, out, n_img, h, w, coef, win);
  return cudaGetLastError();
}

cudaError_t launch_sg_cols(const float* in, float* out, int n_img, int h, int w, const float* coef, int win,
                           cudaStream_t s) {
  if (win > kMaxWin) return cudaErrorInvalidValue;
  k_sg_cols<<<grid_for((size_t)n_img * h * w, 256), 256, 0, s>>>(in, out, n_img, h, w, coef, win);
  return cudaGetLastError();
}

cudaError_t launch_lerp_upsample(const float* in, int nv, int nu, float* out, int n_out, int NV, int NU,
                                 const int* a0, const int* a1, const float* fa, float cubic_a, cudaStream_t s) {
  // row-tiled form when the low-resolution rows one block touches fit in shared memory
  const double sy = (double)nv / (double)NV;
  const int rows = (int)std::ceil((kUpRows - 1) * sy) + 5;
  const size_t smem = (size_t)rows * (NU + nu) * 4;
  if (n_out <= 65535 && smem <= 160 * 1024) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_lerp_upsample_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    k_lerp_upsample_rows<<<dim3((NV + kUpRows - 1) / kUpRows, n_out), 256, smem, s>>>(in, nv, nu, out, NV, NU, a0, a1,
                                                                                        fa, cubic_a);
    return cudaGetLastError();
  }
  const size_t total = (size_t)n_out * NV * ((NU + 3) / 4);
  k_lerp_upsample<<<grid_for(total, 256), 256, 0, s>>>(in, nv, nu, out, n_out, NV, NU, a0, a1, fa, cubic_a);
  return cudaGetLastError();
}

}  // namespace mcx
