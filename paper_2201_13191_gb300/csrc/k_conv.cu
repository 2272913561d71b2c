// 3x3 convolutions of the learned scatter denoiser on the tcgen05 tensor cores.
//
// Tensors are NHWC, BF16, with channel counts that are multiples of 16.
//  - forward: implicit GEMM.  A CTA owns 128 output pixels (M) and all output
//    channels (N <= 256, FP32 accumulators in tensor memory); K = 9 x C_in runs
//    over (tap, channel) in stages of 64, gathered with zero padding into a
//    shared-memory stage (two stages in flight), one thread issuing the MMAs
//    and committing each stage to its mbarrier.  Epilogue: bias, optional ReLU,
//    BF16 or FP32 store.
//  - input gradient: the same kernel with the weights flipped in space and
//    transposed in channels (a 3x3 'same' convolution's adjoint).
//  - weight gradient: dW[co][k] = sum_p dY[p][co] Xcol[p][k]; the tile is 128
//    rows of k by N = C_out, the reduction over pixels runs in stages of 64
//    pixels staged transposed into the K-major layout; CTAs split the pixels and
//    add their FP32 partial tiles into dW.
#include <cuda_bf16.h>
#include <stdint.h>

#include "mc_internal.h"
#include "mc_tc.cuh"

namespace mcx {
namespace {

constexpr int kM = 128;        // pixels (forward) or K rows (weight gradient) per CTA
constexpr int kStageK = 64;    // reduction elements per stage
constexpr int kKG = kStageK / 8;
constexpr int kThreads = 128;  // four warps: one per 32 tensor-memory lanes

template <int N>
struct ConvSmem {
  static constexpr int a_bytes = kM * kStageK * 2;  // 16 KB
  static constexpr int b_bytes = N * kStageK * 2;   // <= 32 KB
  static constexpr int stage_bytes = a_bytes + b_bytes;
  static constexpr int bytes = 2 * stage_bytes + 1024;  // + alignment slack
};

__device__ __forceinline__ uint32_t tmem_cols(int n) { return n <= 32 ? 32u : (uint32_t)n; }

template <int N>
__global__ void __launch_bounds__(kThreads) k_conv3x3_fwd(const ConvParams p) {
  extern __shared__ unsigned char dyn_raw[];
  unsigned char* dyn = reinterpret_cast<unsigned char*>(((uintptr_t)dyn_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_holder;
  __shared__ __align__(8) uint64_t mbar[2];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int K = 9 * p.cin;
  const int n_stages = (K + kStageK - 1) / kStageK;
  const long long npix = (long long)p.n * p.h * p.w;
  const long long pix0 = (long long)blockIdx.x * kM;

  if (warp == 0) tc::tmem_alloc(&tmem_holder, tmem_cols(N));
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_holder;

  // this thread's pixel (row of the A tile)
  const long long pr = pix0 + tid;
  const bool row_ok = pr < npix;
  int py = 0, px = 0, pn = 0;
  if (row_ok) {
    px = (int)(pr % p.w);
    const long long t = pr / p.w;
    py = (int)(t % p.h);
    pn = (int)(t / p.h);
  }
  bool ok = true;
  for (int st = 0; st < n_stages; ++st) {
    const int buf = st & 1;
    unsigned char* sA = dyn + buf * ConvSmem<N>::stage_bytes;
    unsigned char* sB = sA + ConvSmem<N>::a_bytes;
    if (st >= 2) ok &= tc::mbar_wait(&mbar[buf], (uint32_t)((st >> 1) - 1) & 1u);
    const int k0 = st * kStageK;
    // A: row = tid, eight 8-channel groups of (tap, channel)
#pragma unroll
    for (int kg = 0; kg < kKG; ++kg) {
      const int k = k0 + kg * 8;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (row_ok && k < K) {
        const int tap = k / p.cin, c = k - tap * p.cin;
        const int yy = py + tap / 3 - 1, xx = px + tap % 3 - 1;
        if (yy >= 0 && yy < p.h && xx >= 0 && xx < p.w)
          v = __ldg(reinterpret_cast<const uint4*>(p.x + (((long long)pn * p.h + yy) * p.w + xx) * p.cin + c));
      }
      *reinterpret_cast<uint4*>(sA + tc::canon_off(tid, kg * 8, kKG)) = v;
    }
    // B: N rows of the weights, K-major
    for (int q = tid; q < N * kKG; q += kThreads) {
      const int row = q / kKG, kg = q - row * kKG;
      const int k = k0 + kg * 8;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (k < K && row < p.cout) v = __ldg(reinterpret_cast<const uint4*>(p.wt + (long long)row * K + k));
      *reinterpret_cast<uint4*>(sB + tc::canon_off(row, kg * 8, kKG)) = v;
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const int nks = min(kStageK, K - k0) / 16;
      const uint32_t idesc = tc::idesc_bf16(kM, N);
      for (int ks = 0; ks < nks; ++ks) {
        const uint64_t da = tc::sdesc(tc::saddr(sA) + ks * 256, 128, kKG * 128);
        const uint64_t db = tc::sdesc(tc::saddr(sB) + ks * 256, 128, kKG * 128);
        tc::mma_bf16(tmem, da, db, idesc, (st > 0 || ks > 0) ? 1u : 0u);
      }
      tc::commit(&mbar[buf]);
    }
  }
  const int last = n_stages - 1;
  ok &= tc::mbar_wait(&mbar[last & 1], (uint32_t)(last >> 1) & 1u);
  // the other buffer's last commit precedes the final one, so it is complete too
  tc::fence_after();
  if (!ok && tid == 0) atomicOr(p.err, 1);
  if (ok) {
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 8) {
      float v[8];
      tc::tmem_ld8(lane_base + (uint32_t)c0, v);
      if (row_ok && c0 < p.cout) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (p.bias) v[j] += __ldg(p.bias + c0 + j);
          if (p.relu) v[j] = fmaxf(v[j], 0.f);
        }
        if (p.out_f32) {
          float* dst = reinterpret_cast<float*>(p.y) + pr * p.cout + c0;
          *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
          *reinterpret_cast<float4*>(dst + 4) = make_float4(v[4], v[5], v[6], v[7]);
        } else {
          __nv_bfloat162 b[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) b[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
          *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(p.y) + pr * p.cout + c0) =
              *reinterpret_cast<uint4*>(b);
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, tmem_cols(N));
}

// Weight gradient.  CTA (blockIdx.x = k tile, blockIdx.y = pixel split).
template <int N>
__global__ void __launch_bounds__(kThreads) k_conv3x3_wgrad(const WgradParams p) {
  extern __shared__ unsigned char dyn_raw[];
  unsigned char* dyn = reinterpret_cast<unsigned char*>(((uintptr_t)dyn_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_holder;
  __shared__ __align__(8) uint64_t mbar[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = 9 * p.cin;
  const int krow0 = blockIdx.x * kM;
  const long long npix = (long long)p.n * p.h * p.w;
  const long long chunk = (npix + gridDim.y - 1) / gridDim.y;
  const long long pbeg = (long long)blockIdx.y * chunk;
  const long long pend = min(npix, pbeg + chunk);
  const int n_stages = pend > pbeg ? (int)((pend - pbeg + kStageK - 1) / kStageK) : 0;

  if (warp == 0) tc::tmem_alloc(&tmem_holder, tmem_cols(N));
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_holder;
  bool ok = true;
  for (int st = 0; st < n_stages; ++st) {
    const int buf = st & 1;
    unsigned char* sA = dyn + buf * ConvSmem<N>::stage_bytes;
    unsigned char* sB = sA + ConvSmem<N>::a_bytes;
    if (st >= 2) ok &= tc::mbar_wait(&mbar[buf], (uint32_t)((st >> 1) - 1) & 1u);
    const long long q0 = pbeg + (long long)st * kStageK;
    // A[r][j] = X(pixel q0 + j shifted by tap(krow0 + r), channel(krow0 + r)): 16 row groups x 64 pixels
    for (int item = tid; item < (kM / 8) * kStageK; item += kThreads) {
      const int j = item % kStageK, rg = item / kStageK;
      const int k = krow0 + rg * 8;
      const long long q = q0 + j;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (k < K && q < pend) {
        const int tap = k / p.cin, c = k - tap * p.cin;
        const int qx = (int)(q % p.w);
        const long long t = q / p.w;
        const int qy = (int)(t % p.h), qn = (int)(t / p.h);
        const int yy = qy + tap / 3 - 1, xx = qx + tap % 3 - 1;
        if (yy >= 0 && yy < p.h && xx >= 0 && xx < p.w)
          v = __ldg(reinterpret_cast<const uint4*>(p.x + (((long long)qn * p.h + yy) * p.w + xx) * p.cin + c));
      }
      const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
      for (int i = 0; i < 8; ++i)
        *reinterpret_cast<__nv_bfloat16*>(sA + tc::canon_off(rg * 8 + i, j, kKG)) = e[i];
    }
    // B[co][j] = dY(pixel q0 + j, co)
    for (int item = tid; item < (N / 8) * kStageK; item += kThreads) {
      const int j = item % kStageK, cg = item / kStageK;
      const long long q = q0 + j;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (q < pend && cg * 8 < p.cout) v = __ldg(reinterpret_cast<const uint4*>(p.dy + q * p.cout + cg * 8));
      const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
      for (int i = 0; i < 8; ++i)
        *reinterpret_cast<__nv_bfloat16*>(sB + tc::canon_off(cg * 8 + i, j, kKG)) = e[i];
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t idesc = tc::idesc_bf16(kM, N);
      for (int ks = 0; ks < kStageK / 16; ++ks) {
        const uint64_t da = tc::sdesc(tc::saddr(sA) + ks * 256, 128, kKG * 128);
        const uint64_t db = tc::sdesc(tc::saddr(sB) + ks * 256, 128, kKG * 128);
        tc::mma_bf16(tmem, da, db, idesc, (st > 0 || ks > 0) ? 1u : 0u);
      }
      tc::commit(&mbar[buf]);
    }
  }
  if (n_stages > 0) {
    const int last = n_stages - 1;
    ok &= tc::mbar_wait(&mbar[last & 1], (uint32_t)(last >> 1) & 1u);
  }
  tc::fence_after();
  if (!ok && tid == 0) atomicOr(p.err, 1);
  if (ok && n_stages > 0) {
    const int k = krow0 + warp * 32 + lane;  // this lane's accumulator row
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 8) {
      float v[8];
      tc::tmem_ld8(lane_base + (uint32_t)c0, v);
      if (k < K)
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (c0 + j < p.cout) atomicAdd(p.dw + (long long)(c0 + j) * K + k, v[j]);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, tmem_cols(N));
}

template <int N>
cudaError_t launch_fwd_n(const ConvParams& p, cudaStream_t s) {
  const int smem = ConvSmem<N>::bytes;
  cudaError_t e = cudaFuncSetAttribute(k_conv3x3_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const long long npix = (long long)p.n * p.h * p.w;
  k_conv3x3_fwd<N><<<(unsigned)((npix + kM - 1) / kM), kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_wgrad_n(const WgradParams& p, int splits, cudaStream_t s) {
  const int smem = ConvSmem<N>::bytes;
  cudaError_t e = cudaFuncSetAttribute(k_conv3x3_wgrad<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int ktiles = (9 * p.cin + kM - 1) / kM;
  k_conv3x3_wgrad<N><<<dim3(ktiles, splits), kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

// N = cout rounded up to the tile widths 16/32/64/128/256 (cout multiple of 16).
cudaError_t launch_conv3x3_fwd(const ConvParams& p, cudaStream_t s) {
  if (p.cin % 16 || p.cout % 16 || p.cout > 256 || p.cin < 16) return cudaErrorInvalidValue;
  if (p.cout <= 16) return launch_fwd_n<16>(p, s);
  if (p.cout <= 32) return launch_fwd_n<32>(p, s);
  if (p.cout <= 64) return launch_fwd_n<64>(p, s);
  if (p.cout <= 128) return launch_fwd_n<128>(p, s);
  return launch_fwd_n<256>(p, s);
}

cudaError_t launch_conv3x3_wgrad(const WgradParams& p, int splits, cudaStream_t s) {
  if (p.cin % 16 || p.cout % 16 || p.cout > 256 || p.cin < 16 || splits < 1) return cudaErrorInvalidValue;
  if (p.cout <= 16) return launch_wgrad_n<16>(p, splits, s);
  if (p.cout <= 32) return launch_wgrad_n<32>(p, splits, s);
  if (p.cout <= 64) return launch_wgrad_n<64>(p, splits, s);
  if (p.cout <= 128) return launch_wgrad_n<128>(p, splits, s);
  return launch_wgrad_n<256>(p, splits, s);
}

}  // namespace mcx
