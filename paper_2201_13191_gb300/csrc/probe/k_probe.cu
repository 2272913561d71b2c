// Measurement kernels with no counterpart in the paper, built into their own
// library (libmcprobe.so) beside the product library.  They give the rooflines
// of the benchmark measured denominators on the GPU at hand:
//
//   mc_probe_stream  coalesced 16-byte reads over a buffer, pass after pass:
//                    the streaming read bandwidth of the memory level the
//                    buffer lives in (L2 when it fits, HBM otherwise);
//   mc_probe_gather  random 4-byte loads over a buffer, eight in flight per
//                    thread: the access pattern of the transport's voxel reads
//                    without the march arithmetic around them;
//   mc_probe_mma     tcgen05.mma issue rate of one instruction shape.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../../include/mc_probe.h"
#include "../mc_tc.cuh"

namespace {

__device__ __forceinline__ uint32_t xorshift32(uint32_t s) {
  s ^= s << 13;
  s ^= s >> 17;
  s ^= s << 5;
  return s;
}

// Each thread draws its indices from a 32-bit xorshift generator seeded by its
// global index and keeps eight independent loads in flight.  The loaded words
// are folded into one value per thread written to `sink`, so no load can be
// elided.
__global__ void __launch_bounds__(256) k_probe_gather(const uint32_t* __restrict__ buf, uint32_t n_words,
                                                      int rounds, uint32_t* __restrict__ sink) {
  const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t s = (gid + 1u) * 0x9E3779B9u;
  s = s ? s : 1u;
  uint32_t acc = 0u;
#pragma unroll 1
  for (int r = 0; r < rounds; ++r) {
    uint32_t idx[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      s = xorshift32(s);
      idx[j] = (uint32_t)(((uint64_t)s * n_words) >> 32);  // < n_words
    }
    uint32_t v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __ldg(buf + idx[j]);
#pragma unroll
    for (int j = 0; j < 8; ++j) acc = acc * 31u + v[j];
  }
  sink[gid] = acc;
}

// Coalesced streaming reads: the grid walks the buffer in 16-byte words with
// a grid-stride loop, four loads in flight per thread, `passes` times; the
// words are xor-folded into one value per thread so no load can be elided.
__global__ void __launch_bounds__(256) k_probe_stream(const uint4* __restrict__ buf, size_t n16, int passes,
                                                      uint32_t* __restrict__ sink) {
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  uint32_t acc = 0u;
#pragma unroll 1
  for (int p = 0; p < passes; ++p) {
    size_t i = gid;
    for (; i + 3 * stride < n16; i += 4 * stride) {
      const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride), c = __ldcg(buf + i + 2 * stride),
                  d = __ldcg(buf + i + 3 * stride);
      acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
    }
    for (; i < n16; i += stride) {
      const uint4 a = __ldcg(buf + i);
      acc ^= a.x ^ a.y ^ a.z ^ a.w;
    }
  }
  sink[gid] = acc;
}

// Tensor-core issue-rate probe: one CTA per SM issues `rounds` x 4 MMAs
// (M = 128, N, K = 16 each; BF16 operands resident in shared memory, FP32
// accumulator in tensor memory) and waits for them: the sustained rate of the
// instruction shape the convolution kernels use, which depends on N.
template <int N>
__global__ void __launch_bounds__(128, 1) k_probe_mma(int rounds, int* err) {
  extern __shared__ __align__(1024) unsigned char dyn[];
  __shared__ uint32_t holder;
  __shared__ __align__(8) uint64_t bar;
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr int kBytes = (128 * 64 + N * 64) * 2;  // A: 128 x 64, B: N x 64 (BF16, zeros)
  for (int i = tid; i < kBytes / 16; i += 128) reinterpret_cast<uint4*>(dyn)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) mcx::tc::tmem_alloc(&holder, N < 32 ? 32u : (uint32_t)N);
  if (tid == 0) mcx::tc::mbar_init(&bar, 1);
  mcx::tc::fence_async_smem();
  mcx::tc::fence_before();
  __syncthreads();
  mcx::tc::fence_after();
  const uint32_t tmem = holder;
  if (tid == 0) {
    const uint32_t a0 = mcx::tc::saddr(dyn), b0 = a0 + 128 * 64 * 2;
    const uint32_t idesc = mcx::tc::idesc_bf16(128, N);
    for (int r = 0; r < rounds; ++r)
      for (int ks = 0; ks < 4; ++ks)
        mcx::tc::mma_bf16(tmem, mcx::tc::sdesc(a0 + ks * 256, 128, 1024), mcx::tc::sdesc(b0 + ks * 256, 128, 1024),
                          idesc, (r | ks) ? 1u : 0u);
    mcx::tc::commit(&bar);
  }
  __syncwarp();
  if (!mcx::tc::mbar_wait(&bar, 0) && tid == 0) atomicOr(err, 1);
  mcx::tc::fence_before();
  __syncthreads();
  if (warp == 0) mcx::tc::tmem_free(tmem, N < 32 ? 32u : (uint32_t)N);
}

template <int N>
cudaError_t launch_probe_mma(int grid, int rounds, int* err, cudaStream_t s) {
  const int smem = (128 * 64 + N * 64) * 2;
  cudaError_t e = cudaFuncSetAttribute(k_probe_mma<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_probe_mma<N><<<grid, 128, smem, s>>>(rounds, err);
  return cudaGetLastError();
}

}  // namespace

extern "C" int mc_probe_mma(int n, int grid, int rounds, int* err, void* stream) {
  if (!err || grid < 1 || rounds < 1) return MC_PROBE_ERR_INVALID_ARG;
  (void)cudaGetLastError();
  const cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  switch (n) {
    case 16: e = launch_probe_mma<16>(grid, rounds, err, s); break;
    case 32: e = launch_probe_mma<32>(grid, rounds, err, s); break;
    case 64: e = launch_probe_mma<64>(grid, rounds, err, s); break;
    case 128: e = launch_probe_mma<128>(grid, rounds, err, s); break;
    case 256: e = launch_probe_mma<256>(grid, rounds, err, s); break;
    default: return MC_PROBE_ERR_INVALID_ARG;
  }
  return e == cudaSuccess ? MC_PROBE_OK : MC_PROBE_ERR_CUDA;
}

extern "C" int mc_probe_gather(const void* buf, uint64_t n_words, int rounds, int grid, int block, uint32_t* sink,
                               void* stream) {
  if (!buf || !sink || n_words < 1 || n_words > 0xFFFFFFFFull || rounds < 1 || grid < 1 || block < 32 ||
      block > 256 || block % 32)
    return MC_PROBE_ERR_INVALID_ARG;
  (void)cudaGetLastError();
  k_probe_gather<<<grid, block, 0, (cudaStream_t)stream>>>((const uint32_t*)buf, (uint32_t)n_words, rounds, sink);
  return cudaGetLastError() == cudaSuccess ? MC_PROBE_OK : MC_PROBE_ERR_CUDA;
}

extern "C" int mc_probe_stream(const void* buf, uint64_t n_bytes, int passes, int grid, int block, uint32_t* sink,
                               void* stream) {
  if (!buf || !sink || n_bytes < 16 || n_bytes % 16 || ((uintptr_t)buf & 15u) || passes < 1 || grid < 1 ||
      block < 32 || block > 256 || block % 32)
    return MC_PROBE_ERR_INVALID_ARG;
  (void)cudaGetLastError();
  k_probe_stream<<<grid, block, 0, (cudaStream_t)stream>>>((const uint4*)buf, (size_t)(n_bytes / 16), passes, sink);
  return cudaGetLastError() == cudaSuccess ? MC_PROBE_OK : MC_PROBE_ERR_CUDA;
}
