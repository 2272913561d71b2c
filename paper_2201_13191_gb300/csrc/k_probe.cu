// Measurement helper with no counterpart in the paper: random 4-byte gathers
// from a device buffer, i.e. the access pattern of the transport's voxel reads
// without the march arithmetic around them.  Timed on a buffer the size of the
// packed volume, it gives the voxel-gather roofline a measured peak at the
// memory level the volume lives in (L2 when it fits, HBM otherwise).
//
// Each thread draws its indices from a 32-bit xorshift generator seeded by its
// global index and keeps eight independent loads in flight (the transport
// keeps up to eight gathers of a ray in flight).  The loaded words are folded
// into one value per thread written to `sink`, so no load can be elided.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mc_internal.h"

namespace {

__device__ __forceinline__ uint32_t xorshift32(uint32_t s) {
  s ^= s << 13;
  s ^= s >> 17;
  s ^= s << 5;
  return s;
}

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

}  // namespace

extern "C" int mc_probe_gather(const void* buf, uint64_t n_words, int rounds, int grid, int block, uint32_t* sink,
                               void* stream) {
  if (!buf || !sink || n_words < 1 || n_words > 0xFFFFFFFFull || rounds < 1 || grid < 1 || block < 32 ||
      block > 256 || block % 32)
    return MC_ERR_INVALID_ARG;
  (void)cudaGetLastError();
  k_probe_gather<<<grid, block, 0, (cudaStream_t)stream>>>((const uint32_t*)buf, (uint32_t)n_words, rounds, sink);
  return cudaGetLastError() == cudaSuccess ? MC_OK : MC_ERR_CUDA;
}
