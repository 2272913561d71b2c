// Primary image, eq. (Ip) of arXiv 2201.13191 Sec. II-A: for every pixel the
// ray from the source to the pixel centre is marched with the fixed step
// (Sec. II-C.2); the per-material column masses rho*L are summed exactly in
// 64-bit fixed point (each FP16 density is an integer multiple of 2^-24), and
// the spectrum sum S(E) eta(E) exp(-mu(E) L) runs over the energy bins.  The
// file also builds the packed voxel words and measures, at volume load, how
// often neighbouring voxels change material.
#include <cuda_fp16.h>
#include <stdint.h>

#include "mc_device.cuh"

namespace mcx {
namespace {

constexpr float kPi = 3.14159265358979f;
#ifndef MC_PRIMARY_AHEAD
#define MC_PRIMARY_AHEAD 16
#endif
constexpr int kAhead = MC_PRIMARY_AHEAD;  // voxel words in flight per ray

// FP16 bit pattern -> value * 2^24 as an exact integer (finite, non-negative inputs).
__device__ __forceinline__ unsigned long long fp16_fixed24(uint16_t b) {
  const uint32_t e = (b >> 10) & 31u, f = b & 1023u;
  return e == 0 ? (unsigned long long)f : ((unsigned long long)(f | 1024u) << (e - 1));
}

// Column masses per material: a run of voxels of one material is summed in a
// register and added to its material's total when the material changes.  With
// SACC the totals live in shared memory (one add wherever the run ends), which
// suits volumes whose material changes often (a segmented reconstruction's
// misclassified voxels); otherwise in registers, selected by a switch, which
// leaves the L1 cache its full size.  Both sum the same integers exactly.
template <int LAYOUT, bool SACC>
__global__ void __launch_bounds__(256) k_primary(const PrimaryParams P) {
  // shared: [n_bins][n_mat] 0.1 * mu/rho at each bin energy, then (SACC)
  // [n_mat][blockDim] this block's per-thread totals
  extern __shared__ __align__(8) unsigned char s_raw[];
  const int nm = P.tab.n_mat, nb = P.spec.n_bins, ns = P.tab.n_stage;
  float* s_mub = reinterpret_cast<float*>(s_raw);
  unsigned long long* my_acc =
      reinterpret_cast<unsigned long long*>(s_raw + (((size_t)nb * nm * 4 + 7) & ~(size_t)7)) + threadIdx.x;
  if (SACC)
    for (int m = 0; m < nm; ++m) my_acc[m * blockDim.x] = 0ull;
  for (int q = threadIdx.x; q < nb * nm; q += blockDim.x) {
    const int n = q / nm, m = q % nm;
    const float E = P.spec.energy[n];
    const float x = (E - P.tab.E0) * P.tab.inv_dE;
    const int i = max(0, min(__float2int_rd(x), ns - 2));
    const float f = x - (float)i;
    const float2 v = P.tab.blob[(TAB_TOT * nm + m) * ns + i];
    s_mub[q] = 0.1f * fmaf(f, v.y, v.x);
  }
  __syncthreads();
  const GeomView& G = P.geo;
  const VolumeView& V = P.vol;
  const int npix = G.nu * G.nv;
  const int a = blockIdx.y;
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  const int i = pix % G.nu, j = pix / G.nu;
  // Ray from the source to the pixel centre, parameterised from its point o
  // closest to the isocentre (|o| is at most the volume's half diagonal), so
  // that the chord and the midpoints carry rounding of the volume's size, not
  // of the source distance.  With n = (cos b, sin b, 0), e_u = (-sin b, cos b, 0):
  //   D = X - s = -SDD n + u e_u + v e_z,  d^2 = SDD^2 + u^2 + v^2,
  //   o = s - (s.w) w = (SOD / d^2) ((u^2 + v^2) n + SDD (u e_u + v e_z)),
  // both free of cancellation; the source sits at t = -SOD SDD / d.
  float sb, cb;
  sincosf(__ldg(P.angles + a), &sb, &cb);
  const float u = ((float)i + 0.5f - 0.5f * (float)G.nu) * G.pu;
  const float v = ((float)j + 0.5f - 0.5f * (float)G.nv) * G.pv;
  const float r2 = fmaf(u, u, v * v);
  const float d2 = fmaf(G.sdd, G.sdd, r2);
  const float d = sqrtf(d2);
  const float3 w = make_float3(fmaf(-G.sdd, cb, -u * sb) / d, fmaf(-G.sdd, sb, u * cb) / d, v / d);
  const float k = G.sod / d2;
  const float3 o = make_float3(k * fmaf(r2, cb, -G.sdd * (u * sb)), k * fmaf(r2, sb, G.sdd * (u * cb)),
                               k * (G.sdd * v));
  const float t_src = -G.sod * G.sdd / d;
  unsigned long long acc[kMaxMat];
#pragma unroll
  for (int m = 0; m < kMaxMat; ++m) acc[m] = 0ull;
  float ta, tb, h = 0.f;
  if (clip_box(V, o, w, t_src, t_src + d, ta, tb)) {
    const float L = tb - ta;
    const int n = step_count(L, P.step);
    h = L / (float)n;
    VoxRay r;
    r.set(V, o, w);
    int cur = vox_mat(__ldg(V.vox + r.voxel<LAYOUT>(V, fmaf(0.5f, h, ta))));
    unsigned long long run = 0ull;
    // the words of the next kAhead midpoints are loaded before any is used (the
    // step positions are known in advance, so the gathers are independent);
    // midpoints past the chord's end repeat its last one and are not summed
    for (int k0 = 0; k0 < n; k0 += kAhead) {
      uint32_t wd[kAhead];
#pragma unroll
      for (int u = 0; u < kAhead; ++u) {
        const int kk = min(k0 + u, n - 1);
        wd[u] = __ldg(V.vox + r.voxel<LAYOUT>(V, fmaf((float)kk + 0.5f, h, ta)));
      }
#pragma unroll
      for (int u = 0; u < kAhead; ++u) {
        if (k0 + u < n) {
          const int m = vox_mat(wd[u]);
          if (m != cur) {
            if (SACC) my_acc[cur * blockDim.x] += run;
            else switch (cur) {
              case 0: acc[0] += run; break;
              case 1: acc[1] += run; break;
              case 2: acc[2] += run; break;
              case 3: acc[3] += run; break;
              case 4: acc[4] += run; break;
              case 5: acc[5] += run; break;
              case 6: acc[6] += run; break;
              default: acc[7] += run; break;
            }
            cur = m;
            run = 0ull;
          }
          run += fp16_fixed24((uint16_t)(wd[u] & 0xffffu));
        }
      }
    }
    if (SACC) {
      my_acc[cur * blockDim.x] += run;
    } else {
#pragma unroll
      for (int q = 0; q < kMaxMat; ++q) acc[q] += (q == cur) ? run : 0ull;
    }
  }
  float rl[kMaxMat];
#pragma unroll
  for (int m = 0; m < kMaxMat; ++m) {
    const unsigned long long t = SACC ? (m < nm ? my_acc[m * blockDim.x] : 0ull) : acc[m];
    rl[m] = (float)t * 5.9604644775390625e-08f * h;  // 2^-24
  }
  // spectrum sum of eq. (Ip), compensated (Kahan) so that its rounding stays
  // at a few units in the last place whatever the number of bins
  float sum = 0.f, comp = 0.f;
  for (int n = 0; n < nb; ++n) {
    const float S = __ldg(P.spec.sn + n);
    if (S == 0.f) continue;
    float tau = 0.f;
#pragma unroll
    for (int m = 0; m < kMaxMat; ++m)
      if (m < nm) tau = fmaf(s_mub[n * nm + m], rl[m], tau);
    const float y = S * __ldg(P.spec.eta + n) * expf(-tau) - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
  }
  // pixel area x obliquity / (4 pi d^2), obliquity = SDD / d
  P.out[(size_t)a * npix + pix] = sum * ((G.pu * G.pv) * G.sdd) / ((4.f * kPi) * (d2 * d));
}

}  // namespace

cudaError_t launch_primary(const PrimaryParams& p, cudaStream_t s) {
  const int block = 256;
  const int npix = p.geo.nu * p.geo.nv;
  dim3 grid((npix + block - 1) / block, p.n_angles);
  const int smem = ((p.spec.n_bins * p.tab.n_mat * 4 + 7) & ~7) + (p.shared_acc ? p.tab.n_mat * block * 8 : 0);
  const bool brick = p.vol.layout == VOX_BRICK;
  auto k = brick ? (p.shared_acc ? k_primary<VOX_BRICK, true> : k_primary<VOX_BRICK, false>)
                 : (p.shared_acc ? k_primary<VOX_LIN, true> : k_primary<VOX_LIN, false>);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  k<<<grid, block, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace mcx

// Fraction of x-neighbour voxel pairs whose materials differ (how often a ray
// meets a material change); chooses the primary kernel's accumulator variant.
namespace mcx {
namespace {
__global__ void k_mat_changes(const uint8_t* __restrict__ mat, size_t n, int nx, unsigned long long* count) {
  unsigned long long c = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i + 1 < n; i += (size_t)gridDim.x * blockDim.x)
    c += (i % (size_t)nx != (size_t)nx - 1) && mat[i] != mat[i + 1];
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}
}  // namespace

cudaError_t material_change_fraction(const uint8_t* mat, int nx, int ny, int nz, cudaStream_t s, double* frac) {
  *frac = 0.0;
  const size_t n = (size_t)nx * ny * nz;
  const size_t pairs = n - (size_t)ny * nz;
  if (pairs == 0) return cudaSuccess;
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d, 8, s);
  if (e != cudaSuccess) return e;
  unsigned long long h = 0;
  e = cudaMemsetAsync(d, 0, 8, s);
  if (e == cudaSuccess) {
    k_mat_changes<<<152 * 8, 256, 0, s>>>(mat, n, nx, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, 8, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  *frac = (double)h / (double)pairs;
  return e;
}
}  // namespace mcx

// Device-side validation of a volume given by device pointers: every material
// id below n_mat and every density a finite, non-negative binary16.
namespace mcx {
namespace {
__global__ void k_validate_volume(const uint8_t* __restrict__ mat, const uint16_t* __restrict__ rho, size_t n,
                                  int n_mat, int* bad) {
  int b = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const uint16_t h = rho[i];
    b |= (mat[i] >= n_mat) | (((h & 0x8000u) != 0) & ((h & 0x7fffu) != 0)) | (((h >> 10) & 31u) == 31u);
  }
  if (__syncthreads_or(b) && threadIdx.x == 0) atomicOr(bad, 1);
}
}  // namespace

// Packs material + density into voxel words over the padded grid; border
// voxels repeat the nearest edge voxel.
__global__ void k_pack_volume(const uint8_t* __restrict__ mat, const uint16_t* __restrict__ rho, VolumeView v,
                              uint32_t* __restrict__ out) {
  const size_t n = (size_t)v.px * v.py * v.pz;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int px = (int)(i % v.px);
    const size_t r = i / v.px;
    const int py = (int)(r % v.py), pz = (int)(r / v.py);
    const int ix = min(max(px - 1, 0), v.nx - 1), iy = min(max(py - 1, 0), v.ny - 1), iz = min(max(pz - 1, 0), v.nz - 1);
    const size_t src = ((size_t)iz * v.ny + iy) * v.nx + ix;
    const int o = v.layout == VOX_BRICK ? vox_index<VOX_BRICK>(v, px, py, pz) : vox_index<VOX_LIN>(v, px, py, pz);
    out[o] = (uint32_t)rho[src] | ((uint32_t)mat[src] << 16);
  }
}

void padded_dims(int nx, int ny, int nz, int layout, VolumeView* v) {
  v->nx = nx; v->ny = ny; v->nz = nz;
  v->px = nx + 2; v->py = ny + 2; v->pz = nz + 2;
  v->layout = layout;
  v->nbx = (v->px + 3) / 4;
  v->nby = (v->py + 3) / 4;
  const size_t words = layout == VOX_BRICK ? (size_t)v->nbx * v->nby * ((v->pz + 3) / 4) * 64
                                           : (size_t)v->px * v->py * v->pz;
  v->words = (int)words;
  v->pxy = v->px * v->py;
  v->lin_bias = (int)(0x4B000000u * (1u + (uint32_t)v->px + (uint32_t)v->pxy));
}

size_t packed_words(int nx, int ny, int nz, int layout) {
  VolumeView v;
  padded_dims(nx, ny, nz, layout, &v);
  return (size_t)v.words;
}

cudaError_t pack_volume(const uint8_t* mat, const uint16_t* rho, int nx, int ny, int nz, int layout, uint32_t* out,
                        size_t out_words, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, out_words * 4, s);
  if (e != cudaSuccess) return e;
  VolumeView v;
  padded_dims(nx, ny, nz, layout, &v);
  k_pack_volume<<<1024, 256, 0, s>>>(mat, rho, v, out);
  return cudaGetLastError();
}

cudaError_t validate_volume_device(const uint8_t* mat, const uint16_t* rho, size_t n, int n_mat, cudaStream_t s,
                                   int* bad_host) {
  int* d_bad = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d_bad, sizeof(int), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(d_bad, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    k_validate_volume<<<1024, 256, 0, s>>>(mat, rho, n, n_mat, d_bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(bad_host, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d_bad, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}
}  // namespace mcx
