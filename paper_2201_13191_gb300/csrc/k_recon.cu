// Iterative scatter correction plumbing (arXiv 2201.13191 Sec. II-E, Fig.
// flowchart, eq. Correction): conversion of intensities to line integrals,
// FDK (cone-beam filtered backprojection) for the circular orbit of this
// library's geometry, multi-level Otsu segmentation, conversion of the
// segmented volume to material ids and densities, its 2x2x2 down-sampling for
// the Monte Carlo step (Sec. II-C.2), and the correction
// c = a - ln(Ip / (Ip + Is)).
#include <cuda_fp16.h>
#include <stdint.h>

#include "mc_internal.h"

namespace mcx {
namespace {

__device__ __forceinline__ size_t gtid() { return (size_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ size_t gstride() { return (size_t)gridDim.x * blockDim.x; }
int blocks_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

// a = -ln(I / I0) per pixel (I0 is one flat-field image shared by all projections).
__global__ void k_log_norm(const float* __restrict__ I, const float* __restrict__ I0, size_t img, size_t n,
                           float* __restrict__ a) {
  for (size_t i = gtid(); i < n; i += gstride()) {
    const float v = fmaxf(I[i], 1e-30f), f = fmaxf(I0[i % img], 1e-30f);
    a[i] = -logf(v / f);
  }
}

// FDK pre-weighting and ramp filtering of detector rows:
//   q(u_i) = du * sum_j h(i - j) * w(u_j, v) p(u_j),  w = D / sqrt(D^2 + u^2 + v^2)
// with u, v the pixel-centre offsets scaled to the isocentre plane, D = SOD,
// du the isocentre pixel pitch and h the discrete Ram-Lak kernel
// h(0) = 1/(4 du^2), h(odd n) = -1/(n pi du)^2, h(even n != 0) = 0.
// A block filters kFiltRows rows; a warp owns 256 consecutive outputs (8 per
// lane) of each of them.  Walking j, lane l needs the taps h(i0 + m - j),
// m = 0..7, i0 = 8 l + warp base: one step in j shifts that window by one, so
// the new first tap is the previous lane's last one (a shuffle) and only lane 0
// reads a tap from shared memory.  The taps are shared by the rows, so each
// tap register feeds kFiltRows x 8 FMAs.
constexpr int kFiltOut = 8;
constexpr int kFiltRows = 4;
constexpr int kFiltThreads = 256;

__global__ void __launch_bounds__(kFiltThreads) k_fdk_filter(const float* __restrict__ p, int nu, int nv, int rows_total,
                                                             float du_iso, float dv_iso, float sod,
                                                             float* __restrict__ q) {
  extern __shared__ float fsh[];
  const int span = kFiltThreads * kFiltOut;               // outputs per pass of the block
  const int npad = (nu + span - 1) / span * span;
  const int H0 = npad + kFiltOut;                          // hs[d + H0] = h(d), |d| <= H0
  float* hs = fsh;
  float* rows = fsh + 2 * H0 + 1;                          // [kFiltRows][nu]
  const float h0 = 0.25f / (du_iso * du_iso), c = 1.f / (9.8696044f * du_iso * du_iso);
  for (int k = threadIdx.x; k <= 2 * H0; k += blockDim.x) {
    const int d = k - H0;
    hs[k] = d == 0 ? h0 : ((d & 1) ? -c / ((float)d * (float)d) : 0.f);
  }
  const int r0 = blockIdx.x * kFiltRows;
  for (int rr = 0; rr < kFiltRows; ++rr) {
    const int r = r0 + rr;
    const float vv = ((float)((r < rows_total ? r : 0) % nv) - 0.5f * (float)(nv - 1)) * dv_iso;
    for (int i = threadIdx.x; i < nu; i += blockDim.x) {
      const float uu = ((float)i - 0.5f * (float)(nu - 1)) * du_iso;
      rows[rr * nu + i] = r < rows_total ? p[(size_t)r * nu + i] * sod * rsqrtf(sod * sod + uu * uu + vv * vv) : 0.f;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = warp * 256; base < npad; base += span) {
    const int i0 = base + lane * kFiltOut;
    float w[kFiltOut], acc[kFiltRows][kFiltOut];
#pragma unroll
    for (int m = 0; m < kFiltOut; ++m) {
      w[m] = hs[i0 + m + H0];
#pragma unroll
      for (int rr = 0; rr < kFiltRows; ++rr) acc[rr][m] = 0.f;
    }
#pragma unroll 4
    for (int j = 0; j < nu; ++j) {
#pragma unroll
      for (int rr = 0; rr < kFiltRows; ++rr) {
        const float x = rows[rr * nu + j];
#pragma unroll
        for (int m = 0; m < kFiltOut; ++m) acc[rr][m] = fmaf(x, w[m], acc[rr][m]);
      }
      const float carry = __shfl_up_sync(0xffffffffu, w[kFiltOut - 1], 1);
#pragma unroll
      for (int m = kFiltOut - 1; m > 0; --m) w[m] = w[m - 1];
      w[0] = lane == 0 ? hs[base - j - 1 + H0] : carry;
    }
#pragma unroll
    for (int rr = 0; rr < kFiltRows; ++rr) {
      const int r = r0 + rr;
      if (r >= rows_total) continue;
#pragma unroll
      for (int m = 0; m < kFiltOut; ++m)
        if (i0 + m < nu) q[(size_t)r * nu + i0 + m] = acc[rr][m] * du_iso;
    }
  }
}

// Voxel-driven backprojection: f(x) = (dbeta / 2) sum_beta (D / (D - x.n))^2 q(u(x), v(x)),
// q bilinearly interpolated at the voxel's projection (zero outside the panel).
// Voxel-driven backprojection: each thread owns kZB voxels of one (x, y)
// column; per projection the source-side terms (depth, magnification, u and
// its bilinear weights) are computed once for the column, then each voxel adds
// its bilinear sample (the same expressions as one voxel at a time, so the
// same sums).
constexpr int kZB = 4;
__global__ void k_fdk_backproject(const float* __restrict__ q, const float* __restrict__ cb, const float* __restrict__ sb,
                                  int n_proj, int nu, int nv, float du_iso, float dv_iso, float sod, int nx, int ny,
                                  int nz, float dx, float dy, float dz, float scale, float* __restrict__ vol) {
  const int nzb = (nz + kZB - 1) / kZB;
  const size_t n = (size_t)nx * ny * nzb;
  for (size_t i = gtid(); i < n; i += gstride()) {
    const int ix = (int)(i % nx);
    const size_t t = i / nx;
    const int iy = (int)(t % ny), iz0 = (int)(t / ny) * kZB;
    const float x = ((float)ix - 0.5f * (float)(nx - 1)) * dx;
    const float y = ((float)iy - 0.5f * (float)(ny - 1)) * dy;
    float z[kZB], acc[kZB];
#pragma unroll
    for (int j = 0; j < kZB; ++j) {
      z[j] = ((float)(iz0 + j) - 0.5f * (float)(nz - 1)) * dz;
      acc[j] = 0.f;
    }
    for (int k = 0; k < n_proj; ++k) {
      const float c = __ldg(cb + k), s = __ldg(sb + k);
      const float depth = sod - (x * c + y * s);  // distance from the source along the central ray
      const float mag = sod / depth;
      const float u = (-x * s + y * c) * mag;     // isocentre-plane coordinates
      const float fu = u / du_iso + 0.5f * (float)(nu - 1);
      const int u0 = __float2int_rd(fu);
      const float au = fu - (float)u0;
      const bool u_in = u0 >= 0 && u0 + 1 < nu;
      const float* qp = q + (size_t)k * nu * nv;
#pragma unroll
      for (int j = 0; j < kZB; ++j) {
        const float v = z[j] * mag;
        const float fv = v / dv_iso + 0.5f * (float)(nv - 1);
        const int v0 = __float2int_rd(fv);
        const float av = fv - (float)v0;
        float val = 0.f;
        if (u_in && v0 >= 0 && v0 + 1 < nv) {
          const float* r0 = qp + (size_t)v0 * nu + u0;
          val = (1.f - av) * ((1.f - au) * __ldg(r0) + au * __ldg(r0 + 1)) +
                av * ((1.f - au) * __ldg(r0 + nu) + au * __ldg(r0 + nu + 1));
        }
        acc[j] = fmaf(mag * mag, val, acc[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < kZB; ++j)
      if (iz0 + j < nz) vol[((size_t)(iz0 + j) * ny + iy) * nx + ix] = acc[j] * scale;
  }
}

// Histogram of vol over [lo, hi) in nbins bins (values outside are clamped to the end bins).
__global__ void k_hist(const float* __restrict__ vol, size_t n, float lo, float hi, int nbins,
                       unsigned int* __restrict__ hist) {
  extern __shared__ unsigned int sh[];
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  const float sc = (float)nbins / (hi - lo);
  for (size_t i = gtid(); i < n; i += gstride()) {
    const int b = min(max((int)((vol[i] - lo) * sc), 0), nbins - 1);
    atomicAdd(&sh[b], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x)
    if (sh[b]) atomicAdd(&hist[b], sh[b]);
}

// Multi-level Otsu (classes = 2 or 3): thresholds maximising the between-class
// variance of the histogram, exhaustively (one block; nbins <= 256).
__global__ void k_otsu(const unsigned int* __restrict__ hist, int nbins, int classes, int* __restrict__ thr) {
  __shared__ double P[257], S[257];
  __shared__ double best_val[256];
  __shared__ int best_a[256], best_b[256];
  if (threadIdx.x == 0) {
    P[0] = 0;
    S[0] = 0;
    for (int b = 0; b < nbins; ++b) {
      P[b + 1] = P[b] + hist[b];
      S[b + 1] = S[b] + (double)hist[b] * (b + 0.5);
    }
  }
  __syncthreads();
  const double N = P[nbins], mu = S[nbins] / fmax(N, 1.0);
  auto term = [&](int a, int b) {  // class [a, b)
    const double w = P[b] - P[a];
    if (w <= 0) return 0.0;
    const double m = (S[b] - S[a]) / w;
    return w * (m - mu) * (m - mu);
  };
  double bv = -1;
  int ba = 1, bb = nbins;
  for (int a = 1 + threadIdx.x; a < nbins; a += blockDim.x) {
    if (classes == 2) {
      const double v = term(0, a) + term(a, nbins);
      if (v > bv) { bv = v; ba = a; bb = nbins; }
    } else {
      for (int b = a + 1; b < nbins; ++b) {
        const double v = term(0, a) + term(a, b) + term(b, nbins);
        if (v > bv) { bv = v; ba = a; bb = b; }
      }
    }
  }
  best_val[threadIdx.x] = bv;
  best_a[threadIdx.x] = ba;
  best_b[threadIdx.x] = bb;
  __syncthreads();
  if (threadIdx.x == 0) {
    int k = 0;
    for (int t = 1; t < (int)blockDim.x; ++t)
      if (best_val[t] > best_val[k] || (best_val[t] == best_val[k] && (best_a[t] < best_a[k] ||
                                                                     (best_a[t] == best_a[k] && best_b[t] < best_b[k]))))
        k = t;
    thr[0] = best_a[k];
    thr[1] = best_b[k];
  }
}

// Class of each voxel by the thresholds (bins) -> material id and density
// rho = mu / (mu_rho(material) * 0.1), clamped to [0, rho_max]; class 0 -> the
// background material at its nominal density.
__global__ void k_segment(const float* __restrict__ vol, size_t n, float lo, float hi, int nbins,
                          const int* __restrict__ thr, int classes, const int* __restrict__ cls_mat,
                          const float* __restrict__ cls_murho, const float* __restrict__ cls_rho0, float rho_max,
                          uint8_t* __restrict__ mat, uint16_t* __restrict__ rho) {
  const float sc = (float)nbins / (hi - lo);
  const int t0 = thr[0], t1 = thr[1];
  for (size_t i = gtid(); i < n; i += gstride()) {
    const int b = min(max((int)((vol[i] - lo) * sc), 0), nbins - 1);
    const int c = b < t0 ? 0 : ((classes == 2 || b < t1) ? 1 : 2);
    mat[i] = (uint8_t)cls_mat[c];
    float r = c == 0 ? cls_rho0[0] : fminf(fmaxf(vol[i] / (0.1f * cls_murho[c]), 0.f), rho_max);
    rho[i] = __half_as_ushort(__float2half_rn(r));
  }
}

// Down-sampling by 2 per axis for the Monte Carlo step (Sec. II-C.2, II-E):
// each 2x2x2 block becomes one voxel of the material with the block's largest
// mass (ties to the lower id) and the density that keeps the block's summed
// attenuation at the effective energy, sum_v murho[m_v] rho_v / (8 murho[m_b]).
__global__ void k_bin_volume(const uint8_t* __restrict__ mat, const uint16_t* __restrict__ rho, int nx, int ny,
                             int nz, const float* __restrict__ murho, int n_mat, uint8_t* __restrict__ mat_b,
                             uint16_t* __restrict__ rho_b) {
  const int bx = nx / 2, by = ny / 2, bz = nz / 2;
  const size_t n = (size_t)bx * by * bz;
  for (size_t i = gtid(); i < n; i += gstride()) {
    const int x = (int)(i % bx), y = (int)((i / bx) % by), z = (int)(i / ((size_t)bx * by));
    float mass[kMaxMat];
#pragma unroll
    for (int m = 0; m < kMaxMat; ++m) mass[m] = 0.f;
    float mu = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const size_t v = ((size_t)(2 * z + (q >> 2)) * ny + (2 * y + ((q >> 1) & 1))) * nx + (2 * x + (q & 1));
      const int m = mat[v];
      const float r = __half2float(__ushort_as_half(rho[v]));
#pragma unroll
      for (int k = 0; k < kMaxMat; ++k) mass[k] += (k == m) ? r : 0.f;
      mu = fmaf(__ldg(murho + m), r, mu);
    }
    int best = 0;
    for (int m = 1; m < n_mat; ++m)
      if (mass[m] > mass[best]) best = m;
    mat_b[i] = (uint8_t)best;
    rho_b[i] = __half_as_ushort(__float2half_rn(mu / (8.f * __ldg(murho + best))));
  }
}

// c = a - ln(Ip / (Ip + Is)) (eq. Correction).
__global__ void k_correct(const float* __restrict__ a, const float* __restrict__ ip, const float* __restrict__ is,
                          float is_scale, size_t n, float* __restrict__ c) {
  for (size_t i = gtid(); i < n; i += gstride()) {
    const float p = fmaxf(ip[i], 1e-30f), sc = fmaxf(is[i], 0.f) * is_scale;
    c[i] = a[i] - logf(p / (p + sc));
  }
}

}  // namespace

cudaError_t recon_bin_volume(const uint8_t* mat, const uint16_t* rho, int nx, int ny, int nz, const float* murho,
                             int n_mat, uint8_t* mat_b, uint16_t* rho_b, cudaStream_t s) {
  if (nx % 2 || ny % 2 || nz % 2 || n_mat < 1 || n_mat > kMaxMat) return cudaErrorInvalidValue;
  const size_t n = (size_t)(nx / 2) * (ny / 2) * (nz / 2);
  k_bin_volume<<<blocks_for(n), 256, 0, s>>>(mat, rho, nx, ny, nz, murho, n_mat, mat_b, rho_b);
  return cudaGetLastError();
}

cudaError_t recon_log_norm(const float* I, const float* I0, size_t img, size_t n, float* a, cudaStream_t s) {
  k_log_norm<<<blocks_for(n), 256, 0, s>>>(I, I0, img, n, a);
  return cudaGetLastError();
}

cudaError_t recon_fdk(const float* p, int n_proj, const float* d_cos, const float* d_sin, int nu, int nv, float pu,
                      float pv, float sod, float sdd, int nx, int ny, int nz, float dx, float dy, float dz, float* q_tmp,
                      float* vol, cudaStream_t s) {
  const float du = pu * sod / sdd, dv = pv * sod / sdd;  // pixel pitch at the isocentre
  const int span = kFiltThreads * kFiltOut;
  const size_t npad = ((size_t)nu + span - 1) / span * span;
  const size_t smem = ((2 * (npad + kFiltOut) + 1) + (size_t)kFiltRows * nu) * 4;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_fdk_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int rows_total = n_proj * nv;
  k_fdk_filter<<<(rows_total + kFiltRows - 1) / kFiltRows, kFiltThreads, smem, s>>>(p, nu, nv, rows_total, du, dv, sod,
                                                                                    q_tmp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // full orbit: (dbeta / 2) with dbeta = 2 pi / n_proj
  const float scale = 3.14159265358979f / (float)n_proj;
  const size_t n = (size_t)nx * ny * ((nz + kZB - 1) / kZB);
  k_fdk_backproject<<<blocks_for(n), 256, 0, s>>>(q_tmp, d_cos, d_sin, n_proj, nu, nv, du, dv, sod, nx, ny, nz, dx,
                                                  dy, dz, scale, vol);
  return cudaGetLastError();
}

cudaError_t recon_otsu_segment(const float* vol, size_t n, float lo, float hi, int classes, const int* d_cls_mat,
                               const float* d_cls_murho, const float* d_cls_rho0, float rho_max, unsigned int* d_hist,
                               int* d_thr, uint8_t* mat, uint16_t* rho, cudaStream_t s) {
  const int nbins = 256;
  cudaError_t e = cudaMemsetAsync(d_hist, 0, nbins * 4, s);
  if (e != cudaSuccess) return e;
  k_hist<<<blocks_for(n), 256, nbins * 4, s>>>(vol, n, lo, hi, nbins, d_hist);
  k_otsu<<<1, 256, 0, s>>>(d_hist, nbins, classes, d_thr);
  k_segment<<<blocks_for(n), 256, 0, s>>>(vol, n, lo, hi, nbins, d_thr, classes, d_cls_mat, d_cls_murho, d_cls_rho0,
                                          rho_max, mat, rho);
  return cudaGetLastError();
}

cudaError_t recon_correct(const float* a, const float* ip, const float* is, float is_scale, size_t n, float* c,
                          cudaStream_t s) {
  k_correct<<<blocks_for(n), 256, 0, s>>>(a, ip, is, is_scale, n, c);
  return cudaGetLastError();
}

}  // namespace mcx
