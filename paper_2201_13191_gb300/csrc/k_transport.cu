// Persistent photon-transport kernel: source sampling over the binned spectrum,
// fixed-step free flight through the uint8/FP16 voxel volume, interaction
// sampling (photoelectric, Compton by Kahn's method, Rayleigh by form-factor
// inversion plus Thomson rejection) and point-detector scoring split into
// n_split pseudo-particles aimed at random pixels (arXiv 2201.13191 Sec. II-A,
// eqs. Th, pmueforIncoherent, pmueforcoherent, Is; Sec. II-C.1, II-C.2).
//
// Each thread runs whole histories; history h of angle a draws its random
// numbers from Philox4x32-10 keyed by (seed, a, h), in a fixed order, so any
// history can be recomputed on its own.  The cross-section tables are staged
// once per block into shared memory by a bulk asynchronous copy (TMA engine,
// cp.async.bulk) completing on an mbarrier.
#include <cuda_fp16.h>
#include <stdint.h>

#include "mc_device.cuh"

namespace mcx {

namespace {

constexpr float kPi = 3.14159265358979f;
constexpr uint32_t kWaitLimit = 1u << 22;  // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing on `bar`.  Returns false if
// the wait gave up (the caller records the error and leaves).
__device__ bool stage_bulk(void* dst, const void* src, int bytes, uint64_t* bar) {
  const uint32_t b = smem_addr(bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    const int chunk = 16384;
    for (int off = 0; off < bytes; off += chunk) {
      const int n = min(chunk, bytes - off);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_addr((char*)dst + off)),
          "l"((const char*)src + off), "r"(n), "r"(b)
          : "memory");
    }
  }
  uint32_t done = 0;
  for (uint32_t it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(b)
        : "memory");
  }
  return done != 0;
}

struct Counters {
  unsigned long long flight_steps, nee_steps;
  uint32_t nee_rays, photo, compton, rayleigh, escape, limit, fail, hist;
};

// Fill this thread's column of the per-material total attenuation (mm^-1 per
// g/cm^3) at energy E.
__device__ __forceinline__ void fill_mu(const SmemTables& T, float E, float* smu, int stride) {
  int i;
  float f;
  T.locate(E, i, f);
  for (int m = 0; m < T.n_mat; ++m) smu[m * stride] = 0.1f * T.at(TAB_TOT, m, i, f);
}

// Optical depth of the fixed-step march x + t w, t in [0, t1] (Sec. II-C.2),
// material attenuation from smu (this thread's column); counts steps.
__device__ __forceinline__ float march_tau(const VolumeView& V, float3 x, float3 w, float t1, float step,
                                           const float* smu, int stride, unsigned long long& nsteps) {
  float ta, tb;
  if (!clip_box(V, x, w, 0.f, t1, ta, tb)) return 0.f;
  const float L = tb - ta;
  const int n = step_count(L, step);
  const float h = L / (float)n;
  VoxRay r;
  r.set(V, x, w);
  float acc = 0.f;
  int cur = -1;
  float mu = 0.f;
  for (int k = 0; k < n; ++k) {
    const float t = fmaf((float)k + 0.5f, h, ta);
    const int v = r.voxel(V, t);
    const int m = __ldg(V.mat + v);
    const float rho = __half2float(__ldg(V.rho + v));
    if (m != cur) {
      cur = m;
      mu = smu[m * stride];
    }
    acc = fmaf(mu, rho, acc);
  }
  nsteps += (unsigned long long)n;
  return acc * h;
}

// Kahn's rejection method for the Klein-Nishina distribution; returns
// r = E/E' (cos theta = 1 - (r-1)/a).
__device__ __forceinline__ float kahn(Rng& g, float a, bool& fail) {
  const float thr = (1.f + 2.f * a) / (9.f + 2.f * a);
  for (int it = 0; it < 100000; ++it) {
    const float u1 = g.u(), u2 = g.u(), u3 = g.u();
    float r;
    bool acc;
    if (u1 <= thr) {
      r = fmaf(2.f * a, u2, 1.f);
      acc = u3 <= 4.f * (1.f / r - 1.f / (r * r));
    } else {
      r = (1.f + 2.f * a) / fmaf(2.f * a, u2, 1.f);
      const float mu = 1.f - (r - 1.f) / a;
      acc = u3 <= 0.5f * (mu * mu + 1.f / r);
    }
    if (acc) return r;
  }
  fail = true;
  return 1.f;
}

// Rayleigh: component i with probability ~ w_i Z_i^2 G_i(K), inversion of
// (1 + b u)^-4 on [0, K], rejection on (1 + mu^2)/2.  Returns cos theta.
__device__ __forceinline__ float rayleigh(Rng& g, const SmemTables& T, int m, float E, bool& fail) {
  const float K = (E * T.inv_hc) * (E * T.inv_hc);
  const int nc = T.ncomp[m];
  const float2* cp = T.comp + m * kMaxComp;
  float G[kMaxComp];
  float tot = 0.f;
#pragma unroll
  for (int i = 0; i < kMaxComp; ++i) {
    G[i] = 0.f;
    if (i < nc) {
      const float T1 = fmaf(cp[i].y, K, 1.f);
      G[i] = cp[i].x * (1.f - 1.f / (T1 * T1 * T1)) / (3.f * cp[i].y);
      tot += G[i];
    }
  }
  for (int it = 0; it < 100000; ++it) {
    const float u1 = g.u(), u2 = g.u(), u3 = g.u();
    const float target = u1 * tot;
    float acc = 0.f, b = cp[0].y;
#pragma unroll
    for (int i = 0; i < kMaxComp; ++i) {
      if (i < nc) {
        acc += G[i];
        b = cp[i].y;
        if (target < acc) break;
      }
    }
    const float T1 = fmaf(b, K, 1.f);
    const float q = 1.f - u2 * (1.f - 1.f / (T1 * T1 * T1));
    const float u = (rcbrtf(q) - 1.f) / b;
    float mu = 1.f - 2.f * u / K;
    mu = fmaxf(mu, -1.f);
    if (u3 <= 0.5f * (1.f + mu * mu)) return mu;
  }
  fail = true;
  return 1.f;
}

__device__ __forceinline__ float3 rotate(float3 w, float ct, float phi) {
  const float st = sqrtf(fmaxf(0.f, 1.f - ct * ct));
  float sp, cp;
  sincosf(phi, &sp, &cp);
  float3 o;
  if (fabsf(w.z) > 0.99999f) {
    o = make_float3(st * cp, st * sp, w.z > 0.f ? ct : -ct);
  } else {
    const float s = sqrtf(1.f - w.z * w.z);
    const float is = 1.f / s;
    o.x = w.x * ct + st * (w.x * w.z * cp - w.y * sp) * is;
    o.y = w.y * ct + st * (w.y * w.z * cp + w.x * sp) * is;
    o.z = w.z * ct - st * s * cp;
  }
  const float in = rsqrtf(dot3(o, o));
  return make_float3(o.x * in, o.y * in, o.z * in);
}

__global__ void __launch_bounds__(256) k_transport(const TransportParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  const int nm = P.tab.n_mat, ns = P.tab.n_stage;
  // shared layout: [table blob][prefix u64 (n_bins+1)][energy f32][wbin f32][mu columns f32 nm x blockDim]
  float2* s_blob = reinterpret_cast<float2*>(smem);
  unsigned long long* s_pre = reinterpret_cast<unsigned long long*>(smem + P.tab.blob_bytes);
  const int nb = P.spec.n_bins;
  float* s_E = reinterpret_cast<float*>(s_pre + nb + 1);
  float* s_wb = s_E + nb;
  float* s_mu = s_wb + nb;

  const bool staged = stage_bulk(s_blob, P.tab.blob, P.tab.blob_bytes, &bar);
  for (int i = threadIdx.x; i <= nb; i += blockDim.x) s_pre[i] = P.spec.prefix[i];
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    s_E[i] = P.spec.energy[i];
    s_wb[i] = P.spec.wbin[i];
  }
  __syncthreads();
  if (!staged) {
    if (threadIdx.x == 0) atomicAdd(P.stats + S_INTERNAL, 1ull);
    return;
  }
  SmemTables T;
  T.tab = s_blob;
  T.jkn = reinterpret_cast<const float2*>(smem + tab_off_jkn(nm, ns));
  T.comp = reinterpret_cast<const float2*>(smem + tab_off_comp(nm, ns));
  T.ncomp = reinterpret_cast<const int*>(smem + tab_off_ncomp(nm, ns));
  T.n_mat = nm;
  T.n_stage = ns;
  T.E0 = P.tab.E0;
  T.inv_dE = P.tab.inv_dE;
  T.mec2 = P.tab.mec2;
  T.inv_hc = P.tab.inv_hc;

  const VolumeView& V = P.vol;
  const GeomView& G = P.geo;
  const int stride = blockDim.x;
  float* my_mu = s_mu + threadIdx.x;
  const uint32_t npix = (uint32_t)G.nu * (uint32_t)G.nv;
  const float A_det = (float)G.nu * G.pu * (float)G.nv * G.pv;
  const float A_px = G.pu * G.pv;
  const float nee_scale = A_px * ((float)npix / (float)P.n_split) / (2.f * kPi);
  const size_t img = (size_t)npix;

  Counters C = {};
  const unsigned long long total = (unsigned long long)P.n_angles * P.h_count;
  for (unsigned long long w_i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; w_i < total;
       w_i += (unsigned long long)gridDim.x * blockDim.x) {
    const int a = (int)(w_i / P.h_count);
    const unsigned long long h = P.h_begin + (w_i - (unsigned long long)a * P.h_count);
    // energy bin by the stratified prefix sums
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_pre[mid] <= h) lo = mid;
      else hi = mid - 1;
    }
    const int bin = lo;
    float E = s_E[bin];
    Rng g;
    g.init(h, (uint32_t)a, P.seed);
    const Pose ps = make_pose(G, __ldg(P.angles + a));
    double* tally = P.tally + ((size_t)(P.n_batches > 1 ? (int)(h % (unsigned long long)P.n_batches) : 0) *
                                   P.n_angles + a) * img;
    // source: uniform point on the panel, solid-angle Jacobian weight
    const float ua = g.u(), ub = g.u();
    const float3 Q = det_point(G, ps, ua * (float)G.nu, ub * (float)G.nv);
    float3 D = sub3(Q, ps.s);
    float d = sqrtf(dot3(D, D));
    float3 w = make_float3(D.x / d, D.y / d, D.z / d);
    const float W = s_wb[bin] * A_det * (G.sdd / d) / (4.f * kPi * d * d);
    float3 x = ps.s;
    int order = 0;
    ++C.hist;
    for (;;) {
      const float tau_star = -logf(g.u());
      float ta, tb;
      bool hit = false;
      float tint = 0.f;
      int mint = 0;
      if (clip_box(V, x, w, 0.f, __int_as_float(0x7f800000), ta, tb)) {
        fill_mu(T, E, my_mu, stride);
        const float L = tb - ta;
        const int n = step_count(L, P.step);
        const float hh = L / (float)n;
        VoxRay r;
        r.set(V, x, w);
        float tau = 0.f, mu_m = 0.f;
        int cur = -1, k = 0;
        for (; k < n; ++k) {
          const float t = fmaf((float)k + 0.5f, hh, ta);
          const int v = r.voxel(V, t);
          const int m = __ldg(V.mat + v);
          const float rho = __half2float(__ldg(V.rho + v));
          if (m != cur) {
            cur = m;
            mu_m = my_mu[m * stride];
          }
          const float mu = mu_m * rho;
          if (fmaf(mu, hh, tau) >= tau_star) {
            tint = fmaf((float)k, hh, ta) + (tau_star - tau) / mu;
            mint = m;
            hit = true;
            break;
          }
          tau = fmaf(mu, hh, tau);
        }
        C.flight_steps += (unsigned long long)(hit ? k + 1 : n);
      }
      if (!hit) {
        ++C.escape;
        break;
      }
      x = make_float3(fmaf(tint, w.x, x.x), fmaf(tint, w.y, x.y), fmaf(tint, w.z, x.z));
      // interaction type
      int ti;
      float tf;
      T.locate(E, ti, tf);
      const float pe = T.at(TAB_PE, mint, ti, tf), in = T.at(TAB_IN, mint, ti, tf),
                  co = T.at(TAB_CO, mint, ti, tf);
      const float ut = g.u() * (pe + in + co);
      const int type = ut < pe ? 0 : (ut < pe + in ? 1 : 2);
      if (type == 0) {
        ++C.photo;
        break;
      }
      if (type == 1) ++C.compton;
      else ++C.rayleigh;
      // point-detector scoring split into n_split pseudo-particles (eq. Th)
      const float alpha = E / T.mec2;
      const float norm = type == 1 ? 1.f / T.kn_norm(ti, tf) : 1.f / T.at(TAB_ICOH, mint, ti, tf);
      const float K = (E * T.inv_hc) * (E * T.inv_hc);
      g.align();
      for (int s = 0; s < P.n_split; ++s) {
        g.refill();
        const uint32_t rpix = g.buf.x;
        const float va = Rng::u01(g.buf.y), vb = Rng::u01(g.buf.z), vr = Rng::u01(g.buf.w);
        g.idx = 4;
        const uint32_t pix = __umulhi(rpix, npix);
        const uint32_t pi = pix % (uint32_t)G.nu, pj = pix / (uint32_t)G.nu;
        const float3 Pp = det_point(G, ps, (float)pi + va, (float)pj + vb);
        const float3 DD = sub3(Pp, x);
        const float dd2 = dot3(DD, DD);
        const float idd = rsqrtf(dd2);
        const float3 dir = make_float3(DD.x * idd, DD.y * idd, DD.z * idd);
        const float lam = dot3(w, dir);
        const float cosg = -dot3(dir, ps.n);
        float Ep, p;
        if (type == 1) {
          const float ratio = 1.f / fmaf(alpha, 1.f - lam, 1.f);
          Ep = E * ratio;
          p = ratio * ratio * (ratio + 1.f / ratio - 1.f + lam * lam) * norm;
        } else {
          Ep = E;
          const float u = 0.5f * K * (1.f - lam);
          float F2 = 0.f;
          const int nc = T.ncomp[mint];
          const float2* cp = T.comp + mint * kMaxComp;
          for (int i = 0; i < nc; ++i) {
            const float q = fmaf(cp[i].y, u, 1.f);
            const float q2 = q * q;
            F2 += cp[i].x / (q2 * q2);
          }
          p = (1.f + lam * lam) * F2 * norm;
        }
        float x0 = W * Ep * p * cosg * nee_scale / dd2;
        ++C.nee_rays;
        if (P.rr_threshold > 0.f && x0 < P.rr_threshold) {
          if (vr >= x0 / P.rr_threshold) continue;
          x0 = P.rr_threshold;
        }
        // Rayleigh keeps the energy, so the flight's column is still valid.
        if (type == 1) fill_mu(T, Ep, my_mu, stride);
        const float tp = march_tau(V, x, dir, dd2 * idd, P.step, my_mu, stride, C.nee_steps);
        const float sc = x0 * __expf(-tp);
        atomicAdd(tally + pix, (double)sc);
      }
      // new direction
      bool fail = false;
      float ct, Enew = E;
      if (type == 1) {
        const float r = kahn(g, alpha, fail);
        ct = 1.f - (r - 1.f) / alpha;
        Enew = E / r;
      } else {
        ct = rayleigh(g, T, mint, E, fail);
      }
      const float phi = 2.f * kPi * g.u();
      if (fail) ++C.fail;
      w = rotate(w, ct, phi);
      E = Enew;
      ++order;
      if (E < 1.f) break;
      if (order >= P.max_order) {
        ++C.limit;
        break;
      }
    }
  }
  // block-level counter reduction
  __shared__ unsigned long long red[S_NSTAT];
  if (threadIdx.x < S_NSTAT) red[threadIdx.x] = 0ull;
  __syncthreads();
  atomicAdd(&red[S_HIST], (unsigned long long)C.hist);
  atomicAdd(&red[S_FLIGHT_STEPS], C.flight_steps);
  atomicAdd(&red[S_NEE_STEPS], C.nee_steps);
  atomicAdd(&red[S_NEE_RAYS], (unsigned long long)C.nee_rays);
  atomicAdd(&red[S_PHOTO], (unsigned long long)C.photo);
  atomicAdd(&red[S_COMPTON], (unsigned long long)C.compton);
  atomicAdd(&red[S_RAYLEIGH], (unsigned long long)C.rayleigh);
  atomicAdd(&red[S_ESCAPE], (unsigned long long)C.escape);
  atomicAdd(&red[S_LIMIT], (unsigned long long)C.limit);
  atomicAdd(&red[S_SAMPLER_FAIL], (unsigned long long)C.fail);
  __syncthreads();
  if (threadIdx.x < S_NSTAT && red[threadIdx.x]) atomicAdd(P.stats + threadIdx.x, red[threadIdx.x]);
}

__global__ void k_finalize(const double* __restrict__ tally, int B, size_t n, float* __restrict__ out,
                           float* __restrict__ var) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (B == 1) {
      if (out) out[i] = (float)tally[i];
      continue;
    }
    double sum = 0.0;
    for (int b = 0; b < B; ++b) sum += tally[(size_t)b * n + i];
    double ss = 0.0;
    for (int b = 0; b < B; ++b) {
      const double e = (double)B * tally[(size_t)b * n + i] - sum;
      ss += e * e;
    }
    if (out) out[i] = (float)sum;
    if (var) var[i] = (float)(ss / ((double)B * (B - 1)));
  }
}

}  // namespace

int transport_smem_bytes(const TableView& t, int n_bins, int block) {
  return t.blob_bytes + (n_bins + 1) * 8 + n_bins * 8 + kMaxMat * block * 4;
}

cudaError_t transport_occupancy(int block, int smem, int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_transport, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_transport, block, smem);
}

cudaError_t launch_transport(const TransportParams& p, int grid, int block, cudaStream_t s) {
  const int smem = transport_smem_bytes(p.tab, p.spec.n_bins, block);
  cudaError_t e = cudaFuncSetAttribute(k_transport, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_transport<<<grid, block, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double* tally, int n_batches, size_t n, float* out, float* var, cudaStream_t s) {
  const int block = 256;
  const int grid = (int)std::min<size_t>((n + block - 1) / block, 152 * 16);
  k_finalize<<<grid, block, 0, s>>>(tally, n_batches, n, out, var);
  return cudaGetLastError();
}

}  // namespace mcx
