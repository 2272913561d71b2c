// Persistent photon-transport kernel: source sampling over the binned spectrum,
// fixed-step free flight through the uint8/FP16 voxel volume (or exact flights
// through triangle-mesh bodies, the CAD model of Sec. II-A), interaction
// sampling (photoelectric, Compton by Kahn's method, Rayleigh by form-factor
// inversion plus Thomson rejection) and point-detector scoring split into
// n_split pseudo-particles aimed at random pixels, or under forced detection one
// pseudo-particle per pixel (arXiv 2201.13191 Sec. II-A, eqs. Th,
// pmueforIncoherent, pmueforcoherent, Is; Sec. I, II-C.1, II-C.2).
//
// Wavefront structure: each thread carries one photon's walk and runs one free
// flight per iteration; an interaction queues a record in shared memory, and
// its pseudo-particles are then shared out (longest chords first) before the
// next flight: among the warp's own lanes with the plain FP64 tally (no block
// barrier in the loop, so warps run their phases independently), or among the
// whole block with the combined tallies, whose shared images need block-wide
// steps.  History h of angle a draws
// its random numbers from Philox4x32-10 keyed by (seed, a, h), in a fixed
// order, with each pseudo-particle on its own counter block, so any history
// can be recomputed on its own.  The cross-section tables are staged once per
// block into shared memory by a bulk asynchronous copy (TMA engine,
// cp.async.bulk) completing on an mbarrier.
#include <cuda_fp16.h>
#include <stdint.h>

#include "mc_device.cuh"
#include "mc_mesh.cuh"

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
__device__ __forceinline__ void fill_mu(const SmemTables& T, int i, float f, float* smu, int stride) {
  for (int m = 0; m < T.n_mat; ++m) smu[m * stride] = 0.1f * T.at(TAB_TOT, m, i, f);
}
__device__ __forceinline__ void fill_mu(const SmemTables& T, float E, float* smu, int stride) {
  int i;
  float f;
  T.locate(E, i, f);
  fill_mu(T, i, f, smu, stride);
}

// Gathers of the next MC_LOOKAHEAD midpoints are issued before any of them is
// consumed: the step positions are fixed in advance, so the loads are
// independent and several are in flight per warp.  The group's midpoints are
// its first one plus u h v_w (one FMA per axis and step).  Every midpoint is
// loaded, repeats included (they hit the line the previous load brought into
// L1).  A march runs its whole groups without a bound test per step; only the
// last, ragged group masks the steps past the chord's end, whose loads read a
// clamped, in-bounds word that is ignored.
#ifndef MC_LOOKAHEAD
#define MC_LOOKAHEAD 8
#endif
constexpr int kLook = MC_LOOKAHEAD;
// Brick layout (volumes in HBM): every group of a march masks its steps past
// the end (1), or whole groups run unmasked and one tail group is masked (0,
// the linear layout's form).  The single masked loop measured 28% faster for
// bricks (ell512, 36 angles: 4880 -> 3503 ms), with the same steps.
#ifndef MC_BRICK_NOSPLIT
#define MC_BRICK_NOSPLIT 1
#endif

template <int LAYOUT>
__device__ __forceinline__ void gather_group(const VolumeView& V, const VoxRay& r, int k0, float h, float ta,
                                             float3 hv, uint32_t (&wd)[kLook]) {
  const float t0 = fmaf((float)k0 + 0.5f, h, ta);
  const float bx = fmaf(t0, r.vw.x, r.v0.x), by = fmaf(t0, r.vw.y, r.v0.y), bz = fmaf(t0, r.vw.z, r.v0.z);
  int idx[kLook];
#pragma unroll
  for (int u = 0; u < kLook; ++u)
    idx[u] = u == 0 ? r.voxel_p<LAYOUT>(V, bx, by, bz)
                    : r.voxel_p<LAYOUT>(V, fmaf((float)u, hv.x, bx), fmaf((float)u, hv.y, by), fmaf((float)u, hv.z, bz));
#pragma unroll
  for (int u = 0; u < kLook; ++u) wd[u] = __ldg(V.vox + idx[u]);
}

// Adds the group's steps to the optical-depth sum acc (attenuation per unit
// density from this thread's shared-memory column smu); TAIL masks the steps
// k0 + u >= n.
template <int LAYOUT, bool TAIL>
__device__ __forceinline__ void tau_group(const uint32_t (&wd)[kLook], int k0, int n, const float* smu, int stride,
                                          float& acc, int& cur, float& mu) {
  if (LAYOUT == VOX_LIN) {
    // volume in L2 (the linear layout is chosen while it fits): branch-free,
    // every step reads its material's attenuation from shared memory
#pragma unroll
    for (int u = 0; u < kLook; ++u) {
      const float t = fmaf(smu[vox_mat(wd[u]) * stride], vox_rho(wd[u]), acc);
      acc = (!TAIL || k0 + u < n) ? t : acc;
    }
  } else {
    // volume in HBM (bricks): keep the shared-memory pipe free for the gathers,
    // re-read the attenuation only when the material changes
#pragma unroll
    for (int u = 0; u < kLook; ++u) {
      if (!TAIL || k0 + u < n) {
        const int m = vox_mat(wd[u]);
        if (m != cur) {
          cur = m;
          mu = smu[m * stride];
        }
        acc = fmaf(mu, vox_rho(wd[u]), acc);
      }
    }
  }
}

// Optical depth of the fixed-step march x + t w, t in [0, t1] (Sec. II-C.2),
// material attenuation from smu (this thread's column); counts steps.
template <int LAYOUT>
__device__ __forceinline__ float march_tau(const VolumeView& V, float3 x, float3 w, float t1, float step,
                                           const float* smu, int stride, unsigned long long& nsteps) {
  float ta, tb;
  if (!clip_box(V, x, w, 0.f, t1, ta, tb)) return 0.f;
  const float L = tb - ta;
  const int n = step_count(L, step);
  const float h = L / (float)n;
  VoxRay r;
  r.set(V, x, w);
  const float3 hv = make_float3(h * r.vw.x, h * r.vw.y, h * r.vw.z);
  float acc = 0.f, mu = 0.f;
  int cur = -1, k0 = 0;
  if (LAYOUT == VOX_BRICK && MC_BRICK_NOSPLIT) {
    for (; k0 < n; k0 += kLook) {
      uint32_t wd[kLook];
      gather_group<LAYOUT>(V, r, k0, h, ta, hv, wd);
      tau_group<LAYOUT, true>(wd, k0, n, smu, stride, acc, cur, mu);
    }
  }
  for (; k0 + kLook <= n; k0 += kLook) {
    uint32_t wd[kLook];
    gather_group<LAYOUT>(V, r, k0, h, ta, hv, wd);
    tau_group<LAYOUT, false>(wd, k0, n, smu, stride, acc, cur, mu);
  }
  if (k0 < n) {
    uint32_t wd[kLook];
    gather_group<LAYOUT>(V, r, k0, h, ta, hv, wd);
    tau_group<LAYOUT, true>(wd, k0, n, smu, stride, acc, cur, mu);
  }
  nsteps += (unsigned long long)n;
  return acc * h;
}

// Optical depths at two energies along the same march (the expected-value
// score's Compton term at E' and Rayleigh term at E share the midpoints, so
// they share the gathers); material attenuation read from the tables at the
// located energies (ia, fa) and (ib, fb) when the material changes.
template <int LAYOUT>
__device__ __forceinline__ float2 march_tau2(const VolumeView& V, float3 x, float3 w, float t1, float step,
                                             const SmemTables& T, int ia, float fa, int ib, float fb,
                                             unsigned long long& nsteps) {
  float ta, tb;
  if (!clip_box(V, x, w, 0.f, t1, ta, tb)) return make_float2(0.f, 0.f);
  const float L = tb - ta;
  const int n = step_count(L, step);
  const float h = L / (float)n;
  VoxRay r;
  r.set(V, x, w);
  const float3 hv = make_float3(h * r.vw.x, h * r.vw.y, h * r.vw.z);
  float acc_a = 0.f, acc_b = 0.f, mu_a = 0.f, mu_b = 0.f;
  int cur = -1;
  for (int k0 = 0; k0 < n; k0 += kLook) {
    uint32_t wd[kLook];
    gather_group<LAYOUT>(V, r, k0, h, ta, hv, wd);
#pragma unroll
    for (int u = 0; u < kLook; ++u) {
      if (k0 + u < n) {
        const int m = vox_mat(wd[u]);
        if (m != cur) {
          cur = m;
          mu_a = 0.1f * T.at(TAB_TOT, m, ia, fa);
          mu_b = 0.1f * T.at(TAB_TOT, m, ib, fb);
        }
        const float rho = vox_rho(wd[u]);
        acc_a = fmaf(mu_a, rho, acc_a);
        acc_b = fmaf(mu_b, rho, acc_b);
      }
    }
  }
  nsteps += (unsigned long long)n;
  return make_float2(acc_a * h, acc_b * h);
}

// Optical depths through the mesh bodies from x to x + t1 w (exact chords):
// one descent gives the column masses, then one sum per energy.
__device__ __forceinline__ float mesh_tau(const MeshView& M, int nm, float3 x, float3 w, float t1, const float* smu,
                                          int stride, unsigned long long& nsteps) {
  float rl[kMaxMat];
#pragma unroll
  for (int m = 0; m < kMaxMat; ++m) rl[m] = 0.f;
  nsteps += (unsigned long long)mesh::mesh_rhoL(M, x, w, t1, rl, false);
  float tau = 0.f;
  for (int m = 0; m < nm; ++m) tau = fmaf(smu[m * stride], rl[m], tau);
  return tau;
}
__device__ __forceinline__ float2 mesh_tau2(const MeshView& M, float3 x, float3 w, float t1, const SmemTables& T,
                                            int ia, float fa, int ib, float fb, unsigned long long& nsteps) {
  float rl[kMaxMat];
#pragma unroll
  for (int m = 0; m < kMaxMat; ++m) rl[m] = 0.f;
  nsteps += (unsigned long long)mesh::mesh_rhoL(M, x, w, t1, rl, false);
  float a = 0.f, b = 0.f;
  for (int m = 0; m < T.n_mat; ++m) {
    a = fmaf(0.1f * T.at(TAB_TOT, m, ia, fa), rl[m], a);
    b = fmaf(0.1f * T.at(TAB_TOT, m, ib, fb), rl[m], b);
  }
  return make_float2(a, b);
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

// Doppler broadening (impulse approximation).  Element i's electrons share the
// hydrogen-like orbital behind the form factor (exponent zeta_i = 2 pi a0 /
// sqrt(b_i), atomic units), Compton profile J_i ~ (1 + (p_z / zeta_i)^2)^-3.
// A scatter through cos(theta) = c picks element i with probability
// w_i S_i(x) / S_mol(x), draws p_z from J_i (Cauchy proposal, acceptance
// (1 + t^2)^-2) and solves P sqrt(1 + tau^2 - 2 tau c) = tau (1 + kappa (1 - c)) - 1
// for tau = E'/E (P = p_z / m_e c); a draw without a root in 0 < tau <= 1 is
// redrawn.  Three draws per try, from the given stream.
__device__ __forceinline__ float doppler_tau(float kappa, float c, float P) {
  const float a = fmaf(kappa, 1.f - c, 1.f);
  const float P2 = P * P;
  const float den = a * a - P2;
  if (!(den > 0.f)) return 0.f;
  // (a - P^2 c)^2 - (a^2 - P^2)(1 - P^2), rearranged to avoid cancellation at small P
  const float D = P2 * (a * a - 2.f * a * c + 1.f) + P2 * P2 * (c * c - 1.f);
  if (!(D >= 0.f)) return 0.f;
  const float t = (a - P2 * c + copysignf(sqrtf(D), P)) / den;
  if (!(t > 0.f && t <= 1.f)) return 0.f;
  if (P != 0.f && (a * t - 1.f) * P < 0.f) return 0.f;
  return t;
}

__device__ __forceinline__ float sample_doppler(Rng& g, const SmemTables& T, int m, float E, float c, bool& fail) {
  constexpr float kZetaC = 2.f * kPi * 0.529177210903f;  // 2 pi a0 (Angstrom)
  constexpr float kAlpha = 1.f / 137.035999084f;
  const float K = (E * T.inv_hc) * (E * T.inv_hc);
  const float u = 0.5f * K * (1.f - c);
  const float kappa = E / T.mec2;
  const float smax = T.smol(m, u);
  const int nc = T.ncomp[m];
  for (int it = 0; it < 256; ++it) {
    const float ue = g.u() * smax, uc = g.u(), ua = g.u();
    int el = nc - 1;
    float cum = 0.f;
    for (int i = 0; i < nc; ++i) {
      const float bu = T.comp[m * kMaxComp + i].y * u;
      const float q = 1.f + bu, q2 = q * q;
      cum += T.compz[m * kMaxComp + i] * (bu * (2.f + bu) * (q2 + 1.f)) / (q2 * q2);
      if (ue < cum) {
        el = i;
        break;
      }
    }
    const float t = tanf(kPi * (uc - 0.5f));
    const float w1 = fmaf(t, t, 1.f);
    if (ua * w1 * w1 > 1.f) continue;
    const float zeta = kZetaC * rsqrtf(T.comp[m * kMaxComp + el].y);
    const float tau = doppler_tau(kappa, c, t * zeta * kAlpha);
    if (tau > 0.f) return tau;
  }
  fail = true;
  return 1.f / fmaf(kappa, 1.f - c, 1.f);
}

// Side stream of pseudo-particle k (its counter block k = k0 + s): blocks
// (2^31 | k << 6 | j, angle, h_lo, h_hi), disjoint from every history's own blocks.
__device__ __forceinline__ Rng side_stream(uint2 key, uint32_t k, uint32_t a, uint32_t hlo, uint32_t hhi) {
  Rng d;
  d.key = key;
  d.ctr = make_uint4(0x80000000u | (k << 6), a, hlo, hhi);
  d.idx = 4;
  return d;
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

__device__ __forceinline__ int transport_shared_pixels_dev(const TransportParams& p) {
  if (p.tally_mode == TALLY_SHARED) return (int)((size_t)p.n_batches * p.n_angles * p.geo.nu * p.geo.nv);
  if (p.tally_mode == TALLY_TILED) return p.n_batches * p.tile_u * p.tile_v;
  return 0;
}

// Interaction records queued by the flight phase for the pseudo-particle
// phase, one slot per thread of the block (structure of arrays).
struct Records {
  float *X, *Y, *Z, *wx, *wy, *wz, *E, *W, *norm, *cb, *sb, *len;
  int* tm;  // type << 8 | material
  uint32_t *hlo, *hhi, *ang, *k0;
};

// One pseudo-particle (eq. Th): random pixel and point in it from the counter
// block k0 + s of the record's stream, scatter-toward-detector pdf, optional
// Russian roulette, attenuation march to the panel, FP64 tally.
// Adds v to the FP64 image at word offset off (see TallyMode).  Lanes that
// reach this point together (the active mask) and share an offset are combined
// by a shuffle sum; the lowest lane of each group does the one add.
// COMBINE = false: one FP64 atomic add per pseudo-particle, no other code
// (the fastest unstratified tally on every workload measured: the tally is one
// add per ~200 march steps).  COMBINE = true: TALLY_WARP, TALLY_SHARED or
// TALLY_TILED as selected at run time.
template <bool COMBINE>
__device__ __forceinline__ void tally_add(const TransportParams& P, float* s_img, size_t off, float v);

template <>
__device__ __forceinline__ void tally_add<false>(const TransportParams& P, float*, size_t off, float v) {
  atomicAdd(P.tally + off, (double)v);
}

__device__ __noinline__ void tally_combine(const TransportParams& P, float* s_img, size_t off, float v) {
  const unsigned act = __activemask();
  const unsigned peers = __match_any_sync(act, (unsigned long long)off);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  float sum = 0.f;
  for (unsigned m = peers; m; m &= m - 1) sum += __shfl_sync(peers, v, __ffs(m) - 1);
  if (lane != leader) return;
  if (P.tally_mode == TALLY_SHARED || P.tally_mode == TALLY_TILED) atomicAdd(s_img + off, sum);
  else atomicAdd(P.tally + off, (double)sum);
}

template <>
__device__ __forceinline__ void tally_add<true>(const TransportParams& P, float* s_img, size_t off, float v) {
  tally_combine(P, s_img, off, v);
}

// Pixels a block's pseudo-particles aim at under the tile-stratified tally: the
// current chunk's tile (origin, width, height) and the score factor T P_t / P
// (weight T, pixel drawn among the tile's P_t instead of the panel's P).
struct TileSel {
  int u0, v0, wt, ht;
  float scale;
};

template <int LAYOUT, bool COMBINE, bool EV, bool DOP>
__device__ __forceinline__ void pseudo_particle(const TransportParams& P, const SmemTables& T, const Records& R,
                                                int r, int s, float* my_mu, int stride, float nee_scale,
                                                uint32_t npix, size_t img, Counters& C, float* s_img,
                                                uint2 key, const TileSel& ts) {
  const VolumeView& V = P.vol;
  const GeomView& G = P.geo;
  const uint32_t hlo = R.hlo[r], hhi = R.hhi[r], a = R.ang[r];
  const uint4 blk = philox4x32_10(make_uint4(R.k0[r] + (uint32_t)s, a, hlo, hhi), key);
  const float va = Rng::u01(blk.y), vb = Rng::u01(blk.z), vr = Rng::u01(blk.w);
  const unsigned long long hh = ((unsigned long long)hhi << 32) | hlo;
  // batch of the variance estimate: h mod n_batches; under the tile-stratified tally
  // floor(h / T) mod n_batches, so that every batch holds its share of every tile
  const unsigned long long hb = (COMBINE && P.tally_mode == TALLY_TILED) ? hh / (unsigned long long)P.n_tiles : hh;
  const int bt = P.n_batches > 1 ? (int)(hb % (unsigned long long)P.n_batches) : 0;
  uint32_t pi, pj;
  size_t off;
  float tscale = 1.f;
  // the pixel: drawn uniformly (the block's first word), or under forced
  // detection the s-th pixel itself (every pixel once per interaction)
  if (COMBINE && P.tally_mode == TALLY_TILED) {
    const uint32_t Pt = (uint32_t)(ts.wt * ts.ht);
    const uint32_t pt = P.forced ? (uint32_t)s : __umulhi(blk.x, Pt);
    pi = (uint32_t)ts.u0 + pt % (uint32_t)ts.wt;
    pj = (uint32_t)ts.v0 + pt / (uint32_t)ts.wt;
    off = (size_t)bt * Pt + pt;
    tscale = ts.scale;
  } else {
    const uint32_t pix = P.forced ? (uint32_t)s : __umulhi(blk.x, npix);
    pi = pix % (uint32_t)G.nu;
    pj = pix / (uint32_t)G.nu;
    off = ((size_t)bt * P.n_angles + a) * img + pix;
  }
  const float cb = R.cb[r], sb = R.sb[r];
  Pose ps;
  const float rr0 = G.sod - G.sdd;
  ps.c = make_float3(rr0 * cb, rr0 * sb, 0.f);
  ps.eu = make_float3(-sb, cb, 0.f);
  ps.n = make_float3(cb, sb, 0.f);
  const float3 x = make_float3(R.X[r], R.Y[r], R.Z[r]);
  const float3 w = make_float3(R.wx[r], R.wy[r], R.wz[r]);
  const float3 Pp = det_point(G, ps, (float)pi + va, (float)pj + vb);
  const float3 DD = sub3(Pp, x);
  const float dd2 = dot3(DD, DD);
  const float idd = rsqrtf(dd2);
  const float3 dir = make_float3(DD.x * idd, DD.y * idd, DD.z * idd);
  // the scattering cosine, clamped: two rounded unit vectors can give a dot product a unit past +-1, outside
  // the domain of the pdfs and of the Doppler kinematics
  const float lam = fminf(fmaxf(dot3(w, dir), -1.f), 1.f);
  const float cosg = -dot3(dir, ps.n);
  const int tm = R.tm[r];
  const int type = tm >> 8, mint = tm & 255;
  const float E = R.E[r];
  if (EV) {
    // expected value over the interaction type: (mu_incoh/mu) Compton term at
    // E' + (mu_coh/mu) Rayleigh term at E, attenuations from one shared march
    int i0, i1;
    float f0, f1;
    T.locate(E, i0, f0);
    const float pe = T.at(TAB_PE, mint, i0, f0), in = T.at(TAB_IN, mint, i0, f0), co = T.at(TAB_CO, mint, i0, f0);
    const float imu = 1.f / (pe + in + co);
    const float ratio = 1.f / fmaf(E / T.mec2, 1.f - lam, 1.f);
    const float Ep = E * ratio;
    const float K = (E * T.inv_hc) * (E * T.inv_hc);
    const float u = 0.5f * K * (1.f - lam);
    const float pc = ratio * ratio * (ratio + 1.f / ratio - 1.f + lam * lam) *
                     (T.bound ? T.smol(mint, u) / T.at(TAB_IINC, mint, i0, f0) : 1.f / T.kn_norm(i0, f0));
    float F2 = 0.f;
    const int nc = T.ncomp[mint];
    const float2* cp = T.comp + mint * kMaxComp;
    for (int i = 0; i < nc; ++i) {
      const float q = fmaf(cp[i].y, u, 1.f);
      const float q2 = q * q;
      F2 += cp[i].x / (q2 * q2);
    }
    const float pr = (1.f + lam * lam) * F2 * (1.f / T.at(TAB_ICOH, mint, i0, f0));
    float Ep_s = Ep;
    if (DOP) {
      bool df = false;
      Rng d = side_stream(key, R.k0[r] + (uint32_t)s, a, hlo, hhi);
      Ep_s = E * sample_doppler(d, T, mint, E, lam, df);
      if (df) ++C.fail;
    }
    T.locate(Ep_s, i1, f1);
    const float gw = R.W[r] * cosg * (nee_scale * tscale) / dd2;
    float xc = gw * (in * imu) * T.response(i1, f1, Ep_s) * pc;
    float xr = gw * (co * imu) * T.response(i0, f0, E) * pr;
    ++C.nee_rays;
    const float x0 = xc + xr;
    if (P.rr_threshold > 0.f && x0 < P.rr_threshold) {
      if (vr >= x0 / P.rr_threshold) return;
      const float sc = P.rr_threshold / x0;
      xc *= sc;
      xr *= sc;
    }
    float2 tp;
    if constexpr (LAYOUT == GEO_MESH) tp = mesh_tau2(P.mesh, x, dir, dd2 * idd, T, i1, f1, i0, f0, C.nee_steps);
    else tp = march_tau2<LAYOUT>(V, x, dir, dd2 * idd, P.step, T, i1, f1, i0, f0, C.nee_steps);
    tally_add<COMBINE>(P, s_img, off, xc * __expf(-tp.x) + xr * __expf(-tp.y));
    return;
  }
  float Ep, p;
  if (type == 1) {
    const float ratio = 1.f / fmaf(E / T.mec2, 1.f - lam, 1.f);
    Ep = E * ratio;
    p = ratio * ratio * (ratio + 1.f / ratio - 1.f + lam * lam) * R.norm[r];
    if (T.bound) p *= T.smol(mint, 0.5f * (E * T.inv_hc) * (E * T.inv_hc) * (1.f - lam));
    if (DOP) {
      bool df = false;
      Rng d = side_stream(key, R.k0[r] + (uint32_t)s, a, hlo, hhi);
      Ep = E * sample_doppler(d, T, mint, E, lam, df);
      if (df) ++C.fail;
    }
  } else {
    Ep = E;
    const float K = (E * T.inv_hc) * (E * T.inv_hc);
    const float u = 0.5f * K * (1.f - lam);
    float F2 = 0.f;
    const int nc = T.ncomp[mint];
    const float2* cp = T.comp + mint * kMaxComp;
    for (int i = 0; i < nc; ++i) {
      const float q = fmaf(cp[i].y, u, 1.f);
      const float q2 = q * q;
      F2 += cp[i].x / (q2 * q2);
    }
    p = (1.f + lam * lam) * F2 * R.norm[r];
  }
  int ei;
  float ef;
  T.locate(Ep, ei, ef);
  float x0 = R.W[r] * T.response(ei, ef, Ep) * p * cosg * (nee_scale * tscale) / dd2;
  ++C.nee_rays;
  if (P.rr_threshold > 0.f && x0 < P.rr_threshold) {
    if (vr >= x0 / P.rr_threshold) return;
    x0 = P.rr_threshold;
  }
  fill_mu(T, ei, ef, my_mu, stride);
  float tp;
  if constexpr (LAYOUT == GEO_MESH) tp = mesh_tau(P.mesh, T.n_mat, x, dir, dd2 * idd, my_mu, stride, C.nee_steps);
  else tp = march_tau<LAYOUT>(V, x, dir, dd2 * idd, P.step, my_mu, stride, C.nee_steps);
  tally_add<COMBINE>(P, s_img, off, x0 * __expf(-tp));
}

#ifndef MC_MIN_BLOCKS
#define MC_MIN_BLOCKS 2
#endif
// The same for the brick layout (volumes in HBM, where more warps in flight hide
// the longer gathers).
#ifndef MC_MIN_BLOCKS_BRICK
#define MC_MIN_BLOCKS_BRICK MC_MIN_BLOCKS
#endif
// Flights through a linear-layout volume sum each group's optical depth
// branch-free before looking for the interaction step (1), or test every step
// (0); both give the same interaction points.
#ifndef MC_FLIGHT_GROUP
#define MC_FLIGHT_GROUP 1
#endif
// Flights per lane and iteration with the per-warp phases (the block-wide
// phases of the combined tallies take one).
#ifndef MC_FLIGHTS_PER_ITER
#define MC_FLIGHTS_PER_ITER 1
#endif
// Pseudo-particle jobs are handed out longest records first: records are
// bucketed by the chord from the interaction point to the volume boundary
// toward the panel centre, and each warp fetches the next 32 jobs.
#ifndef MC_SORT
#define MC_SORT 1
#endif
constexpr int kBuckets = 16;

// Tile-stratified tally: the block's current chunk of histories, all of one
// angle and one tile (histories h with (h + o_a) mod T = t, o_a the angle's
// tile offset, uniform on [0, T) from the Philox block (2^32 - 1, a, 2^32 - 1,
// 2^32 - 1)).  Local index j runs over [j, j_end); history = first + T j.
struct TileChunk {
  unsigned long long j, j_end, first;
  int a, u0, v0, wt, ht, done;
};

// Thread 0 takes chunks from the global counter until a non-empty one (or none is left).
__device__ void tile_fetch(const TransportParams& P, uint2 key, TileChunk& c) {
  const unsigned long long T = (unsigned long long)P.n_tiles, K = P.tile_k;
  const unsigned long long hb = P.h_begin, he = P.h_begin + P.h_count;
  if (T == 0 || K == 0 || P.tile_chunk == 0) {
    c.done = 1;
    return;
  }
  for (;;) {
    const unsigned long long id = atomicAdd(P.stats + S_WORK, 1ull);
    if (id >= P.n_chunks) {
      c.done = 1;
      return;
    }
    const int a = (int)(id / (T * K));
    const unsigned long long t = (id / K) % T, k = id % K;
    const uint4 ob = philox4x32_10(make_uint4(0xFFFFFFFFu, (uint32_t)a, 0xFFFFFFFFu, 0xFFFFFFFFu), key);
    const unsigned long long o = ((unsigned long long)ob.x * T) >> 32;
    const unsigned long long res = (t + T - o) % T;  // h = res (mod T)
    const unsigned long long first = hb + (res + T - hb % T) % T;
    const unsigned long long cnt = first < he ? (he - first - 1) / T + 1 : 0ull;
    const unsigned long long jb = k * P.tile_chunk;
    const unsigned long long je = min(jb + P.tile_chunk, cnt);
    if (jb >= je) continue;
    c.j = jb;
    c.j_end = je;
    c.first = first;
    c.a = a;
    c.u0 = (int)(t % (unsigned long long)P.n_tu) * P.tile_u;
    c.v0 = (int)(t / (unsigned long long)P.n_tu) * P.tile_v;
    c.wt = min(P.tile_u, P.geo.nu - c.u0);
    c.ht = min(P.tile_v, P.geo.nv - c.v0);
    c.done = 0;
    return;
  }
}

template <int LAYOUT, bool COMBINE, bool EV, bool DOP>
__global__ void __launch_bounds__(256, LAYOUT == VOX_BRICK ? MC_MIN_BLOCKS_BRICK : MC_MIN_BLOCKS)
    k_transport(const TransportParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ int s_nrec, s_job;
  __shared__ int s_bucket[kBuckets + 1];
  __shared__ TileChunk s_tc;
  const bool tiled = COMBINE && P.tally_mode == TALLY_TILED;
  // Block-wide phases (a block queue of records, jobs sorted over the block)
  // for the combined tallies, whose shared images need them, and for volumes
  // in HBM (brick layout), where they were measured faster than per-warp
  // phases; per-warp phases otherwise.
  constexpr bool kBlockPhases = COMBINE || LAYOUT == VOX_BRICK;
  constexpr int kFlights = kBlockPhases ? 1 : MC_FLIGHTS_PER_ITER;
  const int nm = P.tab.n_mat, ns = P.tab.n_stage;
  const int nb = P.spec.n_bins;
  const int B = blockDim.x;
  // shared layout: [table blob][prefix u64 (nb+1)][energy f32 nb][wbin f32 nb]
  //                [mu columns f32 kMaxMat x B][records 16 x B words]
  float2* s_blob = reinterpret_cast<float2*>(smem);
  unsigned long long* s_pre = reinterpret_cast<unsigned long long*>(smem + P.tab.blob_bytes);
  float* s_E = reinterpret_cast<float*>(s_pre + nb + 1);
  float* s_wb = s_E + nb;
  float* s_mu = s_wb + nb;
  float* rec = s_mu + kMaxMat * B;
  Records R;
  R.X = rec; R.Y = rec + B; R.Z = rec + 2 * B; R.wx = rec + 3 * B; R.wy = rec + 4 * B; R.wz = rec + 5 * B;
  R.E = rec + 6 * B; R.W = rec + 7 * B; R.norm = rec + 8 * B; R.cb = rec + 9 * B; R.sb = rec + 10 * B;
  R.tm = reinterpret_cast<int*>(rec + 11 * B);
  R.hlo = reinterpret_cast<uint32_t*>(rec + 12 * B);
  R.hhi = reinterpret_cast<uint32_t*>(rec + 13 * B);
  R.ang = reinterpret_cast<uint32_t*>(rec + 14 * B);
  R.k0 = reinterpret_cast<uint32_t*>(rec + 15 * B);
  R.len = rec + 16 * B;
  int* s_ord = reinterpret_cast<int*>(rec + 17 * B);  // record order for the pseudo-particle phase
  float* s_img = rec + 18 * B;                         // shared tally image (TALLY_SHARED) or tile (TALLY_TILED)
  // the shared image's size; the host sizes the dynamic shared memory with the same rule
  const int n_simg = COMBINE ? transport_shared_pixels_dev(P) : 0;
  {
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const size_t need = (size_t)P.tab.blob_bytes + (size_t)(nb + 1) * 8 + (size_t)nb * 8 + (size_t)kMaxMat * B * 4 +
                        (size_t)18 * B * 4 + (size_t)n_simg * 4;
    if (need > dyn) {  // uniform over the block: no thread has reached a barrier yet
      if (threadIdx.x == 0) atomicAdd(P.stats + S_BAD_SMEM, 1ull);
      return;
    }
  }
  for (int i = threadIdx.x; i < n_simg; i += B) s_img[i] = 0.f;

  const bool staged = stage_bulk(s_blob, P.tab.blob, P.tab.blob_bytes, &bar);
  for (int i = threadIdx.x; i <= nb; i += B) s_pre[i] = P.spec.prefix[i];
  for (int i = threadIdx.x; i < nb; i += B) {
    s_E[i] = P.spec.energy[i];
    s_wb[i] = P.spec.wbin[i];
  }
  if (threadIdx.x == 0) {
    s_nrec = 0;
    s_tc.done = 0;
  }
  __syncthreads();
  if (!staged) {
    if (threadIdx.x == 0) atomicAdd(P.stats + S_INTERNAL, 1ull);
    return;
  }
  SmemTables T;
  T.tab = s_blob;
  T.jkn = reinterpret_cast<const float2*>(smem + tab_off_jkn(nm, ns));
  T.eta = reinterpret_cast<const float2*>(smem + tab_off_eta(nm, ns));
  T.use_eta = P.tab.use_eta;
  T.comp = reinterpret_cast<const float2*>(smem + tab_off_comp(nm, ns));
  T.compz = reinterpret_cast<const float*>(smem + tab_off_compz(nm, ns));
  T.bound = P.tab.bound;
  T.ncomp = reinterpret_cast<const int*>(smem + tab_off_ncomp(nm, ns));
  T.n_mat = nm;
  T.n_stage = ns;
  T.E0 = P.tab.E0;
  T.inv_dE = P.tab.inv_dE;
  T.mec2 = P.tab.mec2;
  T.inv_hc = P.tab.inv_hc;

  const VolumeView& V = P.vol;
  const GeomView& G = P.geo;
  float* my_mu = s_mu + threadIdx.x;
  const uint32_t npix = (uint32_t)G.nu * (uint32_t)G.nv;
  const float A_det = (float)G.nu * G.pu * (float)G.nv * G.pv;
  const size_t img = (size_t)npix;
  // pseudo-particles per interaction: n_split, or under forced detection one per
  // pixel of the panel or of the block's current tile
  auto pseudo_count = [&]() -> int {
    if (!P.forced) return P.n_split;
    return tiled ? s_tc.wt * s_tc.ht : (int)npix;
  };

  Counters C = {};
  const unsigned long long total = (unsigned long long)P.n_angles * P.h_count;
  const unsigned long long stride = (unsigned long long)gridDim.x * B;
  unsigned long long next = (unsigned long long)blockIdx.x * B + threadIdx.x;

  // photon state
  bool alive = false;
  unsigned long long h = 0;
  int a = 0, order = 0;
  float3 x = make_float3(0.f, 0.f, 0.f), w = x;
  float E = 0.f, W = 0.f, cb = 1.f, sb = 0.f;
  float t_start = 0.f;  // parameter of the photon's position on the ray x + t w (negative on a first flight)
  Rng g;
  const unsigned long long seed = P.seed_dev ? __ldg(P.seed_dev) : P.seed;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  g.init(0, 0, seed);
  if (tiled) {
    if (threadIdx.x == 0) tile_fetch(P, key, s_tc);
    __syncthreads();
  }

  for (;;) {
    if (tiled && s_tc.done) break;
    // ---- flight phase: one free flight per live photon; with the per-warp
    // phases a lane whose photon leaves without a record (escape, absorption)
    // starts the next history in the same iteration, up to kFlights flights
    bool has_rec = false;
    for (int fl = 0; fl < kFlights; ++fl) {
      bool fresh = false;
      if (tiled) {
        if (!alive) {
          const unsigned long long j = atomicAdd(&s_tc.j, 1ull);
          if (j < s_tc.j_end) {
            a = s_tc.a;
            h = s_tc.first + (unsigned long long)P.n_tiles * j;
            fresh = true;
          }
        }
      } else if (!alive && next < total) {
        a = (int)(next / P.h_count);
        h = P.h_begin + (next - (unsigned long long)a * P.h_count);
        next += stride;
        fresh = true;
      }
      if (fresh) {
        int lo = 0, hi = nb - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_pre[mid] <= h) lo = mid;
          else hi = mid - 1;
        }
        E = s_E[lo];
        g.init(h, (uint32_t)a, seed);
        sincosf(__ldg(P.angles + a), &sb, &cb);
        const float ua = g.u(), ub = g.u();
        // toward a uniform point Q of the panel: D = Q - s = -SDD n + u e_u + v e_z
        // (n = (cos b, sin b, 0), e_u = (-sin b, cos b, 0)), d^2 = SDD^2 + u^2 + v^2
        const float u = (ua * (float)G.nu - 0.5f * (float)G.nu) * G.pu;
        const float v = (ub * (float)G.nv - 0.5f * (float)G.nv) * G.pv;
        const float r2 = fmaf(u, u, v * v);
        const float d2 = fmaf(G.sdd, G.sdd, r2);
        const float d = sqrtf(d2);
        w = make_float3(fmaf(-G.sdd, cb, -u * sb) / d, fmaf(-G.sdd, sb, u * cb) / d, v / d);
        W = s_wb[lo] * A_det * (G.sdd / d) / (4.f * kPi * d2);
        if constexpr (LAYOUT == GEO_MESH) {
          // the bodies' crossings are collected along the half-line from the source
          x = make_float3(G.sod * cb, G.sod * sb, 0.f);
          t_start = 0.f;
        } else {
          // the first flight runs from the ray's point nearest the isocentre,
          // o = (SOD / d^2) ((u^2 + v^2) n + SDD (u e_u + v e_z)), with the source at
          // t = -SOD SDD / d: its midpoints carry rounding of the volume's size, not
          // of the source distance
          const float k = G.sod / d2;
          x = make_float3(k * fmaf(r2, cb, -G.sdd * (u * sb)), k * fmaf(r2, sb, G.sdd * (u * cb)), k * (G.sdd * v));
          t_start = -G.sod * G.sdd / d;
        }
        order = 0;
        alive = true;
        ++C.hist;
      }
      if (alive) {
        const float tau_star = -logf(g.u());
        float ta, tb;
        bool hit = false;
        float tint = 0.f;
        int mint = 0;
        if constexpr (LAYOUT == GEO_MESH) {
          fill_mu(T, E, my_mu, B);
          hit = mesh::mesh_flight(P.mesh, x, w, tau_star, my_mu, B, tint, mint, C.flight_steps);
          (void)ta;
          (void)tb;
        } else if (clip_box(V, x, w, t_start, __int_as_float(0x7f800000), ta, tb)) {
          fill_mu(T, E, my_mu, B);
          const float L = tb - ta;
          const int n = step_count(L, P.step);
          const float hh = L / (float)n;
          VoxRay vr;
          vr.set(V, x, w);
          const float3 hv = make_float3(hh * vr.vw.x, hh * vr.vw.y, hh * vr.vw.z);
          float tau = 0.f, mu_m = 0.f;
          int cur = -1, k = n;
          // the step whose optical depth reaches tau* holds the interaction,
          // placed inside it by a linear solve
          auto consume = [&](const uint32_t(&wd)[kLook], int k0, bool tail) {
  #pragma unroll
            for (int u = 0; u < kLook; ++u) {
              if (!hit && (!tail || k0 + u < n)) {
                const int m = vox_mat(wd[u]);
                if (m != cur) {
                  cur = m;
                  mu_m = my_mu[m * B];
                }
                const float mu = mu_m * vox_rho(wd[u]);
                if (fmaf(mu, hh, tau) >= tau_star) {
                  tint = fmaf((float)(k0 + u), hh, ta) + (tau_star - tau) / mu;
                  mint = cur;
                  hit = true;
                  k = k0 + u;
                } else {
                  tau = fmaf(mu, hh, tau);
                }
              }
            }
          };
          // volume in L2 (linear layout): a group's optical depth is summed
          // branch-free, with the same per-step products and sums as above; the
          // depth never decreases, so only the group whose end reaches tau* is
          // walked again step by step (consume) to place the interaction
          auto group_reaches = [&](const uint32_t(&wd)[kLook], int k0, bool tail) -> bool {
            float t = tau;
  #pragma unroll
            for (int u = 0; u < kLook; ++u) {
              const float tn = fmaf(my_mu[vox_mat(wd[u]) * B] * vox_rho(wd[u]), hh, t);
              t = (!tail || k0 + u < n) ? tn : t;
            }
            if (t >= tau_star) return true;
            tau = t;
            return false;
          };
          int k0 = 0;
          if (LAYOUT == VOX_BRICK && MC_BRICK_NOSPLIT) {
            for (; k0 < n && !hit; k0 += kLook) {
              uint32_t wd[kLook];
              gather_group<LAYOUT>(V, vr, k0, hh, ta, hv, wd);
              consume(wd, k0, true);
            }
          }
          for (; k0 + kLook <= n && !hit; k0 += kLook) {
            uint32_t wd[kLook];
            gather_group<LAYOUT>(V, vr, k0, hh, ta, hv, wd);
            if (LAYOUT != VOX_LIN || !MC_FLIGHT_GROUP || group_reaches(wd, k0, false)) consume(wd, k0, false);
          }
          if (k0 < n && !hit) {
            uint32_t wd[kLook];
            gather_group<LAYOUT>(V, vr, k0, hh, ta, hv, wd);
            if (LAYOUT != VOX_LIN || !MC_FLIGHT_GROUP || group_reaches(wd, k0, true)) consume(wd, k0, true);
          }
          C.flight_steps += (unsigned long long)(hit ? k + 1 : n);
        }
        if (!hit) {
          ++C.escape;
          alive = false;
        } else {
          x = make_float3(fmaf(tint, w.x, x.x), fmaf(tint, w.y, x.y), fmaf(tint, w.z, x.z));
          t_start = 0.f;
          int ti;
          float tf;
          T.locate(E, ti, tf);
          const float pe = T.at(TAB_PE, mint, ti, tf), in = T.at(TAB_IN, mint, ti, tf),
                      co = T.at(TAB_CO, mint, ti, tf);
          const float ut = g.u() * (pe + in + co);
          const int type = ut < pe ? 0 : (ut < pe + in ? 1 : 2);
          if (type == 0) ++C.photo;
          else if (type == 1) ++C.compton;
          else ++C.rayleigh;
          // absorption sites score only in expected-value mode
          if (type == 0 && !EV) {
            alive = false;
          } else {
            // queue the interaction; its pseudo-particles use the next counter blocks, one each
            g.align();
            // the block-wide queue (block-wide phases) or the lane's own slot (per-warp phases)
            int r;
            if constexpr (kBlockPhases) {
              r = atomicAdd(&s_nrec, 1);
            } else {
              r = threadIdx.x;
              has_rec = true;
            }
            R.X[r] = x.x; R.Y[r] = x.y; R.Z[r] = x.z;
            R.wx[r] = w.x; R.wy[r] = w.y; R.wz[r] = w.z;
            R.E[r] = E; R.W[r] = W; R.cb[r] = cb; R.sb[r] = sb;
            R.norm[r] = type == 1 ? 1.f / (T.bound ? T.at(TAB_IINC, mint, ti, tf) : T.kn_norm(ti, tf))
                                  : 1.f / T.at(TAB_ICOH, mint, ti, tf);
            R.tm[r] = (type << 8) | mint;
            R.hlo[r] = (uint32_t)h; R.hhi[r] = (uint32_t)(h >> 32); R.ang[r] = (uint32_t)a;
            R.k0[r] = g.ctr.x;
            g.ctr.x += (uint32_t)pseudo_count();
            {
              // length key: chord toward the panel centre
              const float rr0 = G.sod - G.sdd;
              const float3 toc = make_float3(rr0 * cb - x.x, rr0 * sb - x.y, -x.z);
              const float il = rsqrtf(dot3(toc, toc));
              float ca, cbb;
              R.len[r] = clip_box(V, x, make_float3(toc.x * il, toc.y * il, toc.z * il), 0.f,
                                  __int_as_float(0x7f800000), ca, cbb) ? cbb : 0.f;
            }
            // new direction (an absorption ends the photon)
            if (type == 0) alive = false;
          }
          if (alive) {
            bool fail = false;
            float ct, Enew = E;
            if (type == 1) {
              const float alpha = E / T.mec2;
              float rk = kahn(g, alpha, fail);
              ct = 1.f - (rk - 1.f) / alpha;
              if (T.bound) {
                // scattering function: accept Kahn's angle with probability S_mol(x) / S_mol(inf)
                const float K = (E * T.inv_hc) * (E * T.inv_hc);
                const float smax = T.smol_max(mint);
                for (int it = 0; it < 100000 && !fail; ++it) {
                  if (g.u() * smax <= T.smol(mint, 0.5f * K * (1.f - ct))) break;
                  rk = kahn(g, alpha, fail);
                  ct = 1.f - (rk - 1.f) / alpha;
                  if (it == 99999) fail = true;
                }
              }
              Enew = DOP ? E * sample_doppler(g, T, mint, E, ct, fail) : E / rk;
            } else {
              ct = rayleigh(g, T, mint, E, fail);
            }
            const float phi = 2.f * kPi * g.u();
            if (fail) ++C.fail;
            w = rotate(w, ct, phi);
            E = Enew;
            ++order;
            if (E < 1.f) {
              alive = false;
            } else if (order >= P.max_order) {
              ++C.limit;
              alive = false;
            }
          }
        }
      }
      if (has_rec || !(alive || next < total)) break;
    }
    if constexpr (!kBlockPhases) {
      // ---- pseudo-particle phase, per warp (no block barrier): the warp marches
      // its own lanes' queued rays, records ranked by chord length, longest first
      const unsigned recmask = __ballot_sync(0xffffffffu, has_rec);
      const int lane = threadIdx.x & 31, wbase = threadIdx.x - lane;
      const float my_len = has_rec ? R.len[threadIdx.x] : 0.f;
      int rank = 0;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float lj = __shfl_sync(0xffffffffu, my_len, j);
        rank += (((recmask >> j) & 1u) != 0u) && (lj > my_len || (lj == my_len && j < lane));
      }
      if (has_rec) s_ord[wbase + rank] = threadIdx.x;
      __syncwarp();
      const int n_split = pseudo_count();
      const int n_jobs = __popc(recmask) * n_split;
      // weight of a pseudo-particle: pixel area x P / n_split / (2 pi) (eq. Th)
      const float nee_scale = G.pu * G.pv * ((float)npix / (float)n_split) / (2.f * kPi);
      const TileSel ts = {0, 0, 0, 0, 1.f};
      for (int base = 0; base < n_jobs; base += 32) {
        const int j = base + lane;
        if (j < n_jobs) {
          const int q = j / n_split;
          pseudo_particle<LAYOUT, COMBINE, EV, DOP>(P, T, R, s_ord[wbase + q], j - q * n_split, my_mu, B, nee_scale,
                                                    npix, img, C, s_img, key, ts);
        }
      }
      // every lane has read the warp's records before they are overwritten
      __syncwarp();
      if (!__any_sync(0xffffffffu, alive || next < total)) break;
      continue;
    }
    __syncthreads();
    // ---- pseudo-particle phase: the block marches every queued ray together
    const int nrec = s_nrec;
    const int n_split = pseudo_count();
    const int n_jobs = nrec * n_split;
    // weight of a pseudo-particle: pixel area x P / n_split / (2 pi) (eq. Th)
    const float nee_scale = G.pu * G.pv * ((float)npix / (float)n_split) / (2.f * kPi);
    TileSel ts = {0, 0, 0, 0, 1.f};
    if (tiled) {
      ts.u0 = s_tc.u0;
      ts.v0 = s_tc.v0;
      ts.wt = s_tc.wt;
      ts.ht = s_tc.ht;
      ts.scale = (float)P.n_tiles * (float)(s_tc.wt * s_tc.ht) / (float)npix;
    }
#if MC_SORT
    {
      // counting sort of the records into length buckets, longest first
      const float lmax = 2.f * sqrtf(V.hx * V.hx + V.hy * V.hy + V.hz * V.hz);  // box diagonal
      if (threadIdx.x <= kBuckets) s_bucket[threadIdx.x] = 0;
      if (threadIdx.x == 0) s_job = 0;
      __syncthreads();
      int bk = 0, slot = 0;
      if (threadIdx.x < nrec) {
        bk = kBuckets - 1 - min(kBuckets - 1, (int)(R.len[threadIdx.x] * (float)kBuckets / lmax));
        slot = atomicAdd(&s_bucket[bk + 1], 1);
      }
      __syncthreads();
      if (threadIdx.x == 0)
        for (int b = 1; b <= kBuckets; ++b) s_bucket[b] += s_bucket[b - 1];
      __syncthreads();
      if (threadIdx.x < nrec) s_ord[s_bucket[bk] + slot] = threadIdx.x;
      __syncthreads();
      const int lane = threadIdx.x & 31;
      for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&s_job, 32);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_jobs) break;
        const int j = base + lane;
        if (j < n_jobs) {
          const int q = j / n_split;
          pseudo_particle<LAYOUT, COMBINE, EV, DOP>(P, T, R, s_ord[q], j - q * n_split, my_mu, B, nee_scale, npix, img, C, s_img, key, ts);
        }
      }
    }
#else
    for (int j = threadIdx.x; j < n_jobs; j += B) {
      const int r = j / n_split;
      pseudo_particle<LAYOUT, COMBINE, EV, DOP>(P, T, R, r, j - r * n_split, my_mu, B, nee_scale, npix, img, C, s_img, key, ts);
    }
#endif
    const bool more = alive || (tiled ? s_tc.j < s_tc.j_end : next < total);
    __syncthreads();
    if (threadIdx.x == 0) s_nrec = 0;
    if (!__syncthreads_or(more)) {
      if (!tiled) break;
      // the chunk is finished: its tile goes into the FP64 image, then the next chunk
      const int Pt = s_tc.wt * s_tc.ht;
      for (int i = threadIdx.x; i < P.n_batches * Pt; i += B) {
        const float v = s_img[i];
        if (v != 0.f) {
          const int bt = i / Pt, pt = i - bt * Pt;
          const size_t pix = (size_t)(s_tc.v0 + pt / s_tc.wt) * G.nu + (size_t)(s_tc.u0 + pt % s_tc.wt);
          atomicAdd(P.tally + ((size_t)bt * P.n_angles + s_tc.a) * img + pix, (double)v);
          s_img[i] = 0.f;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) tile_fetch(P, key, s_tc);
      __syncthreads();
    }
  }
  if (COMBINE && P.tally_mode == TALLY_SHARED && n_simg) {
    __syncthreads();
    for (int i = threadIdx.x; i < n_simg; i += B)
      if (s_img[i] != 0.f) atomicAdd(P.tally + i, (double)s_img[i]);
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

int transport_shared_pixels(const TransportParams& p) {
  if (p.tally_mode == TALLY_SHARED) return (int)((size_t)p.n_batches * p.n_angles * p.geo.nu * p.geo.nv);
  if (p.tally_mode == TALLY_TILED) return p.n_batches * p.tile_u * p.tile_v;
  return 0;
}

int transport_smem_bytes(const TableView& t, int n_bins, int block, int shared_pixels) {
  return t.blob_bytes + (n_bins + 1) * 8 + n_bins * 8 + kMaxMat * block * 4 + 18 * block * 4 + shared_pixels * 4;
}

namespace {
template <int LAYOUT, bool COMBINE, bool EV, bool DOP>
cudaError_t launch_one(const TransportParams& p, int grid, int block, int smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_transport<LAYOUT, COMBINE, EV, DOP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_transport<LAYOUT, COMBINE, EV, DOP><<<grid, block, smem, s>>>(p);
  return cudaGetLastError();
}
}  // namespace

cudaError_t transport_occupancy(int block, int smem, int* blocks_per_sm, bool mesh, int layout) {
  auto* k = mesh                    ? k_transport<GEO_MESH, false, false, false>
            : layout == VOX_BRICK ? k_transport<VOX_BRICK, false, false, false>
                                  : k_transport<VOX_LIN, false, false, false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, block, smem);
}

cudaError_t launch_transport(const TransportParams& p, int grid, int block, cudaStream_t s) {
  const int smem = transport_smem_bytes(p.tab, p.spec.n_bins, block, transport_shared_pixels(p));
  const bool combine = p.tally_mode != TALLY_GLOBAL;
  const bool ev = p.nee_mode == 1;
  // the mesh geometry takes the global tally (the modes give the same image)
  const int variant = p.geometry == GEO_MESH
                          ? 16 | (ev ? 2 : 0) | (p.doppler ? 1 : 0)
                          : (p.vol.layout == VOX_BRICK ? 8 : 0) | (combine ? 4 : 0) | (ev ? 2 : 0) | (p.doppler ? 1 : 0);
  switch (variant) {
#define MC_LAUNCH(V, L, C, E, D) \
  case V:                        \
    return launch_one<L, C, E, D>(p, grid, block, smem, s);
    MC_LAUNCH(0, VOX_LIN, false, false, false)
    MC_LAUNCH(1, VOX_LIN, false, false, true)
    MC_LAUNCH(2, VOX_LIN, false, true, false)
    MC_LAUNCH(3, VOX_LIN, false, true, true)
    MC_LAUNCH(4, VOX_LIN, true, false, false)
    MC_LAUNCH(5, VOX_LIN, true, false, true)
    MC_LAUNCH(6, VOX_LIN, true, true, false)
    MC_LAUNCH(7, VOX_LIN, true, true, true)
    MC_LAUNCH(8, VOX_BRICK, false, false, false)
    MC_LAUNCH(9, VOX_BRICK, false, false, true)
    MC_LAUNCH(10, VOX_BRICK, false, true, false)
    MC_LAUNCH(11, VOX_BRICK, false, true, true)
    MC_LAUNCH(12, VOX_BRICK, true, false, false)
    MC_LAUNCH(13, VOX_BRICK, true, false, true)
    MC_LAUNCH(14, VOX_BRICK, true, true, false)
    MC_LAUNCH(15, VOX_BRICK, true, true, true)
    MC_LAUNCH(16, GEO_MESH, false, false, false)
    MC_LAUNCH(17, GEO_MESH, false, false, true)
    MC_LAUNCH(18, GEO_MESH, false, true, false)
    MC_LAUNCH(19, GEO_MESH, false, true, true)
#undef MC_LAUNCH
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_finalize(const double* tally, int n_batches, size_t n, float* out, float* var, cudaStream_t s) {
  const int block = 256;
  const int grid = (int)std::min<size_t>((n + block - 1) / block, 152 * 16);
  k_finalize<<<grid, block, 0, s>>>(tally, n_batches, n, out, var);
  return cudaGetLastError();
}

}  // namespace mcx
