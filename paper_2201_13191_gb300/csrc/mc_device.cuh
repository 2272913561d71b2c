// Device helpers of the transport and primary kernels: counter-based random
// numbers, cross-section table lookups, scanner geometry and the fixed-step
// voxel march.  Everything here is FP32 (FP64 is used only for tallies).
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

#include "mc_internal.h"

namespace mcx {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 32x32->64 products of the counter words with fixed multipliers, the high
// halves xor-ed with the other counter words and the round key; the key is
// bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// One history's stream: key = seed, counter = (block, angle, h_lo, h_hi);
// the four words of each block are consumed in order.
struct Rng {
  uint2 key;
  uint4 ctr;
  uint4 buf;
  int idx;
  __device__ __forceinline__ void init(unsigned long long h, uint32_t angle, unsigned long long seed) {
    key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    ctr = make_uint4(0u, angle, (uint32_t)h, (uint32_t)(h >> 32));
    idx = 4;
  }
  __device__ __forceinline__ void refill() {
    buf = philox4x32_10(ctr, key);
    ctr.x += 1u;
    idx = 0;
  }
  __device__ __forceinline__ uint32_t next() {
    if (idx == 4) refill();
    const uint32_t v = idx == 0 ? buf.x : idx == 1 ? buf.y : idx == 2 ? buf.z : buf.w;
    ++idx;
    return v;
  }
  // Start of the next block of four.
  __device__ __forceinline__ void align() { idx = 4; }
  // Uniform on (0,1): ((x >> 9) + 1/2) 2^-23, exactly representable.
  __device__ __forceinline__ float u() { return u01(next()); }
  static __device__ __forceinline__ float u01(uint32_t x) {
    return __fmul_rn((float)(x >> 9) + 0.5f, 1.1920928955078125e-07f);
  }
};

// ---------------------------------------------------------------------------
// Tables in shared memory: float2 (v_i, v_{i+1} - v_i) per node; linear in E.
struct SmemTables {
  const float2* tab;   // [kTabKinds][n_mat][n_stage]
  const float2* jkn;   // [n_stage]
  const float2* eta;   // [n_stage] detector response (used when use_eta)
  const float2* comp;  // [n_mat][kMaxComp] (w Z^2, b)
  const float* compz;  // [n_mat][kMaxComp] w Z
  const int* ncomp;    // [n_mat]
  int n_mat, n_stage, use_eta, bound;
  float E0, inv_dE, mec2, inv_hc;

  __device__ __forceinline__ void locate(float E, int& i, float& f) const {
    const float x = (E - E0) * inv_dE;
    int k = __float2int_rd(x);
    k = max(0, min(k, n_stage - 2));
    i = k;
    f = x - (float)k;
  }
  __device__ __forceinline__ float at(int kind, int m, int i, float f) const {
    const float2 v = tab[(kind * n_mat + m) * n_stage + i];
    return fmaf(f, v.y, v.x);
  }
  __device__ __forceinline__ float kn_norm(int i, float f) const {
    const float2 v = jkn[i];
    return fmaf(f, v.y, v.x);
  }
  // Molecular incoherent scattering function at x^2 = u (moles of electrons
  // per gram): sum_i w_i Z_i (1 - (1 + b_i u)^-4), written as
  // b u (2 + b u) (q^2 + 1) / q^4 (q = 1 + b u) to avoid cancellation near u = 0.
  __device__ __forceinline__ float smol(int m, float u) const {
    float s = 0.f;
    const int nc = ncomp[m];
    for (int i = 0; i < nc; ++i) {
      const float bu = comp[m * kMaxComp + i].y * u;
      const float q = 1.f + bu;
      const float q2 = q * q;
      s += compz[m * kMaxComp + i] * (bu * (2.f + bu) * (q2 + 1.f)) / (q2 * q2);
    }
    return s;
  }
  __device__ __forceinline__ float smol_max(int m) const {
    float s = 0.f;
    const int nc = ncomp[m];
    for (int i = 0; i < nc; ++i) s += compz[m * kMaxComp + i];
    return s;
  }
  // Detector response eta(E) at the located energy (Sec. II-D.2); E itself
  // (energy integrating) unless a response table was set.
  __device__ __forceinline__ float response(int i, float f, float E) const {
    if (!use_eta) return E;
    const float2 v = eta[i];
    return fmaf(f, v.y, v.x);
  }
};

// Byte offsets of the blob sections (all multiples of 8; total padded to 16).
__host__ __device__ inline int tab_off_jkn(int n_mat, int n_stage) { return kTabKinds * n_mat * n_stage * 8; }
__host__ __device__ inline int tab_off_eta(int n_mat, int n_stage) { return tab_off_jkn(n_mat, n_stage) + n_stage * 8; }
__host__ __device__ inline int tab_off_comp(int n_mat, int n_stage) {
  return tab_off_eta(n_mat, n_stage) + n_stage * 8;
}
__host__ __device__ inline int tab_off_compz(int n_mat, int n_stage) {
  return tab_off_comp(n_mat, n_stage) + n_mat * kMaxComp * 8;
}
__host__ __device__ inline int tab_off_ncomp(int n_mat, int n_stage) {
  return tab_off_compz(n_mat, n_stage) + n_mat * kMaxComp * 4;
}
__host__ __device__ inline int tab_blob_bytes(int n_mat, int n_stage) {
  return (tab_off_ncomp(n_mat, n_stage) + n_mat * 4 + 15) & ~15;
}

// ---------------------------------------------------------------------------
// Geometry of one angle (source on the circle of radius SOD about z).
struct Pose {
  float3 s, c, eu, n;  // source, panel centre, panel u axis, panel normal (toward source); e_v = z
};
__device__ __forceinline__ Pose make_pose(const GeomView& g, float beta) {
  float sb, cb;
  sincosf(beta, &sb, &cb);
  Pose p;
  p.s = make_float3(g.sod * cb, g.sod * sb, 0.f);
  const float r = g.sod - g.sdd;
  p.c = make_float3(r * cb, r * sb, 0.f);
  p.eu = make_float3(-sb, cb, 0.f);
  p.n = make_float3(cb, sb, 0.f);
  return p;
}
// Panel point at continuous pixel coordinates (a, b); pixel (i, j) spans [i, i+1) x [j, j+1).
__device__ __forceinline__ float3 det_point(const GeomView& g, const Pose& p, float a, float b) {
  const float ou = (a - 0.5f * (float)g.nu) * g.pu;
  const float ov = (b - 0.5f * (float)g.nv) * g.pv;
  return make_float3(fmaf(ou, p.eu.x, p.c.x), fmaf(ou, p.eu.y, p.c.y), p.c.z + ov);
}

__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }

// Slab clip of x + t w, t in [t0, t1], against the centred box of half extents h.
__device__ __forceinline__ bool clip_box(const VolumeView& v, float3 x, float3 w, float t0, float t1, float& ta,
                                         float& tb) {
  float a = t0, b = t1;
  const float px[3] = {x.x, x.y, x.z}, wx[3] = {w.x, w.y, w.z}, hx[3] = {v.hx, v.hy, v.hz};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (wx[k] == 0.f) {
      if (px[k] < -hx[k] || px[k] > hx[k]) return false;
    } else {
      float u = (-hx[k] - px[k]) / wx[k], q = (hx[k] - px[k]) / wx[k];
      if (u > q) {
        const float t = u;
        u = q;
        q = t;
      }
      a = fmaxf(a, u);
      b = fminf(b, q);
    }
  }
  ta = a;
  tb = b;
  return b > a;
}

// Word index of padded voxel (ix, iy, iz) in the packed volume.
template <int LAYOUT>
__device__ __host__ __forceinline__ int vox_index(const VolumeView& vol, int ix, int iy, int iz) {
  if (LAYOUT == VOX_LIN) return (iz * vol.py + iy) * vol.px + ix;
  const int brick = ((iz >> 2) * vol.nby + (iy >> 2)) * vol.nbx + (ix >> 2);
  const int lx = ix & 3, ly = iy & 3, lz = iz & 3;
  const int m = (lx & 1) | ((ly & 1) << 1) | ((lz & 1) << 2) | ((lx & 2) << 2) | ((ly & 2) << 3) | ((lz & 2) << 4);
  return (brick << 6) | m;
}

// floor(y) for 0 <= y < 2^22 by one round-down add: 2^23 + y rounded toward
// minus infinity is 2^23 + floor(y), whose bit pattern minus that of 2^23 is
// the integer (full-rate FP add instead of a conversion).
__device__ __forceinline__ int floor_pos(float y) {
  return __float_as_int(__fadd_rd(y, 8388608.0f)) - 0x4B000000;
}

// Ray in padded voxel units: v(t) = v0 + t vw, voxel = floor(v).
struct VoxRay {
  float3 v0, vw;
  __device__ __forceinline__ void set(const VolumeView& vol, float3 x, float3 w) {
    v0 = make_float3(fmaf(x.x, vol.inv_dx, 0.5f * (float)vol.nx + 1.f),
                     fmaf(x.y, vol.inv_dy, 0.5f * (float)vol.ny + 1.f),
                     fmaf(x.z, vol.inv_dz, 0.5f * (float)vol.nz + 1.f));
    vw = make_float3(w.x * vol.inv_dx, w.y * vol.inv_dy, w.z * vol.inv_dz);
  }
  // Word index of the voxel holding the point at parameter t (a point inside
  // the clipped chord; the border absorbs rounding, the final clamp only
  // guards the array bounds).
  template <int LAYOUT>
  __device__ __forceinline__ int voxel(const VolumeView& vol, float t) const {
    return voxel_p<LAYOUT>(vol, fmaf(t, vw.x, v0.x), fmaf(t, vw.y, v0.y), fmaf(t, vw.z, v0.z));
  }
  // The same for a point given in padded voxel units.
  template <int LAYOUT>
  __device__ __forceinline__ int voxel_p(const VolumeView& vol, float px, float py, float pz) const {
    if (LAYOUT == VOX_LIN) {
      // (bx - C) + px (by - C) + px py (bz - C) with b the bit patterns of the
      // round-down adds (C = 0x4B000000, see floor_pos): the offsets fold into
      // one precomputed bias (exact in 32-bit wraparound arithmetic); the
      // unsigned min only guards the array bounds
      const unsigned bx = __float_as_uint(__fadd_rd(px, 8388608.0f));
      const unsigned by = __float_as_uint(__fadd_rd(py, 8388608.0f));
      const unsigned bz = __float_as_uint(__fadd_rd(pz, 8388608.0f));
      const unsigned idx = bx + (unsigned)vol.px * by + (unsigned)vol.pxy * bz - (unsigned)vol.lin_bias;
      return (int)min(idx, (unsigned)(vol.words - 1));
    }
    const int ix = floor_pos(px);
    const int iy = floor_pos(py);
    const int iz = floor_pos(pz);
    return min(max(vox_index<LAYOUT>(vol, ix, iy, iz), 0), vol.words - 1);
  }
};

__device__ __forceinline__ int vox_mat(uint32_t w) { return (int)((w >> 16) & 255u); }
__device__ __forceinline__ float vox_rho(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu))); }

__device__ __forceinline__ int step_count(float L, float step) { return max(1, (int)ceilf(L / step)); }

}  // namespace mcx
