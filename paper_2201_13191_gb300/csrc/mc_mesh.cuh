// Device geometry of the triangle-mesh (CAD) bodies: the paper's original
// surface model (Sec. II-A, "CAD surface model using triangular elements";
// Sec. III, "closed triangulated surfaces").  Bodies are closed, outward-
// oriented triangle surfaces with a material, a density and optionally a
// parent body whose material they replace; outside every body is vacuum.
//
// Rays descend a bounding-volume hierarchy (explicit stack) and test leaf
// triangles with the watertight shear-and-edge-function test; an edge function
// exactly zero counts as inside for only one of the two triangles sharing that
// edge (half-open rule on the edge's projected direction, normalised by the
// facing), so every surface crossing counts once.
//
//   mesh_rhoL    per-material column masses along a segment: each crossing of
//                body b adds +-t to b's inside length (+ leaving, - entering),
//                which sums to the length inside b because crossings of a
//                closed surface alternate (also when the segment starts inside);
//   mesh_flight  exact free flight: the crossings of the half-line ahead, in
//                order, with the medium between them (below).
#pragma once
#include <stdint.h>

#include "mc_device.cuh"

namespace mcx {
namespace mesh {

constexpr int kStack = 64;  // the host builder keeps the depth (stack entries - 1) below 63
constexpr int kWin = 8;     // crossings held per window of the free flight

struct Shear {
  int kx, ky, kz;
  float Sx, Sy, Sz;
};

__device__ __forceinline__ float comp(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

__device__ __forceinline__ Shear shear_of(float3 d) {
  Shear h;
  int kz = 0;
  if (fabsf(d.y) > fabsf(comp(d, kz))) kz = 1;
  if (fabsf(d.z) > fabsf(comp(d, kz))) kz = 2;
  int kx = kz == 2 ? 0 : kz + 1, ky = kx == 2 ? 0 : kx + 1;
  if (comp(d, kz) < 0.f) {
    const int t = kx;
    kx = ky;
    ky = t;
  }
  h.kx = kx;
  h.ky = ky;
  h.kz = kz;
  h.Sx = comp(d, kx) / comp(d, kz);
  h.Sy = comp(d, ky) / comp(d, kz);
  h.Sz = 1.f / comp(d, kz);
  return h;
}

__device__ __forceinline__ bool edge_incl(float ex, float ey) { return ey > 0.f || (ey == 0.f && ex < 0.f); }

// Watertight test; true and *t (ray parameter from org) on a hit.
__device__ __forceinline__ bool ray_tri(float3 org, const Shear& h, float3 v0, float3 v1, float3 v2, float& t) {
  const float3 A = sub3(v0, org), B = sub3(v1, org), C = sub3(v2, org);
  const float Az = comp(A, h.kz), Bz = comp(B, h.kz), Cz = comp(C, h.kz);
  const float Ax = comp(A, h.kx) - h.Sx * Az, Ay = comp(A, h.ky) - h.Sy * Az;
  const float Bx = comp(B, h.kx) - h.Sx * Bz, By = comp(B, h.ky) - h.Sy * Bz;
  const float Cx = comp(C, h.kx) - h.Sx * Cz, Cy = comp(C, h.ky) - h.Sy * Cz;
  const float U = Cx * By - Cy * Bx, V = Ax * Cy - Ay * Cx, W = Bx * Ay - By * Ax;
  const float det = U + V + W;
  if (det == 0.f) return false;
  const float sg = det > 0.f ? 1.f : -1.f;
  if (!(sg * U > 0.f || (U == 0.f && edge_incl(sg * (Cx - Bx), sg * (Cy - By))))) return false;
  if (!(sg * V > 0.f || (V == 0.f && edge_incl(sg * (Ax - Cx), sg * (Ay - Cy))))) return false;
  if (!(sg * W > 0.f || (W == 0.f && edge_incl(sg * (Bx - Ax), sg * (By - Ay))))) return false;
  t = h.Sz * (U * Az + V * Bz + W * Cz) / det;
  return true;
}

// Slab test of the ray against a box over (t_lo, t_hi).
__device__ __forceinline__ bool hit_box(float3 org, float3 inv, float4 lo, float4 hi, float t_lo, float t_hi) {
  float ta = (lo.x - org.x) * inv.x, tb = (hi.x - org.x) * inv.x;
  float t0 = fminf(ta, tb), t1 = fmaxf(ta, tb);
  ta = (lo.y - org.y) * inv.y;
  tb = (hi.y - org.y) * inv.y;
  t0 = fmaxf(t0, fminf(ta, tb));
  t1 = fminf(t1, fmaxf(ta, tb));
  ta = (lo.z - org.z) * inv.z;
  tb = (hi.z - org.z) * inv.z;
  t0 = fmaxf(t0, fminf(ta, tb));
  t1 = fminf(t1, fmaxf(ta, tb));
  // padded by a relative epsilon so that a hit exactly on a face of the box is not lost
  const float pad = 1e-5f * fmaxf(fabsf(t0), fabsf(t1)) + 1e-6f;
  return t0 - pad <= fminf(t1, t_hi) + pad && t1 + pad >= t_lo;
}

// Calls f(k, t, v0, v1, v2) for every leaf triangle k the ray org + t w crosses
// with t_lo < t < t_hi.  An inner node tests both children's boxes and
// descends into a hit child directly, stacking the other only when both are
// hit, so the (local-memory) stack sees one entry per two-way branch.  The
// descent to the next leaf and the leaf's triangle tests are separate loops
// ("while-while"), so the lanes of a warp that reach leaves at different
// depths test their triangles together.
template <class F>
__device__ __forceinline__ void visit(const MeshView& M, float3 org, float3 w, float t_lo, float t_hi, F&& f) {
  const Shear h = shear_of(w);
  const float3 inv = make_float3(1.f / w.x, 1.f / w.y, 1.f / w.z);
  int stack[kStack];
  int sp = 0;
  int ni = 0;
  {
    const float4 lo = __ldg(M.nodes), hi = __ldg(M.nodes + 1);
    if (!hit_box(org, inv, lo, hi, t_lo, t_hi)) return;
  }
  for (;;) {
    // descend until ni is a leaf (or nothing is left)
    int first, count;
    bool done = false;
    for (;;) {
      const float4 lo = __ldg(M.nodes + 2 * ni), hi = __ldg(M.nodes + 2 * ni + 1);
      first = __float_as_int(lo.w);
      count = __float_as_int(hi.w);
      if (count != 0) break;
      const float4 al = __ldg(M.nodes + 2 * first), ah = __ldg(M.nodes + 2 * first + 1);
      const float4 bl = __ldg(M.nodes + 2 * first + 2), bh = __ldg(M.nodes + 2 * first + 3);
      const bool ha = hit_box(org, inv, al, ah, t_lo, t_hi), hb = hit_box(org, inv, bl, bh, t_lo, t_hi);
      if (ha || hb) {
        // the host builder bounds the depth by kStack - 1, so the stack cannot overflow
        if (ha && hb) stack[sp++] = first + 1;
        ni = ha ? first : first + 1;
      } else if (sp > 0) {
        ni = stack[--sp];
      } else {
        done = true;
        break;
      }
    }
    if (done) break;
    for (int k = first; k < first + count; ++k) {
      const float4 a = __ldg(M.tris + 3 * k), b = __ldg(M.tris + 3 * k + 1), c = __ldg(M.tris + 3 * k + 2);
      const float3 v0 = make_float3(a.x, a.y, a.z), v1 = make_float3(b.x, b.y, b.z), v2 = make_float3(c.x, c.y, c.z);
      float t;
      if (!ray_tri(org, h, v0, v1, v2, t)) continue;
      if (!(t > t_lo && t < t_hi)) continue;
      f(k, t, v0, v1, v2);
    }
    if (sp == 0) break;
    ni = stack[--sp];
  }
}

__device__ __forceinline__ bool leaving(float3 v0, float3 v1, float3 v2, float3 w) {
  const float3 e1 = sub3(v1, v0), e2 = sub3(v2, v0);
  const float3 n = make_float3(e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x);
  return dot3(n, w) > 0.f;
}

// Per-material column masses rho L (g/cm^3 x mm) along x + t w, t in (0, t1);
// returns the number of surface crossings.  With `shift` the ray is tested
// from the point closest to the world origin (small parameters for a start
// far away, e.g. the source); the signed sum then assumes x outside every
// body.  Without it the ray is tested from x, which may lie inside bodies.
__device__ __forceinline__ int mesh_rhoL(const MeshView& M, float3 x, float3 w, float t1, float* rl, bool shift) {
  const float t0 = shift ? -dot3(x, w) : 0.f;
  const float3 org = shift ? make_float3(fmaf(t0, w.x, x.x), fmaf(t0, w.y, x.y), fmaf(t0, w.z, x.z)) : x;
  int n = 0;
  visit(M, org, w, -t0, t1 - t0, [&](int k, float t, float3 v0, float3 v1, float3 v2) {
    const float st = leaving(v0, v1, v2, w) ? t : -t;
    const int body = __float_as_int(__ldg(M.tris + 3 * k).w);
    const int4 bd = __ldg(M.bodies + body);  // material, parent, parent material, density bits
    rl[bd.x] += __int_as_float(bd.w) * st;
    if (bd.y >= 0) rl[bd.z] -= __ldg(M.body_rho + bd.y) * st;
    ++n;
  });
  return n;
}

// Order-preserving map of a float's bits to an unsigned key.
__device__ __forceinline__ uint32_t fkey(float t) {
  const uint32_t b = __float_as_uint(t);
  return b ^ ((b >> 31) ? 0xFFFFFFFFu : 0x80000000u);
}
__device__ __forceinline__ float funkey(uint32_t k) {
  return __uint_as_float(k ^ ((k >> 31) ? 0x80000000u : 0xFFFFFFFFu));
}

// One window of the free flight: the kWin smallest crossings (key = t bits,
// triangle) greater than `after` among those with t > t_lo, ascending in win[]
// (unused slots ~0), and in *parity the xor of (1 << body) over every crossing
// with t > t_lo: the bodies containing the ray point at t_lo.  Returns the
// number of crossings in the window.  One out-of-line copy serves every call,
// so a crossing computed again in a later window has the same bits.
static __device__ __noinline__ int mesh_window(const MeshView& M, float3 org, float3 w, float t_lo, unsigned long long after,
                                        unsigned long long* win_out, unsigned long long* parity) {
  unsigned long long win[kWin];
#pragma unroll
  for (int i = 0; i < kWin; ++i) win[i] = ~0ull;
  unsigned long long par = 0ull;
  visit(M, org, w, t_lo, __int_as_float(0x7f800000), [&](int k, float t, float3, float3, float3) {
    const int body = __float_as_int(__ldg(M.tris + 3 * k).w);
    par ^= 1ull << body;
    unsigned long long key = ((unsigned long long)fkey(t) << 32) | (uint32_t)k;
    if (key > after && key < win[kWin - 1]) {
#pragma unroll
      for (int i = 0; i < kWin; ++i) {
        if (key < win[i]) {
          const unsigned long long tmp = win[i];
          win[i] = key;
          key = tmp;
        }
      }
    }
  });
  int n = 0;
#pragma unroll
  for (int i = 0; i < kWin; ++i) {
    win_out[i] = win[i];
    n += win[i] != ~0ull;
  }
  *parity = par;
  return n;
}

// Exact free flight from x along w (the CAD model's ray tracing).  Body b
// contains x when the half-line ahead crosses its closed surface an odd number
// of times, so the start medium follows from the crossings themselves; each
// crossing toggles its body, and the medium is the deepest body containing the
// point (parents precede children, so the highest index).  Inside body b the
// optical depth grows by rho_b * smu[m_b] per mm (smu: 0.1 mu/rho per
// material, stride apart).  Returns true with the distance *tint and material
// *mint where the depth reaches tau_star; false after the last crossing
// (escape).  *nseg += segments walked (crossings passed, plus the last one).
__device__ __forceinline__ bool mesh_flight(const MeshView& M, float3 x, float3 w, float tau_star, const float* smu,
                                            int stride, float& tint, int& mint, unsigned long long& nseg) {
  const float t0 = -dot3(x, w);
  const float3 org = make_float3(fmaf(t0, w.x, x.x), fmaf(t0, w.y, x.y), fmaf(t0, w.z, x.z));
  const float t_lo = -t0;  // x's parameter on the shifted ray
  unsigned long long win[kWin], inside = 0ull, after = 0ull;
  float tprev = t_lo, tau = 0.f;
  bool first = true;
  for (;;) {
    unsigned long long par;
    const int n = mesh_window(M, org, w, t_lo, after, win, &par);
    if (first) inside = par;
    first = false;
    for (int i = 0; i < n; ++i) {
      const float tc = funkey((uint32_t)(win[i] >> 32));
      const int k = (int)(uint32_t)win[i];
      ++nseg;
      if (inside) {
        const int b = 63 - __clzll((long long)inside);
        const int4 bd = __ldg(M.bodies + b);
        const float mu = __int_as_float(bd.w) * smu[bd.x * stride];
        const float len = tc - tprev;
        if (mu > 0.f && fmaf(mu, len, tau) >= tau_star) {
          tint = (tprev - t_lo) + (tau_star - tau) / mu;
          mint = bd.x;
          return true;
        }
        tau = fmaf(mu, len, tau);
      }
      tprev = tc;
      inside ^= 1ull << __float_as_int(__ldg(M.tris + 3 * k).w);
    }
    if (n < kWin) break;
    after = win[kWin - 1];
  }
  ++nseg;
  return false;
}

}  // namespace mesh
}  // namespace mcx
