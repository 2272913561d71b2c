// Triangle-mesh (CAD) geometry: the paper's original surface model (Sec. II-A,
// "CAD surface model using triangular elements"; Sec. III, "closed triangulated
// surfaces").  Bodies are closed, outward-oriented triangle surfaces with a
// material, a density and optionally a parent body whose material they replace;
// outside every body is vacuum.
//
// Host: a bounding-volume hierarchy over the triangles (median split of the
// centroids along the longest axis, leaves of up to kLeaf triangles), children
// stored next to each other.  Device: one thread per pixel casts the source ray
// through the hierarchy (explicit stack) and tests leaf triangles with the
// watertight shear-and-edge-function test; an edge function exactly zero counts
// as inside for only one of the two triangles sharing that edge (half-open rule
// on the edge's projected direction, normalised by the facing), so every
// surface crossing counts once.  A body's inside length is the signed sum of its
// crossing parameters (+ leaving, - entering), taken about the ray point
// closest to the origin; the primary image then follows eq. (Ip) with exact
// per-material column masses.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "mc_device.cuh"

namespace mcx {
namespace {

constexpr int kLeaf = 4;
constexpr int kStack = 64;
constexpr float kPi = 3.14159265358979f;

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

// Per-material column masses rho L (g/cm^3 x mm) along x + t w, t in (0, t1).
__device__ __forceinline__ void mesh_rhoL(const MeshView& M, float3 x, float3 w, float t1, float* rl) {
  const float t0 = -dot3(x, w);
  const float3 org = make_float3(fmaf(t0, w.x, x.x), fmaf(t0, w.y, x.y), fmaf(t0, w.z, x.z));
  const float lo_t = -t0, hi_t = t1 - t0;
  const Shear h = shear_of(w);
  const float3 inv = make_float3(1.f / w.x, 1.f / w.y, 1.f / w.z);
  int stack[kStack];
  int sp = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    const int ni = stack[--sp];
    const float4 lo = __ldg(M.nodes + 2 * ni), hi = __ldg(M.nodes + 2 * ni + 1);
    if (!hit_box(org, inv, lo, hi, lo_t, hi_t)) continue;
    const int first = __float_as_int(lo.w), count = __float_as_int(hi.w);
    if (count == 0) {
      if (sp + 2 <= kStack) {
        stack[sp++] = first;
        stack[sp++] = first + 1;
      }
      continue;
    }
    for (int k = first; k < first + count; ++k) {
      const float4 a = __ldg(M.tris + 3 * k), b = __ldg(M.tris + 3 * k + 1), c = __ldg(M.tris + 3 * k + 2);
      const float3 v0 = make_float3(a.x, a.y, a.z), v1 = make_float3(b.x, b.y, b.z), v2 = make_float3(c.x, c.y, c.z);
      float t;
      if (!ray_tri(org, h, v0, v1, v2, t)) continue;
      if (!(t > lo_t && t < hi_t)) continue;
      const float3 e1 = sub3(v1, v0), e2 = sub3(v2, v0);
      const float3 n = make_float3(e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x);
      const float st = dot3(n, w) > 0.f ? t : -t;
      const int body = __float_as_int(a.w);
      const int4 bd = __ldg(M.bodies + body);  // material, parent, parent material, density bits
      rl[bd.x] += __int_as_float(bd.w) * st;
      if (bd.y >= 0) rl[bd.z] -= __ldg(M.body_rho + bd.y) * st;
    }
  }
}

__global__ void __launch_bounds__(256) k_primary_mesh(const PrimaryParams P, const MeshView M) {
  extern __shared__ float s_mub[];  // [n_bins][n_mat]: 0.1 * mu/rho at each bin energy
  const int nm = P.tab.n_mat, nb = P.spec.n_bins, ns = P.tab.n_stage;
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
  const int npix = G.nu * G.nv;
  const int a = blockIdx.y;
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  const int i = pix % G.nu, j = pix / G.nu;
  const Pose ps = make_pose(G, __ldg(P.angles + a));
  const float3 X = det_point(G, ps, (float)i + 0.5f, (float)j + 0.5f);
  const float3 D = sub3(X, ps.s);
  const float d = sqrtf(dot3(D, D));
  const float3 w = make_float3(D.x / d, D.y / d, D.z / d);
  float rl[kMaxMat];
#pragma unroll
  for (int m = 0; m < kMaxMat; ++m) rl[m] = 0.f;
  mesh_rhoL(M, ps.s, w, d, rl);
  float sum = 0.f;
  for (int n = 0; n < nb; ++n) {
    const float S = __ldg(P.spec.sn + n);
    if (S == 0.f) continue;
    float tau = 0.f;
    for (int m = 0; m < nm; ++m) tau = fmaf(s_mub[n * nm + m], rl[m], tau);
    sum = fmaf(S * __ldg(P.spec.eta + n), expf(-tau), sum);
  }
  const float cosg = G.sdd / d;
  P.out[(size_t)a * npix + pix] = sum * (G.pu * G.pv) * cosg / (4.f * kPi * d * d);
}

struct Box {
  float lo[3], hi[3];
};

// Bit pattern of an int as a float (host side of the node/triangle packing).
float bits_f(int i) {
  float f;
  std::memcpy(&f, &i, 4);
  return f;
}

}  // namespace

// Bounding-volume hierarchy over the triangles: nodes as pairs of float4 (lo.xyz
// + first, hi.xyz + count; count 0 marks an inner node whose children are
// first and first + 1), triangles reordered into leaf order as three float4
// each (vertex xyz, the first also carrying the body id).
void build_mesh_bvh(const float* v, const int* tris, const int* tri_body, int nt, std::vector<float4>& nodes,
                    std::vector<float4>& out_tris) {
  std::vector<int> idx(nt);
  std::vector<float> cen((size_t)nt * 3);
  for (int k = 0; k < nt; ++k) {
    idx[k] = k;
    for (int a = 0; a < 3; ++a)
      cen[3 * k + a] = (v[3 * tris[3 * k] + a] + v[3 * tris[3 * k + 1] + a] + v[3 * tris[3 * k + 2] + a]) / 3.f;
  }
  struct Item {
    int node, lo, hi;
  };
  nodes.assign(2, make_float4(0.f, 0.f, 0.f, 0.f));
  std::vector<Item> work{{0, 0, nt}};
  auto bounds = [&](int lo, int hi) {
    Box b;
    for (int a = 0; a < 3; ++a) {
      b.lo[a] = 3.4e38f;
      b.hi[a] = -3.4e38f;
    }
    for (int q = lo; q < hi; ++q)
      for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a) {
          const float x = v[3 * tris[3 * idx[q] + c] + a];
          b.lo[a] = std::min(b.lo[a], x);
          b.hi[a] = std::max(b.hi[a], x);
        }
    return b;
  };
  while (!work.empty()) {
    const Item it = work.back();
    work.pop_back();
    const Box b = bounds(it.lo, it.hi);
    const int n = it.hi - it.lo;
    if (n <= kLeaf) {
      int first_i = it.lo, count_i = n;
      nodes[2 * it.node] = make_float4(b.lo[0], b.lo[1], b.lo[2], bits_f(first_i));
      nodes[2 * it.node + 1] = make_float4(b.hi[0], b.hi[1], b.hi[2], bits_f(count_i));
      continue;
    }
    int axis = 0;
    for (int a = 1; a < 3; ++a)
      if (b.hi[a] - b.lo[a] > b.hi[axis] - b.lo[axis]) axis = a;
    const int mid = it.lo + n / 2;
    std::nth_element(idx.begin() + it.lo, idx.begin() + mid, idx.begin() + it.hi,
                     [&](int p, int q) { return cen[3 * p + axis] < cen[3 * q + axis]; });
    const int left = (int)(nodes.size() / 2);
    nodes.resize(nodes.size() + 4, make_float4(0.f, 0.f, 0.f, 0.f));
    nodes[2 * it.node] = make_float4(b.lo[0], b.lo[1], b.lo[2], bits_f(left));
    nodes[2 * it.node + 1] = make_float4(b.hi[0], b.hi[1], b.hi[2], bits_f(0));
    work.push_back({left, it.lo, mid});
    work.push_back({left + 1, mid, it.hi});
  }
  out_tris.resize((size_t)nt * 3);
  for (int q = 0; q < nt; ++q) {
    const int k = idx[q];
    for (int c = 0; c < 3; ++c) {
      const float* p = v + 3 * tris[3 * k + c];
      out_tris[3 * q + c] = make_float4(p[0], p[1], p[2], c == 0 ? bits_f(tri_body[k]) : 0.f);
    }
  }
}

cudaError_t launch_primary_mesh(const PrimaryParams& p, const MeshView& m, cudaStream_t s) {
  const int block = 256;
  const int npix = p.geo.nu * p.geo.nv;
  dim3 grid((npix + block - 1) / block, p.n_angles);
  const int smem = p.spec.n_bins * p.tab.n_mat * 4;
  k_primary_mesh<<<grid, block, smem, s>>>(p, m);
  return cudaGetLastError();
}

}  // namespace mcx
