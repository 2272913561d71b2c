// Triangle-mesh (CAD) geometry, host side and primary images: the paper's
// original surface model (Sec. II-A, "CAD surface model using triangular
// elements"; Sec. III, "closed triangulated surfaces").  The device ray
// casting (hierarchy descent, watertight triangle test, signed chord sums,
// exact free flights) is in mc_mesh.cuh, shared with the transport kernel.
//
// Host: a bounding-volume hierarchy over the triangles (binned surface-area
// heuristic, median splits near the depth limit; build_mesh_bvh below),
// children stored next to each other.  Device: one thread per pixel casts the
// source ray; the primary image then follows eq. (Ip) with exact per-material
// column masses.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "mc_mesh.cuh"

namespace mcx {
namespace {

constexpr int kLeaf = 4;
constexpr float kPi = 3.14159265358979f;

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
  mesh::mesh_rhoL(M, ps.s, w, d, rl, true);
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
//
// Splits follow the surface-area heuristic over 16 centroid bins per axis (the
// expected cost of a ray that meets the node: one box test plus, per child,
// its triangles times the probability area(child)/area(node) of meeting it);
// a node of up to kMaxLeaf triangles stays a leaf when splitting does not pay.
// Long thin triangles (a finely tessellated cylinder's sides) thus go to
// children split across them rather than along them.  Near the depth limit,
// or when the binned split puts every triangle on one side, the node splits
// at the median centroid of its longest axis instead, which bounds the depth
// by about log2(triangles) + 2 and keeps the device stack within mesh::kStack.
// Returns the depth of the deepest leaf (root = 1).
int build_mesh_bvh(const float* v, const int* tris, const int* tri_body, int nt, std::vector<float4>& nodes,
                   std::vector<float4>& out_tris) {
  constexpr int kBins = 16, kMaxLeaf = 8;
  std::vector<int> idx(nt);
  std::vector<Box> tb(nt);
  std::vector<float> cen((size_t)nt * 3);
  for (int k = 0; k < nt; ++k) {
    idx[k] = k;
    for (int a = 0; a < 3; ++a) {
      const float x0 = v[3 * tris[3 * k] + a], x1 = v[3 * tris[3 * k + 1] + a], x2 = v[3 * tris[3 * k + 2] + a];
      tb[k].lo[a] = std::min(x0, std::min(x1, x2));
      tb[k].hi[a] = std::max(x0, std::max(x1, x2));
      cen[3 * k + a] = (x0 + x1 + x2) / 3.f;
    }
  }
  auto empty = [] {
    Box b;
    for (int a = 0; a < 3; ++a) {
      b.lo[a] = 3.4e38f;
      b.hi[a] = -3.4e38f;
    }
    return b;
  };
  auto grow = [](Box& b, const Box& o) {
    for (int a = 0; a < 3; ++a) {
      b.lo[a] = std::min(b.lo[a], o.lo[a]);
      b.hi[a] = std::max(b.hi[a], o.hi[a]);
    }
  };
  auto area = [](const Box& b) {
    const double dx = std::max(0.f, b.hi[0] - b.lo[0]), dy = std::max(0.f, b.hi[1] - b.lo[1]),
                 dz = std::max(0.f, b.hi[2] - b.lo[2]);
    return dx * dy + dy * dz + dz * dx;
  };
  auto ceil_log2 = [](int n) {
    int d = 0;
    while ((1ll << d) < (long long)n) ++d;
    return d;
  };
  struct Item {
    int node, lo, hi, depth;
  };
  nodes.assign(2, make_float4(0.f, 0.f, 0.f, 0.f));
  std::vector<Item> work{{0, 0, nt, 1}};
  int max_depth = 0;
  while (!work.empty()) {
    const Item it = work.back();
    work.pop_back();
    const int n = it.hi - it.lo;
    Box b = empty(), cb = empty();
    for (int q = it.lo; q < it.hi; ++q) {
      grow(b, tb[idx[q]]);
      for (int a = 0; a < 3; ++a) {
        cb.lo[a] = std::min(cb.lo[a], cen[3 * idx[q] + a]);
        cb.hi[a] = std::max(cb.hi[a], cen[3 * idx[q] + a]);
      }
    }
    auto make_leaf = [&] {
      nodes[2 * it.node] = make_float4(b.lo[0], b.lo[1], b.lo[2], bits_f(it.lo));
      nodes[2 * it.node + 1] = make_float4(b.hi[0], b.hi[1], b.hi[2], bits_f(n));
      max_depth = std::max(max_depth, it.depth);
    };
    if (n <= kLeaf) {
      make_leaf();
      continue;
    }
    // binned surface-area heuristic
    int best_axis = -1, best_bin = -1;
    double best_cost = 1e300;
    const bool sah_ok = it.depth + ceil_log2(n) + 2 <= mesh::kStack - 8;
    for (int a = 0; a < 3 && sah_ok; ++a) {
      const float ext = cb.hi[a] - cb.lo[a];
      if (!(ext > 0.f)) continue;
      Box bb[kBins];
      int cnt[kBins] = {};
      for (int i = 0; i < kBins; ++i) bb[i] = empty();
      const float sc = (float)kBins / ext;
      for (int q = it.lo; q < it.hi; ++q) {
        const int k = idx[q];
        const int i = std::min(kBins - 1, std::max(0, (int)((cen[3 * k + a] - cb.lo[a]) * sc)));
        ++cnt[i];
        grow(bb[i], tb[k]);
      }
      double right_area[kBins];
      int right_cnt[kBins];
      Box acc = empty();
      int c = 0;
      for (int i = kBins - 1; i > 0; --i) {
        grow(acc, bb[i]);
        c += cnt[i];
        right_area[i] = area(acc);
        right_cnt[i] = c;
      }
      acc = empty();
      c = 0;
      for (int i = 0; i < kBins - 1; ++i) {
        grow(acc, bb[i]);
        c += cnt[i];
        if (c == 0 || right_cnt[i + 1] == 0) continue;
        const double cost = c * area(acc) + right_cnt[i + 1] * right_area[i + 1];
        if (cost < best_cost) {
          best_cost = cost;
          best_axis = a;
          best_bin = i;
        }
      }
    }
    const double pa = area(b);
    int mid = -1;
    if (best_axis >= 0) {
      // split cost (one box test ~ one triangle test) against the leaf's n triangle tests
      if (n <= kMaxLeaf && pa > 0.0 && pa + best_cost >= n * pa) {
        make_leaf();
        continue;
      }
      const int a = best_axis;
      const float sc = (float)kBins / (cb.hi[a] - cb.lo[a]);
      const auto m = std::partition(idx.begin() + it.lo, idx.begin() + it.hi, [&](int k) {
        return std::min(kBins - 1, std::max(0, (int)((cen[3 * k + a] - cb.lo[a]) * sc))) <= best_bin;
      });
      mid = (int)(m - idx.begin());
    }
    if (mid <= it.lo || mid >= it.hi) {
      int axis = 0;
      for (int a = 1; a < 3; ++a)
        if (b.hi[a] - b.lo[a] > b.hi[axis] - b.lo[axis]) axis = a;
      mid = it.lo + n / 2;
      std::nth_element(idx.begin() + it.lo, idx.begin() + mid, idx.begin() + it.hi,
                       [&](int p, int q) { return cen[3 * p + axis] < cen[3 * q + axis]; });
    }
    const int left = (int)(nodes.size() / 2);
    nodes.resize(nodes.size() + 4, make_float4(0.f, 0.f, 0.f, 0.f));
    nodes[2 * it.node] = make_float4(b.lo[0], b.lo[1], b.lo[2], bits_f(left));
    nodes[2 * it.node + 1] = make_float4(b.hi[0], b.hi[1], b.hi[2], bits_f(0));
    work.push_back({left, it.lo, mid, it.depth + 1});
    work.push_back({left + 1, mid, it.hi, it.depth + 1});
  }
  out_tris.resize((size_t)nt * 3);
  for (int q = 0; q < nt; ++q) {
    const int k = idx[q];
    for (int c = 0; c < 3; ++c) {
      const float* p = v + 3 * tris[3 * k + c];
      out_tris[3 * q + c] = make_float4(p[0], p[1], p[2], c == 0 ? bits_f(tri_body[k]) : 0.f);
    }
  }
  return max_depth;
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
