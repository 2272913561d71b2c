// C ABI of the GB300 Monte Carlo scatter forward projection (include/mc.h):
// context, argument validation, table/volume/spectrum staging, launches.
// Host code only marshals inputs and sequences kernels; every step of the
// method runs in the kernels of k_transport.cu, k_primary.cu, k_mesh.cu,
// k_post.cu and k_recon.cu (and the denoiser's in k_conv.cu / k_nn.cu).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mc_device.cuh"
#include "mc_internal.h"
#include "mc_nn.h"

using namespace mcx;

struct mc_ctx {
  int device = 0;
  int sm_count = 0;
  mc_options opt{};
  std::string err;
  // tables (host FP64 copies, file order)
  bool have_tables = false;
  int n_mat = 0, n_E = 0;
  double E0 = 0, dE = 1, r0 = 0, mec2 = 0, hc = 0;
  std::vector<double> pe, in, co, icoh;  // [n_mat][n_E]
  bool bound = false;                    // incoherent scattering function in use (table version 2)
  std::vector<double> iincoh;            // [n_mat][n_E] its normalisation
  int n_comp[kMaxMat] = {};
  double comp[kMaxMat][kMaxComp][3] = {};
  // detector response eta(E) at the table nodes (empty: eta(E) = E)
  std::vector<double> eta;
  // staged FP32 blob (device)
  float2* d_blob = nullptr;
  int blob_bytes = 0, blob_stage = 0;
  bool blob_dirty = true;
  // triangle-mesh geometry (replaces the volume while mesh_mode)
  bool have_mesh = false, mesh_mode = false;
  float4 *d_mesh_nodes = nullptr, *d_mesh_tris = nullptr;
  int4* d_mesh_bodies = nullptr;
  float* d_mesh_rho = nullptr;
  int mesh_nodes = 0, mesh_tris = 0, mesh_bodies = 0;
  double mesh_rmax = 0;  // largest distance of a vertex from the rotation axis
  double mat_change = 0;  // fraction of x-neighbour voxel pairs of different materials
  float mesh_half[3] = {0.f, 0.f, 0.f};  // half extents of a box about the origin holding every vertex
  // volume
  bool have_volume = false;
  uint32_t* d_vox = nullptr;  // packed voxel words (material | FP16 density)
  size_t vox_cap = 0;
  int layout = VOX_LIN;
  int nx = 0, ny = 0, nz = 0;
  float dx = 0, dy = 0, dz = 0;
  // spectrum
  bool have_spectrum = false;
  std::vector<double> S;
  std::vector<float> Ebin;
  void* d_spec = nullptr;  // prefix u64[n+1] | energy f32[n] | wbin f32[n] | sn f32[n] | eta f32[n]
  size_t d_spec_cap = 0;
  // geometry
  bool have_geometry = false;
  float sod = 0, sdd = 0, pu = 0, pv = 0;
  int nu = 0, nv = 0;
  // scratch
  double* d_tally = nullptr;
  size_t tally_cap = 0;
  unsigned long long* d_stats = nullptr;
  float* d_angles = nullptr;
  int angles_cap = 0;
  float* d_post = nullptr;  // post-processing scratch
  size_t post_cap = 0;
  double stats[MC_STAT_N] = {};
  cudaEvent_t ev[4] = {};
  // pinned host staging (spectrum block + seed, angles, counters) and the
  // cached CUDA graph of one projection
  unsigned char* h_pin = nullptr;
  size_t h_pin_cap = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<unsigned char> graph_key;
  int graph_builds = 0;
  Denoiser* denoiser = nullptr;  // learned denoiser (mc_denoise_*)
};

namespace {

int fail(mc_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(mc_ctx* c, cudaError_t e, const char* where) {
  const int code = (e == cudaErrorMemoryAllocation) ? MC_ERR_OOM : MC_ERR_CUDA;
  return fail(c, code, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                           \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

template <class T>
cudaError_t ensure(T*& p, size_t& cap, size_t n) {
  if (n <= cap && p) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc((void**)&p, n * sizeof(T));
  if (e == cudaSuccess) cap = n;
  return e;
}

int validate_options(const mc_options* o, std::string& why) {
  if (o->n_split < 1 || o->n_split > 4096) return why = "n_split must be in [1, 4096]", -1;
  if (!(o->rr_threshold >= 0.f)) return why = "rr_threshold must be >= 0", -1;
  if (o->max_scatter_order < 1) return why = "max_scatter_order must be >= 1", -1;
  if (o->n_batches < 1 || o->n_batches > 1024) return why = "n_batches must be in [1, 1024]", -1;
  if (o->block_size != 0 && (o->block_size < 32 || o->block_size > 256 || o->block_size % 32))
    return why = "block_size must be 0 or a multiple of 32 in [32, 256]", -1;
  if (o->blocks_per_sm < 0 || o->blocks_per_sm > 64) return why = "blocks_per_sm must be in [0, 64]", -1;
  if (o->tally_mode < 0 || o->tally_mode > 4) return why = "tally_mode must be 0 .. 4", -1;
  if (o->tile_u < 1 || o->tile_v < 1 || o->tile_u > 4096 || o->tile_v > 4096)
    return why = "tile_u and tile_v must be in 1 .. 4096", -1;
  if (o->sg_order < 0 || o->sg_window < o->sg_order + 2 || o->sg_window % 2 == 0 || o->sg_window > 31)
    return why = "sg_window must be odd, >= sg_order + 2 and <= 31", -1;
  if (!(o->cubic_a < 0.f && o->cubic_a > -3.f)) return why = "cubic_a must be in (-3, 0)", -1;
  if (o->denoise_mode < 0 || o->denoise_mode > 2) return why = "denoise_mode must be 0, 1 or 2", -1;
  if (o->voxel_layout < 0 || o->voxel_layout > 2) return why = "voxel_layout must be 0, 1 or 2", -1;
  if (o->use_graph < 0 || o->use_graph > 1) return why = "use_graph must be 0 or 1", -1;
  if (o->nee_mode < 0 || o->nee_mode > 1) return why = "nee_mode must be 0 or 1", -1;
  if (o->doppler < 0 || o->doppler > 1) return why = "doppler must be 0 or 1", -1;
  if (o->forced_detection < 0 || o->forced_detection > 1) return why = "forced_detection must be 0 or 1", -1;
  return 0;
}

// Klein-Nishina total per electron / (pi r0^2), closed form with its series
// where the closed form cancels.
double kn_norm(double E, double mec2) {
  const double k = E / mec2;
  if (k < 1e-3) return 8.0 / 3.0 * (1.0 - 2.0 * k + 5.2 * k * k - 13.3 * k * k * k);
  const double l = std::log1p(2.0 * k);
  const double a = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / (1.0 + 2.0 * k) - l / k);
  return 2.0 * (a + l / (2.0 * k) - (1.0 + 3.0 * k) / ((1.0 + 2.0 * k) * (1.0 + 2.0 * k)));
}

// Number of table nodes the spectrum can reach (staged into shared memory).
int stage_nodes(const mc_ctx* ctx) {
  double Emax = ctx->E0 + 1.0;
  for (size_t n = 0; n < ctx->S.size(); ++n) Emax = std::max(Emax, (double)ctx->Ebin[n]);
  const int ns = (int)std::floor((Emax - ctx->E0) / ctx->dE) + 2;
  return std::max(2, std::min(ns, ctx->n_E));
}

// The FP32 shared-memory blob for the first ns nodes: per kind and material
// (v_i, v_{i+1} - v_i), the Klein-Nishina normalisation, the detector response
// (eta(E_i) = E_i when none is set), the form-factor components.
void write_blob(const mc_ctx* ctx, int ns, unsigned char* dst) {
  const int nm = ctx->n_mat;
  std::memset(dst, 0, tab_blob_bytes(nm, ns));
  float2* tab = reinterpret_cast<float2*>(dst);
  for (int kind = 0; kind < kTabKinds; ++kind)
    for (int m = 0; m < nm; ++m)
      for (int i = 0; i < ns; ++i) {
        auto val = [&](int j) {
          const size_t q = (size_t)m * ctx->n_E + j;
          switch (kind) {
            case TAB_TOT: return ctx->pe[q] + ctx->in[q] + ctx->co[q];
            case TAB_PE: return ctx->pe[q];
            case TAB_IN: return ctx->in[q];
            case TAB_CO: return ctx->co[q];
            case TAB_ICOH: return ctx->icoh[q];
            default: return ctx->bound ? ctx->iincoh[q] : 0.0;
          }
        };
        const double v0 = val(i), v1 = val(std::min(i + 1, ctx->n_E - 1));
        tab[(kind * nm + m) * ns + i] = make_float2((float)v0, (float)(v1 - v0));
      }
  float2* jkn = reinterpret_cast<float2*>(dst + tab_off_jkn(nm, ns));
  float2* eta = reinterpret_cast<float2*>(dst + tab_off_eta(nm, ns));
  for (int i = 0; i < ns; ++i) {
    const double E = ctx->E0 + ctx->dE * i;
    const double j0 = kn_norm(E, ctx->mec2), j1 = kn_norm(E + ctx->dE, ctx->mec2);
    jkn[i] = make_float2((float)j0, (float)(j1 - j0));
    const int i1 = std::min(i + 1, ctx->n_E - 1);
    const double e0 = ctx->eta.empty() ? E : ctx->eta[i];
    const double e1 = ctx->eta.empty() ? ctx->E0 + ctx->dE * i1 : ctx->eta[i1];
    eta[i] = make_float2((float)e0, (float)(e1 - e0));
  }
  float2* comp = reinterpret_cast<float2*>(dst + tab_off_comp(nm, ns));
  float* compz = reinterpret_cast<float*>(dst + tab_off_compz(nm, ns));
  int* ncomp = reinterpret_cast<int*>(dst + tab_off_ncomp(nm, ns));
  for (int m = 0; m < nm; ++m) {
    ncomp[m] = ctx->n_comp[m];
    for (int i = 0; i < kMaxComp; ++i) {
      const double Z = ctx->comp[m][i][0], w = ctx->comp[m][i][1], b = ctx->comp[m][i][2];
      const bool on = i < ctx->n_comp[m];
      comp[m * kMaxComp + i] = on ? make_float2((float)(w * Z * Z), (float)b) : make_float2(0.f, 1.f);
      compz[m * kMaxComp + i] = on ? (float)(w * Z) : 0.f;
    }
  }
}

// Detector response at energy E (linear between the table nodes), or E.
double response_at(const mc_ctx* ctx, double E) {
  if (ctx->eta.empty()) return E;
  const double x = (E - ctx->E0) / ctx->dE;
  const int i = std::max(0, std::min((int)std::floor(x), ctx->n_E - 2));
  const double f = x - i;
  return ctx->eta[i] + f * (ctx->eta[i + 1] - ctx->eta[i]);
}

// Build and upload the FP32 shared-memory blob for the nodes the spectrum can reach.
int stage_tables(mc_ctx* ctx) {
  if (!ctx->blob_dirty && ctx->d_blob) return MC_OK;
  const int ns = stage_nodes(ctx);
  const int bytes = tab_blob_bytes(ctx->n_mat, ns);
  std::vector<unsigned char> blob(bytes, 0);
  write_blob(ctx, ns, blob.data());
  if (ctx->d_blob) cudaFree(ctx->d_blob);
  ctx->d_blob = nullptr;
  CK(cudaMalloc((void**)&ctx->d_blob, bytes), "table blob allocation");
  CK(cudaMemcpy(ctx->d_blob, blob.data(), bytes, cudaMemcpyHostToDevice), "table blob upload");
  ctx->blob_bytes = bytes;
  ctx->blob_stage = ns;
  ctx->blob_dirty = false;
  return MC_OK;
}

TableView table_view(const mc_ctx* c) {
  TableView t;
  t.blob = c->d_blob;
  t.n_mat = c->n_mat;
  t.n_stage = c->blob_stage;
  t.blob_bytes = c->blob_bytes;
  t.E0 = (float)c->E0;
  t.dE = (float)c->dE;
  t.inv_dE = (float)(1.0 / c->dE);
  t.mec2 = (float)c->mec2;
  t.inv_hc = (float)(1.0 / c->hc);
  t.use_eta = c->eta.empty() ? 0 : 1;
  t.bound = c->bound ? 1 : 0;
  return t;
}

VolumeView volume_view(const mc_ctx* c) {
  VolumeView v;
  padded_dims(c->nx, c->ny, c->nz, c->layout, &v);
  v.vox = c->d_vox;
  v.dx = c->dx; v.dy = c->dy; v.dz = c->dz;
  v.inv_dx = 1.f / c->dx; v.inv_dy = 1.f / c->dy; v.inv_dz = 1.f / c->dz;
  v.hx = 0.5f * c->nx * c->dx; v.hy = 0.5f * c->ny * c->dy; v.hz = 0.5f * c->nz * c->dz;
  return v;
}

GeomView geom_view(const mc_ctx* c) {
  GeomView g;
  g.sod = c->sod; g.sdd = c->sdd; g.pu = c->pu; g.pv = c->pv; g.nu = c->nu; g.nv = c->nv;
  return g;
}

// Stratified counts (largest remainder, at least one photon per non-empty bin)
// written into the host block that mirrors the device spectrum block:
//   seed u64 | prefix u64[n+1] | energy f32[n] | wbin f32[n] | sn f32[n]
size_t spectrum_block_bytes(int n) { return 8 + (size_t)(n + 1) * 8 + (size_t)n * 16; }

int fill_spectrum(mc_ctx* ctx, uint64_t N, uint64_t seed, unsigned char* host, bool histories = true) {
  const int n = (int)ctx->S.size();
  std::vector<uint64_t> M(n, 0);
  std::vector<int> elig(n, 0);
  std::vector<double> fr(n, 0.0);
  uint64_t sum = 0;
  // a primary-only call runs no histories: no photon counts, every count zero
  if (!histories) N = 0;
  for (int i = 0; i < n && histories; ++i) {
    const double x = (double)N * ctx->S[i];
    const double fl = std::floor(x);
    if (ctx->S[i] <= 0) M[i] = 0;
    else if (fl < 1.0) M[i] = 1;
    else {
      M[i] = (uint64_t)fl;
      elig[i] = 1;
      fr[i] = x - fl;
    }
    sum += M[i];
  }
  if (sum > N) return fail(ctx, MC_ERR_INVALID_ARG, "n_photons is smaller than the number of non-empty energy bins");
  uint64_t rem = N - sum;
  while (rem > 0) {
    int best = -1;
    for (int i = 0; i < n; ++i)
      if (elig[i] == 1 && (best < 0 || fr[i] > fr[best])) best = i;
    if (best < 0) break;
    M[best] += 1;
    elig[best] = 2;
    --rem;
  }
  if (rem) return fail(ctx, MC_ERR_INTERNAL, "stratification did not place every photon");
  std::memcpy(host, &seed, 8);
  auto* pre = reinterpret_cast<unsigned long long*>(host + 8);
  float* en = reinterpret_cast<float*>(pre + n + 1);
  float* wb = en + n;
  float* sn = wb + n;
  float* eb = sn + n;
  pre[0] = 0;
  for (int i = 0; i < n; ++i) {
    pre[i + 1] = pre[i] + M[i];
    en[i] = ctx->Ebin[i];
    wb[i] = M[i] ? (float)(ctx->S[i] / (double)M[i]) : 0.f;
    sn[i] = (float)ctx->S[i];
    eb[i] = (float)response_at(ctx, (double)ctx->Ebin[i]);
  }
  return MC_OK;
}

SpectrumView spectrum_view(const mc_ctx* ctx) {
  const int n = (int)ctx->S.size();
  unsigned char* base = (unsigned char*)ctx->d_spec + 8;
  SpectrumView sv;
  sv.prefix = reinterpret_cast<const unsigned long long*>(base);
  sv.energy = reinterpret_cast<const float*>(base + (size_t)(n + 1) * 8);
  sv.wbin = sv.energy + n;
  sv.sn = sv.wbin + n;
  sv.eta = sv.sn + n;
  sv.n_bins = n;
  return sv;
}

int check_ready(mc_ctx* ctx) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!ctx->have_tables) return fail(ctx, MC_ERR_STATE, "tables not loaded");
  if (ctx->mesh_mode ? !ctx->have_mesh : !ctx->have_volume)
    return fail(ctx, MC_ERR_STATE, ctx->mesh_mode ? "mesh not loaded" : "volume not loaded");
  if (!ctx->have_spectrum) return fail(ctx, MC_ERR_STATE, "spectrum not set");
  if (!ctx->have_geometry) return fail(ctx, MC_ERR_STATE, "geometry not set");
  if (ctx->opt.doppler && !ctx->bound)
    return fail(ctx, MC_ERR_STATE, "Doppler broadening needs the bound-electron tables (version 2)");
  const double rmax = ctx->mesh_mode ? ctx->mesh_rmax
                                     : 0.5 * std::sqrt((double)ctx->nx * ctx->dx * ctx->nx * ctx->dx +
                                                       (double)ctx->ny * ctx->dy * ctx->ny * ctx->dy);
  if (!(rmax < ctx->sod) || !(rmax < (double)ctx->sdd - ctx->sod))
    return fail(ctx, MC_ERR_INVALID_ARG, "the volume must lie strictly between source and detector");
  return MC_OK;
}

// Shared body of mc_project / mc_project_histories.  Inputs are staged in a
// pinned host buffer and the whole projection is one enqueue sequence: spectrum
// block (with the seed) and angles to the device, counter and tally resets,
// primary, transport, finalize, counters back.  With opt.use_graph the sequence
// is captured once into a CUDA graph and replayed while its launch shape
// (sizes, pointers, options) stays the same; the seed is read on the device, so
// one graph serves every seed.
MeshView mesh_view(const mc_ctx* c) {
  MeshView m;
  m.nodes = c->d_mesh_nodes;
  m.tris = c->d_mesh_tris;
  m.bodies = c->d_mesh_bodies;
  m.body_rho = c->d_mesh_rho;
  m.n_nodes = c->mesh_nodes;
  m.n_tris = c->mesh_tris;
  m.n_bodies = c->mesh_bodies;
  return m;
}

int project_impl(mc_ctx* ctx, const float* angles, int n_angles, uint64_t N, uint64_t h_begin, uint64_t h_count,
                 float step, uint64_t seed, float* primary_out, float* scatter_out, float* var_out, void* stream) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  (void)cudaGetLastError();  // a failed call elsewhere must not be blamed on this one
  if (!(step > 0.f) || !std::isfinite(step)) return fail(ctx, MC_ERR_INVALID_ARG, "step_mm must be > 0");
  {
    // bound the steps of one march: the longest chord is the volume diagonal
    const double diag = std::sqrt((double)ctx->nx * ctx->dx * ctx->nx * ctx->dx + (double)ctx->ny * ctx->dy * ctx->ny * ctx->dy +
                                  (double)ctx->nz * ctx->dz * ctx->nz * ctx->dz);
    if (diag / step > 4.0e6) return fail(ctx, MC_ERR_INVALID_ARG, "step_mm too small: more than 4e6 steps per chord");
  }
  if (N < 1) return fail(ctx, MC_ERR_INVALID_ARG, "n_photons must be >= 1");
  if (h_begin > N || h_count > N - h_begin) return fail(ctx, MC_ERR_INVALID_ARG, "history range outside the run");
  if (var_out && ctx->opt.n_batches < 2) return fail(ctx, MC_ERR_INVALID_ARG, "scatter_var_out needs n_batches >= 2");
  if (!angles || n_angles < 1) return fail(ctx, MC_ERR_INVALID_ARG, "n_angles must be >= 1 with a host angle array");
  for (int i = 0; i < n_angles; ++i)
    if (!std::isfinite(angles[i])) return fail(ctx, MC_ERR_INVALID_ARG, "angles must be finite");
  const int nb_img = var_out ? ctx->opt.n_batches : 1;
  rc = stage_tables(ctx);
  if (rc) return rc;
  const size_t img = (size_t)ctx->nu * ctx->nv * n_angles;

  // ---- buffers (allocated before any capture)
  const int nbins = (int)ctx->S.size();
  const size_t spec_bytes = spectrum_block_bytes(nbins);
  const size_t ang_off = (spec_bytes + 255) / 256 * 256;
  const size_t st_off = (ang_off + (size_t)n_angles * 4 + 255) / 256 * 256;
  const size_t pin_bytes = st_off + S_NSTAT * 8;
  if (pin_bytes > ctx->h_pin_cap) {
    if (ctx->h_pin) cudaFreeHost(ctx->h_pin);
    ctx->h_pin = nullptr;
    ctx->h_pin_cap = 0;
    CK(cudaMallocHost((void**)&ctx->h_pin, pin_bytes), "pinned staging allocation");
    ctx->h_pin_cap = pin_bytes;
  }
  {
    unsigned char* d = (unsigned char*)ctx->d_spec;
    CK(ensure(d, ctx->d_spec_cap, spec_bytes), "spectrum allocation");
    ctx->d_spec = d;
  }
  if (n_angles > ctx->angles_cap) {
    if (ctx->d_angles) cudaFree(ctx->d_angles);
    ctx->d_angles = nullptr;
    ctx->angles_cap = 0;
    CK(cudaMalloc((void**)&ctx->d_angles, (size_t)n_angles * 4), "angle allocation");
    ctx->angles_cap = n_angles;
  }
  if (scatter_out) CK(ensure(ctx->d_tally, ctx->tally_cap, img * nb_img), "tally allocation");
  // the previous call synchronised its stream, so the pinned buffer is free
  rc = fill_spectrum(ctx, N, seed, ctx->h_pin, scatter_out != nullptr);
  if (rc) return rc;
  std::memcpy(ctx->h_pin + ang_off, angles, (size_t)n_angles * 4);
  const SpectrumView sv = spectrum_view(ctx);

  // ---- kernel parameters (zeroed first: they also form the graph key)
  PrimaryParams pp;
  TransportParams tp;
  std::memset((void*)&pp, 0, sizeof(pp));
  std::memset((void*)&tp, 0, sizeof(tp));
  int grid = 0, block = 0;
  if (primary_out) {
    pp.tab = table_view(ctx);
    pp.vol = volume_view(ctx);
    pp.geo = geom_view(ctx);
    pp.spec = sv;
    pp.angles = ctx->d_angles;
    pp.n_angles = n_angles;
    pp.step = step;
    pp.out = primary_out;
    // measured crossover (2048^2 x 512^3): shared totals win above ~7% changing neighbour pairs
    pp.shared_acc = ctx->mat_change > 0.07 ? 1 : 0;
  }
  if (scatter_out) {
    tp.tab = table_view(ctx);
    if (ctx->mesh_mode) {
      // the box only orders the point-detector jobs by their chord toward the panel
      tp.vol.hx = ctx->mesh_half[0];
      tp.vol.hy = ctx->mesh_half[1];
      tp.vol.hz = ctx->mesh_half[2];
      tp.geometry = GEO_MESH;
      tp.mesh = mesh_view(ctx);
    } else {
      tp.vol = volume_view(ctx);
      tp.geometry = tp.vol.layout;
    }
    tp.geo = geom_view(ctx);
    tp.spec = sv;
    tp.angles = ctx->d_angles;
    tp.n_angles = n_angles;
    tp.n_photons = N;
    tp.h_begin = h_begin;
    tp.h_count = h_count;
    tp.step = step;
    tp.seed = 0;
    tp.seed_dev = reinterpret_cast<const unsigned long long*>(ctx->d_spec);
    tp.n_split = ctx->opt.n_split;
    tp.nee_mode = ctx->opt.nee_mode;
    tp.doppler = ctx->opt.doppler;
    tp.forced = ctx->opt.forced_detection;
    tp.rr_threshold = ctx->opt.rr_threshold;
    tp.max_order = ctx->opt.max_scatter_order;
    tp.n_batches = nb_img;
    tp.tally = ctx->d_tally;
    tp.stats = ctx->d_stats;
    const size_t tally_pixels = img * nb_img;
    if (ctx->opt.tally_mode == MC_TALLY_SHARED) {
      if (tally_pixels > (size_t)kSharedTallyMaxPixels)
        return fail(ctx, MC_ERR_INVALID_ARG, "tally_mode SHARED needs n_batches x n_angles x nu x nv <= 12288");
      tp.tally_mode = TALLY_SHARED;
    } else if (ctx->opt.tally_mode == MC_TALLY_TILED && !ctx->mesh_mode) {
      const int tu = std::min(ctx->opt.tile_u, ctx->nu), tv = std::min(ctx->opt.tile_v, ctx->nv);
      if ((size_t)nb_img * tu * tv > (size_t)kSharedTallyMaxPixels)
        return fail(ctx, MC_ERR_INVALID_ARG, "tally_mode TILED needs n_batches x tile_u x tile_v <= 12288");
      tp.tally_mode = TALLY_TILED;
      tp.tile_u = tu;
      tp.tile_v = tv;
      tp.n_tu = (ctx->nu + tu - 1) / tu;
      tp.n_tiles = tp.n_tu * ((ctx->nv + tv - 1) / tv);
    } else if (ctx->opt.tally_mode == MC_TALLY_WARP) {
      tp.tally_mode = TALLY_WARP;
    } else {
      // automatic and global: plain FP64 adds, the fastest of the unstratified tallies (measured down to
      // an 8 x 8 panel); the tile-stratified tally is chosen explicitly or by the autotuner
      tp.tally_mode = TALLY_GLOBAL;
    }
    if (tp.forced) {
      const size_t fp = tp.tally_mode == TALLY_TILED ? (size_t)tp.tile_u * tp.tile_v : (size_t)ctx->nu * ctx->nv;
      if (fp > (size_t)MC_FORCED_MAX_PIXELS)
        return fail(ctx, MC_ERR_INVALID_ARG,
                    "forced_detection needs at most MC_FORCED_MAX_PIXELS (65536) pixels per panel or tile");
    }
    block = ctx->opt.block_size ? ctx->opt.block_size : 256;
    const int smem = transport_smem_bytes(tp.tab, sv.n_bins, block, transport_shared_pixels(tp));
    int per_sm = ctx->opt.blocks_per_sm;
    if (per_sm == 0) {
      CK(transport_occupancy(block, smem, &per_sm, ctx->mesh_mode, ctx->layout), "occupancy query");
      per_sm = std::max(1, per_sm);
    }
    const unsigned long long work = (unsigned long long)n_angles * h_count;
    const unsigned long long need = (work + block - 1) / block;
    grid = (int)std::max<unsigned long long>(1, std::min<unsigned long long>(need, (unsigned long long)ctx->sm_count * per_sm));
    if (work == 0) grid = 0;
    if (tp.tally_mode == TALLY_TILED && grid > 0) {
      // chunks of one (angle, tile): about 8 per block for balance, at least 4 histories per thread so
      // that the wait for a chunk's last photon stays short, at most a tile's share of the run
      const unsigned long long per_tile = (h_count + tp.n_tiles - 1) / tp.n_tiles;
      unsigned long long c = work / ((unsigned long long)grid * 8);
      c = std::max<unsigned long long>(c, 4ull * block);
      c = std::max<unsigned long long>(1, std::min(c, per_tile));
      tp.tile_chunk = c;
      tp.tile_k = (per_tile + c - 1) / c;
      tp.n_chunks = (unsigned long long)n_angles * tp.n_tiles * std::max<unsigned long long>(1, tp.tile_k);
    }
  }

  // ---- the enqueue sequence
  unsigned long long* h_st = reinterpret_cast<unsigned long long*>(ctx->h_pin + st_off);
  // under capture an event record must be an external record node to time the replay
  auto record = [&](cudaEvent_t ev, cudaStream_t q, bool capture) {
    return cudaEventRecordWithFlags(ev, q, capture ? cudaEventRecordExternal : cudaEventRecordDefault);
  };
  auto enqueue = [&](cudaStream_t q, bool capture) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(ctx->d_spec, ctx->h_pin, spec_bytes, cudaMemcpyHostToDevice, q);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->d_angles, ctx->h_pin + ang_off, (size_t)n_angles * 4, cudaMemcpyHostToDevice, q);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_stats, 0, S_NSTAT * 8, q);
    if (e == cudaSuccess && primary_out) {
      e = record(ctx->ev[2], q, capture);
      if (e == cudaSuccess) e = ctx->mesh_mode ? launch_primary_mesh(pp, mesh_view(ctx), q) : launch_primary(pp, q);
      if (e == cudaSuccess) e = record(ctx->ev[3], q, capture);
    }
    if (e == cudaSuccess && scatter_out) {
      e = cudaMemsetAsync(ctx->d_tally, 0, img * nb_img * sizeof(double), q);
      if (e == cudaSuccess) e = record(ctx->ev[0], q, capture);
      if (e == cudaSuccess && grid > 0) e = launch_transport(tp, grid, block, q);
      if (e == cudaSuccess) e = record(ctx->ev[1], q, capture);
      if (e == cudaSuccess) e = launch_finalize(ctx->d_tally, nb_img, img, scatter_out, var_out, q);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_st, ctx->d_stats, S_NSTAT * 8, cudaMemcpyDeviceToHost, q);
    return e;
  };
  if (ctx->opt.use_graph && !ctx->mesh_mode) {
    // graph key: every parameter and size the captured sequence depends on
    std::vector<unsigned char> key(sizeof(pp) + sizeof(tp) + 64);
    std::memcpy(key.data(), &pp, sizeof(pp));
    std::memcpy(key.data() + sizeof(pp), (const void*)&tp, sizeof(tp));
    const uint64_t extra[8] = {(uint64_t)grid, (uint64_t)block, (uint64_t)nb_img, (uint64_t)img, (uint64_t)(uintptr_t)var_out,
                               (uint64_t)(uintptr_t)scatter_out, (uint64_t)(uintptr_t)ctx->h_pin, (uint64_t)spec_bytes};
    std::memcpy(key.data() + sizeof(pp) + sizeof(tp), extra, 64);
    if (!ctx->graph_exec || key != ctx->graph_key) {
      if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
      ctx->graph_exec = nullptr;
      if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking), "capture stream");
      CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal), "graph capture");
      const cudaError_t e = enqueue(ctx->cap_stream, true);
      cudaGraph_t graph = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &graph);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(ctx, e != cudaSuccess ? e : e2, "graph capture");
      }
      const cudaError_t e3 = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e3 != cudaSuccess) return cuda_fail(ctx, e3, "graph instantiate");
      ctx->graph_key.swap(key);
      ++ctx->graph_builds;
    }
    CK(cudaGraphLaunch(ctx->graph_exec, s), "graph launch");
  } else {
    CK(enqueue(s, false), "projection enqueue");
  }
  CK(cudaStreamSynchronize(s), "stream synchronize");
  float ms_t = 0, ms_p = 0;
  if (scatter_out) CK(cudaEventElapsedTime(&ms_t, ctx->ev[0], ctx->ev[1]), "event time");
  if (primary_out) CK(cudaEventElapsedTime(&ms_p, ctx->ev[2], ctx->ev[3]), "event time");
  unsigned long long st[S_NSTAT];
  std::memcpy(st, h_st, sizeof(st));
  const int map[10] = {S_HIST, S_FLIGHT_STEPS, S_NEE_STEPS, S_NEE_RAYS, S_PHOTO, S_COMPTON, S_RAYLEIGH, S_ESCAPE, S_LIMIT, S_SAMPLER_FAIL};
  for (int i = 0; i < 10; ++i) ctx->stats[i] = (double)st[map[i]];
  ctx->stats[10] = ms_t;
  ctx->stats[11] = ms_p;
  if (st[S_INTERNAL]) return fail(ctx, MC_ERR_TIMEOUT, "a block gave up waiting for its table copy");
  if (st[S_BAD_SMEM]) return fail(ctx, MC_ERR_INTERNAL, "transport launched with less shared memory than its layout");
  if (st[S_LIMIT] || st[S_SAMPLER_FAIL])
    return fail(ctx, MC_ERR_LIMIT, "histories hit the scatter-order or sampler cap (outputs valid)");
  return MC_OK;
}

// Savitzky-Golay hat matrix H = V (V^T V)^-1 V^T for window win, order k (FP64,
// Gauss-Jordan on the (k+1)^2 normal matrix).
void sg_hat(int win, int k, std::vector<float>& H) {
  const int m = win / 2, q = k + 1;
  std::vector<double> V(win * q), A(q * q, 0.0), Ai(q * q, 0.0);
  for (int j = 0; j < win; ++j)
    for (int c = 0; c < q; ++c) V[j * q + c] = std::pow((double)(j - m), c);
  for (int r = 0; r < q; ++r)
    for (int c = 0; c < q; ++c) {
      double s = 0;
      for (int j = 0; j < win; ++j) s += V[j * q + r] * V[j * q + c];
      A[r * q + c] = s;
    }
  for (int r = 0; r < q; ++r) Ai[r * q + r] = 1.0;
  for (int col = 0; col < q; ++col) {
    int piv = col;
    for (int r = col + 1; r < q; ++r)
      if (std::fabs(A[r * q + col]) > std::fabs(A[piv * q + col])) piv = r;
    for (int c = 0; c < q; ++c) {
      std::swap(A[col * q + c], A[piv * q + c]);
      std::swap(Ai[col * q + c], Ai[piv * q + c]);
    }
    const double d = A[col * q + col];
    for (int c = 0; c < q; ++c) {
      A[col * q + c] /= d;
      Ai[col * q + c] /= d;
    }
    for (int r = 0; r < q; ++r) {
      if (r == col) continue;
      const double f = A[r * q + col];
      for (int c = 0; c < q; ++c) {
        A[r * q + c] -= f * A[col * q + c];
        Ai[r * q + c] -= f * Ai[col * q + c];
      }
    }
  }
  H.assign(win * win, 0.f);
  for (int p = 0; p < win; ++p)
    for (int j = 0; j < win; ++j) {
      double s = 0;
      for (int r = 0; r < q; ++r)
        for (int c = 0; c < q; ++c) s += V[p * q + r] * Ai[r * q + c] * V[j * q + c];
      H[p * win + j] = (float)s;
    }
}

}  // namespace

extern "C" {

void mc_default_options(mc_options* o) {
  if (!o) return;
  o->n_split = 10;
  o->rr_threshold = 0.f;
  o->max_scatter_order = 64;
  o->n_batches = 1;
  o->block_size = 0;
  o->blocks_per_sm = 0;
  o->tally_mode = MC_TALLY_AUTO;
  o->sg_window = 9;
  o->sg_order = 3;
  o->cubic_a = -0.5f;
  o->denoise_mode = 0;
  o->voxel_layout = 0;
  o->use_graph = 0;
  o->nee_mode = 0;
  o->doppler = 0;
  o->forced_detection = 0;
  o->tile_u = 64;
  o->tile_v = 64;
}

int mc_create(mc_ctx** out, int cuda_device, const mc_options* opt) {
  if (!out) return MC_ERR_INVALID_ARG;
  *out = nullptr;
  mc_ctx* ctx = new (std::nothrow) mc_ctx();
  if (!ctx) return MC_ERR_OOM;
  mc_default_options(&ctx->opt);
  if (opt) {
    std::string why;
    if (validate_options(opt, why)) {
      delete ctx;
      return MC_ERR_INVALID_ARG;
    }
    ctx->opt = *opt;
  }
  ctx->device = cuda_device;
  cudaError_t e = cudaSetDevice(cuda_device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, cuda_device);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_stats, S_NSTAT * 8);
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->ev[i]);
  if (e != cudaSuccess) {
    mc_destroy(ctx);
    return e == cudaErrorMemoryAllocation ? MC_ERR_OOM : MC_ERR_CUDA;
  }
  *out = ctx;
  return MC_OK;
}

void mc_destroy(mc_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  cudaFree(ctx->d_blob);
  cudaFree(ctx->d_vox);
  cudaFree(ctx->d_mesh_nodes);
  cudaFree(ctx->d_mesh_tris);
  cudaFree(ctx->d_mesh_bodies);
  cudaFree(ctx->d_mesh_rho);
  cudaFree(ctx->d_spec);
  cudaFree(ctx->d_tally);
  cudaFree(ctx->d_stats);
  cudaFree(ctx->d_angles);
  cudaFree(ctx->d_post);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  denoiser_destroy(ctx->denoiser);
  if (ctx->h_pin) cudaFreeHost(ctx->h_pin);
  delete ctx;
}

int mc_set_options(mc_ctx* ctx, const mc_options* opt) {
  if (!ctx || !opt) return MC_ERR_INVALID_ARG;
  std::string why;
  if (validate_options(opt, why)) return fail(ctx, MC_ERR_INVALID_ARG, why);
  ctx->opt = *opt;
  return MC_OK;
}

const char* mc_last_error(const mc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int mc_load_tables(mc_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(ctx, MC_ERR_INVALID_ARG, "null argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(ctx, MC_ERR_IO, std::string("cannot open table file ") + path);
  char magic[8];
  int32_t hdr[4];
  double e2[2], k6[6];
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "MCXTAB01", 8) == 0 &&
            std::fread(hdr, 4, 4, f) == 4 && std::fread(e2, 8, 2, f) == 2 && std::fread(k6, 8, 6, f) == 6;
  if (!ok || (hdr[0] != 1 && hdr[0] != 2) || hdr[3] != kMaxComp || hdr[2] < 2) {
    std::fclose(f);
    return fail(ctx, MC_ERR_IO, "malformed table header");
  }
  if (hdr[1] < 1 || hdr[1] > kMaxMat) {
    std::fclose(f);
    return fail(ctx, MC_ERR_INVALID_ARG, "the table holds more materials than MC_MAX_MATERIALS");
  }
  const int nm = hdr[1], nE = hdr[2];
  int ncomp[kMaxMat];
  double comp[kMaxMat][kMaxComp][3];
  for (int m = 0; m < nm; ++m) {
    char name[16];
    double dens;
    int32_t nc[2];
    double buf[kMaxComp * 3];
    if (std::fread(name, 1, 16, f) != 16 || std::fread(&dens, 8, 1, f) != 1 || std::fread(nc, 4, 2, f) != 2 ||
        std::fread(buf, 8, kMaxComp * 3, f) != (size_t)kMaxComp * 3 || nc[0] < 1 || nc[0] > kMaxComp) {
      std::fclose(f);
      return fail(ctx, MC_ERR_IO, "malformed material record");
    }
    ncomp[m] = nc[0];
    for (int i = 0; i < kMaxComp; ++i)
      for (int j = 0; j < 3; ++j) comp[m][i][j] = buf[i * 3 + j];
    for (int i = 0; i < nc[0]; ++i)
      if (!(comp[m][i][2] > 0)) {
        std::fclose(f);
        return fail(ctx, MC_ERR_IO, "form-factor width must be positive");
      }
  }
  const size_t n = (size_t)nm * nE;
  std::vector<double> a(n), b(n), c(n), d(n), e(hdr[0] == 2 ? n : 0);
  ok = std::fread(a.data(), 8, n, f) == n && std::fread(b.data(), 8, n, f) == n && std::fread(c.data(), 8, n, f) == n &&
       std::fread(d.data(), 8, n, f) == n && (hdr[0] != 2 || std::fread(e.data(), 8, n, f) == n);
  std::fclose(f);
  if (!ok) return fail(ctx, MC_ERR_IO, "truncated table arrays");
  ctx->n_mat = nm;
  ctx->n_E = nE;
  ctx->E0 = e2[0];
  ctx->dE = e2[1];
  ctx->r0 = k6[0];
  ctx->mec2 = k6[1];
  ctx->hc = k6[2];
  ctx->pe.swap(a);
  ctx->in.swap(b);
  ctx->co.swap(c);
  ctx->icoh.swap(d);
  ctx->iincoh.swap(e);
  ctx->bound = hdr[0] == 2;
  for (int m = 0; m < nm; ++m) {
    ctx->n_comp[m] = ncomp[m];
    std::memcpy(ctx->comp[m], comp[m], sizeof(comp[m]));
  }
  ctx->have_tables = true;
  ctx->eta.clear();  // a response belongs to the previous tables' nodes
  ctx->blob_dirty = true;
  return MC_OK;
}

int mc_load_volume(mc_ctx* ctx, const uint8_t* mat, const uint16_t* rho_fp16, int nx, int ny, int nz, float dx,
                   float dy, float dz, int is_device_ptr, void* stream) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!ctx->have_tables) return fail(ctx, MC_ERR_STATE, "load tables before the volume");
  if (!mat || !rho_fp16 || nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0) || !(dz > 0))
    return fail(ctx, MC_ERR_INVALID_ARG, "bad volume arguments");
  const size_t n = (size_t)nx * ny * nz;
  if (n > (size_t)INT32_MAX || packed_words(nx, ny, nz, VOX_BRICK) > (size_t)INT32_MAX)
    return fail(ctx, MC_ERR_INVALID_ARG, "volume larger than 2^31 voxels");
  if (nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20))
    return fail(ctx, MC_ERR_INVALID_ARG, "volume dimension above 2^20");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)stream;
  if (!is_device_ptr) {
    // host data: validate here
    for (size_t i = 0; i < n; ++i) {
      if (mat[i] >= ctx->n_mat) return fail(ctx, MC_ERR_INVALID_ARG, "material id outside the table");
      const uint16_t h = rho_fp16[i];
      if ((h & 0x8000u) && (h & 0x7fffu)) return fail(ctx, MC_ERR_INVALID_ARG, "negative density");
      if (((h >> 10) & 31u) == 31u) return fail(ctx, MC_ERR_INVALID_ARG, "non-finite density");
    }
  }
  ctx->have_volume = false;
  // stage the two arrays on the device, validate, pack into voxel words
  uint8_t* st_mat = nullptr;
  uint16_t* st_rho = nullptr;
  CK(cudaMallocAsync((void**)&st_mat, n, s), "volume staging allocation");
  cudaError_t e = cudaMallocAsync((void**)&st_rho, n * 2, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(st_mat, s);
    return cuda_fail(ctx, e, "volume staging allocation");
  }
  auto release = [&]() {
    cudaFreeAsync(st_mat, s);
    cudaFreeAsync(st_rho, s);
  };
  const cudaMemcpyKind kind = is_device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  e = cudaMemcpyAsync(st_mat, mat, n, kind, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(st_rho, rho_fp16, n * 2, kind, s);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(ctx, e, "volume copy");
  }
  if (is_device_ptr) {
    // device data: validate on the device (material ids, finite non-negative densities)
    int bad = 0;
    e = validate_volume_device(st_mat, st_rho, n, ctx->n_mat, s, &bad);
    if (e != cudaSuccess || bad) {
      release();
      if (e != cudaSuccess) return cuda_fail(ctx, e, "volume validation");
      return fail(ctx, MC_ERR_INVALID_ARG, "volume holds an unknown material id or an invalid density");
    }
  }
  // default layout: x fastest while the packed volume fits in 3/4 of L2 (measured faster there);
  // 4^3 bricks once it streams from HBM (every ray direction then reuses its sectors)
  int layout = ctx->opt.voxel_layout == 2 ? VOX_BRICK : VOX_LIN;
  if (ctx->opt.voxel_layout == 0) {
    int l2 = 0;
    CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device), "L2 size query");
    if ((double)packed_words(nx, ny, nz, VOX_LIN) * 4.0 > 0.75 * (double)l2) layout = VOX_BRICK;
  }
  const size_t words = packed_words(nx, ny, nz, layout);
  e = ensure(ctx->d_vox, ctx->vox_cap, words);
  if (e == cudaSuccess) e = pack_volume(st_mat, st_rho, nx, ny, nz, layout, ctx->d_vox, words, s);
  double change = 0.0;
  if (e == cudaSuccess) e = material_change_fraction(st_mat, nx, ny, nz, s, &change);
  release();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "volume packing");
  CK(cudaStreamSynchronize(s), "volume load");
  ctx->layout = layout;
  ctx->mat_change = change;
  ctx->nx = nx; ctx->ny = ny; ctx->nz = nz;
  ctx->dx = dx; ctx->dy = dy; ctx->dz = dz;
  ctx->have_volume = true;
  ctx->mesh_mode = false;
  return MC_OK;
}

int mc_load_mesh(mc_ctx* ctx, const float* vertices, int n_vertices, const int* triangles, const int* tri_body,
                 int n_triangles, const int* body_material, const float* body_density, const int* body_parent,
                 int n_bodies) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!ctx->have_tables) return fail(ctx, MC_ERR_STATE, "load tables before the mesh");
  if (!vertices || !triangles || !tri_body || !body_material || !body_density || !body_parent || n_vertices < 3 ||
      n_triangles < 1 || n_bodies < 1 || n_bodies > MC_MAX_BODIES)
    return fail(ctx, MC_ERR_INVALID_ARG, "bad mesh sizes");
  for (int b = 0; b < n_bodies; ++b)
    if (body_material[b] < 0 || body_material[b] >= ctx->n_mat || !(body_density[b] >= 0.f) ||
        !std::isfinite(body_density[b]) || body_parent[b] < -1 || body_parent[b] >= b)
      return fail(ctx, MC_ERR_INVALID_ARG, "bad body (material, density >= 0, parent -1 or an earlier body)");
  double rmax = 0;
  float half[3] = {0.f, 0.f, 0.f};
  for (int i = 0; i < n_vertices; ++i) {
    const float* p = vertices + 3 * i;
    if (!std::isfinite(p[0]) || !std::isfinite(p[1]) || !std::isfinite(p[2]))
      return fail(ctx, MC_ERR_INVALID_ARG, "non-finite vertex");
    rmax = std::max(rmax, std::sqrt((double)p[0] * p[0] + (double)p[1] * p[1]));
    for (int a = 0; a < 3; ++a) half[a] = std::max(half[a], std::fabs(p[a]));
  }
  for (int k = 0; k < n_triangles; ++k) {
    if (tri_body[k] < 0 || tri_body[k] >= n_bodies) return fail(ctx, MC_ERR_INVALID_ARG, "triangle body out of range");
    for (int q = 0; q < 3; ++q)
      if (triangles[3 * k + q] < 0 || triangles[3 * k + q] >= n_vertices)
        return fail(ctx, MC_ERR_INVALID_ARG, "triangle vertex out of range");
  }
  std::vector<float4> nodes, tris;
  const int depth = build_mesh_bvh(vertices, triangles, tri_body, n_triangles, nodes, tris);
  if (depth >= 63) return fail(ctx, MC_ERR_INTERNAL, "bounding-volume hierarchy deeper than the device stack");
  std::vector<int4> bodies(n_bodies);
  std::vector<float> rho(n_bodies);
  for (int b = 0; b < n_bodies; ++b) {
    const int pb = body_parent[b];
    float dens = body_density[b];
    int dbits;
    std::memcpy(&dbits, &dens, 4);
    bodies[b] = make_int4(body_material[b], pb, pb >= 0 ? body_material[pb] : 0, dbits);
    rho[b] = body_density[b];
  }
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  cudaFree(ctx->d_mesh_nodes);
  cudaFree(ctx->d_mesh_tris);
  cudaFree(ctx->d_mesh_bodies);
  cudaFree(ctx->d_mesh_rho);
  ctx->d_mesh_nodes = ctx->d_mesh_tris = nullptr;
  ctx->d_mesh_bodies = nullptr;
  ctx->d_mesh_rho = nullptr;
  ctx->have_mesh = ctx->mesh_mode = false;
  CK(cudaMalloc((void**)&ctx->d_mesh_nodes, nodes.size() * sizeof(float4)), "mesh allocation");
  CK(cudaMalloc((void**)&ctx->d_mesh_tris, tris.size() * sizeof(float4)), "mesh allocation");
  CK(cudaMalloc((void**)&ctx->d_mesh_bodies, bodies.size() * sizeof(int4)), "mesh allocation");
  CK(cudaMalloc((void**)&ctx->d_mesh_rho, rho.size() * sizeof(float)), "mesh allocation");
  CK(cudaMemcpy(ctx->d_mesh_nodes, nodes.data(), nodes.size() * sizeof(float4), cudaMemcpyHostToDevice), "mesh upload");
  CK(cudaMemcpy(ctx->d_mesh_tris, tris.data(), tris.size() * sizeof(float4), cudaMemcpyHostToDevice), "mesh upload");
  CK(cudaMemcpy(ctx->d_mesh_bodies, bodies.data(), bodies.size() * sizeof(int4), cudaMemcpyHostToDevice), "mesh upload");
  CK(cudaMemcpy(ctx->d_mesh_rho, rho.data(), rho.size() * sizeof(float), cudaMemcpyHostToDevice), "mesh upload");
  ctx->mesh_nodes = (int)(nodes.size() / 2);
  ctx->mesh_tris = n_triangles;
  ctx->mesh_bodies = n_bodies;
  ctx->mesh_rmax = rmax;
  for (int a = 0; a < 3; ++a) ctx->mesh_half[a] = half[a];
  ctx->have_mesh = ctx->mesh_mode = true;
  return MC_OK;
}

int mc_set_spectrum(mc_ctx* ctx, const double* weights, const float* energies, int n) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!ctx->have_tables) return fail(ctx, MC_ERR_STATE, "load tables before the spectrum");
  if (!weights || !energies || n < 1 || n > MC_MAX_BINS) return fail(ctx, MC_ERR_INVALID_ARG, "bad spectrum size");
  const double Emax = ctx->E0 + ctx->dE * (ctx->n_E - 1);
  double sum = 0;
  for (int i = 0; i < n; ++i) {
    if (!(weights[i] >= 0) || !std::isfinite(weights[i])) return fail(ctx, MC_ERR_INVALID_ARG, "weights must be >= 0");
    if (!((double)energies[i] >= ctx->E0) || !((double)energies[i] <= Emax))
      return fail(ctx, MC_ERR_INVALID_ARG, "energy outside the table range");
    sum += weights[i];
  }
  if (!(sum > 0)) return fail(ctx, MC_ERR_INVALID_ARG, "weights sum to zero");
  ctx->S.assign(n, 0.0);
  ctx->Ebin.assign(energies, energies + n);
  for (int i = 0; i < n; ++i) ctx->S[i] = weights[i] / sum;
  ctx->have_spectrum = true;
  ctx->blob_dirty = true;
  return MC_OK;
}

int mc_set_detector_response(mc_ctx* ctx, const double* eta, int n) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!ctx->have_tables) return fail(ctx, MC_ERR_STATE, "load tables before the detector response");
  if (!eta) {
    ctx->eta.clear();
  } else {
    if (n != ctx->n_E) return fail(ctx, MC_ERR_INVALID_ARG, "the response needs one value per table energy node");
    for (int i = 0; i < n; ++i)
      if (!(eta[i] >= 0.0) || !std::isfinite(eta[i])) return fail(ctx, MC_ERR_INVALID_ARG, "response values must be >= 0");
    ctx->eta.assign(eta, eta + n);
  }
  ctx->blob_dirty = true;
  return MC_OK;
}

int mc_set_geometry(mc_ctx* ctx, float sod, float sdd, int nu, int nv, float pu, float pv) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!(sod > 0) || !(sdd > sod) || nu < 1 || nv < 1 || !(pu > 0) || !(pv > 0) || (double)nu * nv > 1.0e9)
    return fail(ctx, MC_ERR_INVALID_ARG, "bad geometry");
  ctx->sod = sod; ctx->sdd = sdd; ctx->nu = nu; ctx->nv = nv; ctx->pu = pu; ctx->pv = pv;
  ctx->have_geometry = true;
  return MC_OK;
}

int mc_project(mc_ctx* ctx, const float* angles, int n_angles, uint64_t n_photons, float step_mm, uint64_t seed,
               float* primary_out, float* scatter_out, float* scatter_var_out, void* stream) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  const int rc = check_ready(ctx);
  if (rc) return rc;
  if (!primary_out && !scatter_out) return fail(ctx, MC_ERR_INVALID_ARG, "no output requested");
  if (scatter_var_out && !scatter_out) return fail(ctx, MC_ERR_INVALID_ARG, "variance needs scatter_out");
  return project_impl(ctx, angles, n_angles, n_photons, 0, n_photons, step_mm, seed, primary_out, scatter_out,
                      scatter_var_out, stream);
}

int mc_project_histories(mc_ctx* ctx, const float* angles, int n_angles, uint64_t n_photons, uint64_t h_begin,
                         uint64_t h_count, float step_mm, uint64_t seed, float* scatter_out, void* stream) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  const int rc = check_ready(ctx);
  if (rc) return rc;
  if (!scatter_out) return fail(ctx, MC_ERR_INVALID_ARG, "scatter_out is required");
  return project_impl(ctx, angles, n_angles, n_photons, h_begin, h_count, step_mm, seed, nullptr, scatter_out,
                      nullptr, stream);
}

int mc_autotune(mc_ctx* ctx, const float* angles, int n_angles, uint64_t probe, float step_min, float step_max,
                float step_tol, mc_tuning* out, void* stream) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (ctx->mesh_mode) return fail(ctx, MC_ERR_STATE, "the autotuner tunes the voxel march: load a volume");
  if (!out || !angles || n_angles < 1 || probe < 1 || !(step_min > 0.f) || !(step_max >= step_min) || !(step_tol > 0.f))
    return fail(ctx, MC_ERR_INVALID_ARG, "bad autotune arguments");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const size_t n = (size_t)ctx->nu * ctx->nv * n_angles;
  float *d_ref = nullptr, *d_img = nullptr;
  CK(cudaMalloc((void**)&d_ref, n * 4), "autotune allocation");
  cudaError_t e = cudaMalloc((void**)&d_img, n * 4);
  if (e != cudaSuccess) {
    cudaFree(d_ref);
    return cuda_fail(ctx, e, "autotune allocation");
  }
  std::vector<float> ref(n), img(n);
  auto finish = [&](int code) {
    cudaFree(d_ref);
    cudaFree(d_img);
    return code;
  };
  // 1. largest step within tolerance of the finest
  rc = project_impl(ctx, angles, n_angles, 1, 0, 1, step_min, 1, d_ref, nullptr, nullptr, stream);
  if (rc) return finish(rc);
  e = cudaMemcpy(ref.data(), d_ref, n * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return finish(cuda_fail(ctx, e, "autotune readback"));
  double rn = 0;
  for (float v : ref) rn += (double)v * v;
  float best_step = step_min;
  double best_err = 0;
  const int n_cand = 8;
  for (int c = 0; c < n_cand; ++c) {
    const float st = step_max * std::pow(step_min / step_max, (float)c / (n_cand - 1));
    if (st <= step_min) break;
    rc = project_impl(ctx, angles, n_angles, 1, 0, 1, st, 1, d_img, nullptr, nullptr, stream);
    if (rc) return finish(rc);
    e = cudaMemcpy(img.data(), d_img, n * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return finish(cuda_fail(ctx, e, "autotune readback"));
    double dn = 0;
    for (size_t i = 0; i < n; ++i) dn += ((double)img[i] - ref[i]) * ((double)img[i] - ref[i]);
    const double err = rn > 0 ? std::sqrt(dn / rn) : 0;
    if (err <= step_tol) {
      best_step = st;
      best_err = err;
      break;
    }
  }
  // 2. launch shape at the chosen step
  const mc_options saved = ctx->opt;
  int smem = 0, max_per_sm = 1;
  {
    const TableView tv = table_view(ctx);
    smem = transport_smem_bytes(tv, (int)ctx->S.size(), 256, 0);
    e = transport_occupancy(256, smem, &max_per_sm, ctx->mesh_mode, ctx->layout);
    if (e != cudaSuccess) return finish(cuda_fail(ctx, e, "occupancy query"));
  }
  double best_rate = -1;
  mc_options best = saved;
  const int blocks[3] = {128, 192, 256};
  const int tallies[2] = {MC_TALLY_GLOBAL, MC_TALLY_WARP};
  for (int bi = 0; bi < 3; ++bi) {
    int occ = 1;
    e = transport_occupancy(blocks[bi], transport_smem_bytes(table_view(ctx), (int)ctx->S.size(), blocks[bi], 0), &occ,
                            ctx->mesh_mode, ctx->layout);
    if (e != cudaSuccess) return finish(cuda_fail(ctx, e, "occupancy query"));
    for (int per = 1; per <= std::max(1, occ); ++per) {
      for (int ti = 0; ti < 2; ++ti) {
        ctx->opt = saved;
        ctx->opt.block_size = blocks[bi];
        ctx->opt.blocks_per_sm = per;
        ctx->opt.tally_mode = tallies[ti];
        ctx->opt.use_graph = 0;
        double ms = 1e30;
        for (int rep = 0; rep < 2; ++rep) {
          rc = project_impl(ctx, angles, n_angles, probe, 0, probe, best_step, 7 + rep, nullptr, d_img, nullptr, stream);
          if (rc && rc != MC_ERR_LIMIT) {
            ctx->opt = saved;
            return finish(rc);
          }
          ms = std::min(ms, ctx->stats[10]);
        }
        const double rate = (double)probe * n_angles / (ms / 1e3);
        if (rate > best_rate) {
          best_rate = rate;
          best = ctx->opt;
        }
      }
    }
  }
  ctx->opt = saved;
  ctx->opt.block_size = best.block_size;
  ctx->opt.blocks_per_sm = best.blocks_per_sm;
  ctx->opt.tally_mode = best.tally_mode;
  // 3. Russian roulette threshold (Sec. II-C.1) by figure of merit 1 / (noise^2 x time): the noise is the
  //    batch estimate of the scatter image's relative L2 error; thresholds are multiples of the mean
  //    attenuated pseudo-particle score of a run without roulette
  float best_rr = 0.f;
  double fom0 = 0, best_fom = 0, rr_top = 0, tile_gain = 1.0;
  int best_tu = 0, best_tv = 0;
  {
    float* d_var = nullptr;
    e = cudaMalloc((void**)&d_var, n * 4);
    if (e != cudaSuccess) return finish(cuda_fail(ctx, e, "autotune allocation"));
    std::vector<float> var(n);
    mc_options shape = ctx->opt;  // the configuration whose figure of merit fom_of measures
    auto fom_of = [&](float rr, double* mean_score) -> int {
      ctx->opt = shape;
      ctx->opt.rr_threshold = rr;
      ctx->opt.n_batches = 8;
      ctx->opt.use_graph = 0;
      int r = project_impl(ctx, angles, n_angles, probe, 0, probe, best_step, 11, nullptr, d_img, d_var, stream);
      if (r && r != MC_ERR_LIMIT) return r;
      if (cudaMemcpy(img.data(), d_img, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(var.data(), d_var, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_fail(ctx, cudaGetLastError(), "autotune readback");
      double s2 = 0, v = 0, sum = 0;
      for (size_t i = 0; i < n; ++i) {
        s2 += (double)img[i] * img[i];
        v += var[i];
        sum += img[i];
      }
      const double ms = ctx->stats[10];
      if (mean_score) *mean_score = ctx->stats[3] > 0 ? sum / ctx->stats[3] : 0.0;
      best_fom = (s2 > 0 && v > 0 && ms > 0) ? s2 / (v * ms) : 0.0;  // 1 / (rel noise^2 x ms)
      return MC_OK;
    };
    double xbar = 0;
    rc = fom_of(0.f, &xbar);
    if (rc) {
      cudaFree(d_var);
      ctx->opt = saved;
      return finish(rc);
    }
    fom0 = best_fom;
    double top = fom0;
    const float mult[4] = {0.3f, 1.f, 3.f, 10.f};
    for (int c = 0; c < 4 && xbar > 0; ++c) {
      const float thr = (float)(mult[c] * xbar);
      rc = fom_of(thr, nullptr);
      if (rc) {
        cudaFree(d_var);
        ctx->opt = saved;
        return finish(rc);
      }
      if (best_fom > top) {
        top = best_fom;
        best_rr = thr;
      }
    }
    best_fom = top;
    rr_top = top;
    // 4. tally pixels (reading 28): the tile-stratified point-detector pixels change the noise as well as the
    //    speed, so tile shapes are compared with the tuned configuration by the same figure of merit; a tile
    //    shape is kept only if it beats it (n_batches x tile pixels must fit the shared tile image)
    const double untiled = top;
    const int shapes[2][2] = {{16, 16}, {32, 32}};
    for (int c = 0; c < 2; ++c) {
      const int tu = std::min(shapes[c][0], ctx->nu), tv = std::min(shapes[c][1], ctx->nv);
      if ((size_t)8 * tu * tv > (size_t)kSharedTallyMaxPixels) continue;
      mc_options trial = shape;
      trial.tally_mode = MC_TALLY_TILED;
      trial.tile_u = tu;
      trial.tile_v = tv;
      const mc_options keep = shape;
      shape = trial;
      rc = fom_of(best_rr, nullptr);
      shape = keep;
      if (rc) {
        cudaFree(d_var);
        ctx->opt = saved;
        return finish(rc);
      }
      if (best_fom > top) {
        top = best_fom;
        best_tu = tu;
        best_tv = tv;
      }
    }
    tile_gain = untiled > 0 ? top / untiled : 1.0;
    cudaFree(d_var);
  }
  ctx->opt = saved;
  ctx->opt.block_size = best.block_size;
  ctx->opt.blocks_per_sm = best.blocks_per_sm;
  ctx->opt.tally_mode = best.tally_mode;
  ctx->opt.rr_threshold = best_rr;
  if (best_tu > 0) {
    ctx->opt.tally_mode = MC_TALLY_TILED;
    ctx->opt.tile_u = best_tu;
    ctx->opt.tile_v = best_tv;
  }
  out->rr_threshold = best_rr;
  out->rr_fom_gain = fom0 > 0 ? rr_top / fom0 : 1.0;
  out->tile_u = best_tu;
  out->tile_v = best_tv;
  out->tile_fom_gain = tile_gain;
  out->step_mm = best_step;
  out->block_size = best.block_size;
  out->blocks_per_sm = best.blocks_per_sm;
  out->tally_mode = ctx->opt.tally_mode;  // the tile-stratified tally when step 4 kept a tile shape
  out->histories_per_s = best_rate;
  out->step_error = best_err;
  (void)max_per_sm;
  return finish(MC_OK);
}

// ---------------------------------------------------------------------------
// Correction plumbing
int mc_fdk(mc_ctx* ctx, const float* p, int n_proj, const float* angles, int NU, int NV, int nx, int ny, int nz,
           float dx, float dy, float dz, float* vol, void* stream) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!ctx->have_geometry) return fail(ctx, MC_ERR_STATE, "geometry not set");
  if (!p || !vol || !angles || n_proj < 1 || NU < 2 || NV < 2 || nx < 1 || ny < 1 || nz < 1 || !(dx > 0) ||
      !(dy > 0) || !(dz > 0) || NU > 50000)
    return fail(ctx, MC_ERR_INVALID_ARG, "bad reconstruction arguments");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)stream;
  const float pu = ctx->pu * (float)ctx->nu / (float)NU, pv = ctx->pv * (float)ctx->nv / (float)NV;
  std::vector<float> cs(2 * (size_t)n_proj);
  for (int k = 0; k < n_proj; ++k) {
    cs[k] = std::cos((double)angles[k]);
    cs[n_proj + k] = std::sin((double)angles[k]);
  }
  float *d_cs = nullptr, *q = nullptr;
  CK(cudaMalloc((void**)&d_cs, cs.size() * 4), "fdk allocation");
  cudaError_t e = cudaMalloc((void**)&q, (size_t)n_proj * NU * NV * 4);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_cs, cs.data(), cs.size() * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = recon_fdk(p, n_proj, d_cs, d_cs + n_proj, NU, NV, pu, pv, ctx->sod, ctx->sdd, nx, ny, nz, dx, dy, dz, q, vol, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(q);
  cudaFree(d_cs);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fdk");
  return MC_OK;
}

namespace {
// Total mass attenuation (cm^2/g) of every table material at energy E (linear between nodes).
std::vector<float> murho_at(const mc_ctx* ctx, double E) {
  const double x = (E - ctx->E0) / ctx->dE;
  const int i = std::max(0, std::min((int)std::floor(x), ctx->n_E - 2));
  const double f = x - i;
  std::vector<float> out(ctx->n_mat);
  for (int m = 0; m < ctx->n_mat; ++m) {
    auto tot = [&](int j) {
      const size_t q = (size_t)m * ctx->n_E + j;
      return ctx->pe[q] + ctx->in[q] + ctx->co[q];
    };
    out[m] = (float)(tot(i) + f * (tot(i + 1) - tot(i)));
  }
  return out;
}
}  // namespace

namespace {
// Class tables of the segmentation (Sec. II-E): the material of each class and,
// for classes k >= 1, the mass attenuation of that material at the effective
// energy (cm^2/g, linear between nodes); cmu[3] holds class 0's density.
void class_tables(const mc_ctx* ctx, int classes, const int* class_material, float class_density0, float e_eff,
                  int cm[3], float cmu[6]) {
  const std::vector<float> mr = murho_at(ctx, e_eff);
  for (int k = 0; k < 3; ++k) {
    cm[k] = k < classes ? class_material[k] : 0;
    cmu[k] = mr[cm[k]];
  }
  cmu[3] = class_density0;
  cmu[4] = cmu[5] = 0.f;
}

bool in_table(const mc_ctx* ctx, float E) { return E >= ctx->E0 && E <= ctx->E0 + ctx->dE * (ctx->n_E - 1); }
}  // namespace

int mc_line_integrals(mc_ctx* ctx, const float* I, const float* I0, int n_proj, int NU, int NV, float* a_out,
                      void* stream) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!I || !I0 || !a_out || n_proj < 1 || NU < 1 || NV < 1)
    return fail(ctx, MC_ERR_INVALID_ARG, "line integrals need device buffers and positive sizes");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  (void)cudaGetLastError();
  const size_t img = (size_t)NU * NV;
  const cudaError_t e = recon_log_norm(I, I0, img, img * n_proj, a_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "line integrals");
  return MC_OK;
}

int mc_segment(mc_ctx* ctx, const float* vol, int nx, int ny, int nz, int classes, const int* class_material,
               float class_density0, float e_eff_keV, float mu_lo, float mu_hi, uint32_t* hist_out,
               int* thresholds_out, uint8_t* mat_out, uint16_t* rho_out, void* stream) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!ctx->have_tables) return fail(ctx, MC_ERR_STATE, "tables not loaded");
  if (!vol || !mat_out || !rho_out || !class_material || nx < 1 || ny < 1 || nz < 1 ||
      (classes != 2 && classes != 3) || !(mu_hi > mu_lo) || !std::isfinite(mu_lo) || !std::isfinite(mu_hi) ||
      !in_table(ctx, e_eff_keV) || !(class_density0 >= 0.f) || !std::isfinite(class_density0))
    return fail(ctx, MC_ERR_INVALID_ARG, "bad segmentation arguments");
  for (int k = 0; k < classes; ++k)
    if (class_material[k] < 0 || class_material[k] >= ctx->n_mat)
      return fail(ctx, MC_ERR_INVALID_ARG, "class material outside the table");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)stream;
  int cm[3];
  float cmu[6];
  class_tables(ctx, classes, class_material, class_density0, e_eff_keV, cm, cmu);
  // device scratch: histogram [256], thresholds [2], class materials [3], class tables [6]
  unsigned char* d = nullptr;
  CK(cudaMallocAsync((void**)&d, 256 * 4 + 2 * 4 + 3 * 4 + 6 * 4, s), "segmentation scratch");
  unsigned int* hist = reinterpret_cast<unsigned int*>(d);
  int* thr = reinterpret_cast<int*>(d + 1024);
  int* d_cm = thr + 2;
  float* d_cmu = reinterpret_cast<float*>(d_cm + 3);
  cudaError_t e = cudaMemcpyAsync(d_cm, cm, sizeof(cm), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_cmu, cmu, sizeof(cmu), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = recon_otsu_segment(vol, (size_t)nx * ny * nz, mu_lo, mu_hi, classes, d_cm, d_cmu, d_cmu + 3, 30.f, hist, thr,
                           mat_out, rho_out, s);
  if (e == cudaSuccess && hist_out) e = cudaMemcpyAsync(hist_out, hist, 256 * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && thresholds_out) e = cudaMemcpyAsync(thresholds_out, thr, 2 * 4, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d, s);
  // the host class tables must outlive their copies; the read-backs must land
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "segmentation");
  return MC_OK;
}

int mc_correct_images(mc_ctx* ctx, const float* a, const float* ip, const float* is, float is_scale, size_t n,
                      float* c_out, void* stream) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!a || !ip || !is || !c_out || n < 1 || !(is_scale >= 0.f) || !std::isfinite(is_scale))
    return fail(ctx, MC_ERR_INVALID_ARG, "correction needs device buffers, n >= 1 and a finite is_scale >= 0");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  (void)cudaGetLastError();
  const cudaError_t e = recon_correct(a, ip, is, is_scale, n, c_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "correction");
  return MC_OK;
}

int mc_bin_volume(mc_ctx* ctx, const uint8_t* mat, const uint16_t* rho, int nx, int ny, int nz, float e_eff_keV,
                  uint8_t* mat_out, uint16_t* rho_out, void* stream) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!ctx->have_tables) return fail(ctx, MC_ERR_STATE, "tables not loaded");
  if (!mat || !rho || !mat_out || !rho_out || nx < 2 || ny < 2 || nz < 2 || nx % 2 || ny % 2 || nz % 2)
    return fail(ctx, MC_ERR_INVALID_ARG, "bin_volume needs even dimensions and device buffers");
  if (!(e_eff_keV >= ctx->E0) || !(e_eff_keV <= ctx->E0 + ctx->dE * (ctx->n_E - 1)))
    return fail(ctx, MC_ERR_INVALID_ARG, "energy outside the table");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  const std::vector<float> mr = murho_at(ctx, e_eff_keV);
  float* d = nullptr;
  CK(cudaMallocAsync((void**)&d, mr.size() * 4, s), "bin_volume table");
  cudaError_t e = cudaMemcpyAsync(d, mr.data(), mr.size() * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = recon_bin_volume(mat, rho, nx, ny, nz, d, ctx->n_mat, mat_out, rho_out, s);
  cudaFreeAsync(d, s);
  // the host table must outlive the copy
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "bin_volume");
  return MC_OK;
}

int mc_correct_iter(mc_ctx* ctx, const float* raw_I, const float* I0, int n_proj, const float* angles, int NU, int NV,
                    int n_iter, const mc_correct_params* prm, float* c_out, float* vol_out, double* iter_seconds,
                    void* stream) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!ctx->have_tables || !ctx->have_spectrum || !ctx->have_geometry)
    return fail(ctx, MC_ERR_STATE, "tables, spectrum and geometry are needed");
  if (!raw_I || !I0 || !angles || !prm || !c_out || n_proj < 2 || NU < 2 || NV < 2 || n_iter < 0)
    return fail(ctx, MC_ERR_INVALID_ARG, "bad correction arguments");
  const mc_correct_params& P = *prm;
  if (P.nx < 1 || P.ny < 1 || P.nz < 1 || !(P.dx > 0) || !(P.dy > 0) || !(P.dz > 0) || P.sim_nu < 1 || P.sim_nv < 1 ||
      P.sim_angle_stride < 1 || P.photons < 1 || !(P.step_mm > 0) || (P.classes != 2 && P.classes != 3) ||
      !(P.mu_hi > P.mu_lo) || !(P.e_eff_keV >= ctx->E0) || !(P.e_eff_keV <= ctx->E0 + ctx->dE * (ctx->n_E - 1)))
    return fail(ctx, MC_ERR_INVALID_ARG, "bad correction parameters");
  const bool binned = P.mc_bin == 2;
  if (P.mc_bin < 0 || P.mc_bin > 2 || (binned && (P.nx % 2 || P.ny % 2 || P.nz % 2)))
    return fail(ctx, MC_ERR_INVALID_ARG, "mc_bin must be 0, 1 or 2 (even volume dimensions)");
  for (int k = 0; k < P.classes; ++k)
    if (P.class_material[k] < 0 || P.class_material[k] >= ctx->n_mat)
      return fail(ctx, MC_ERR_INVALID_ARG, "class material outside the table");
  for (int k = 1; k < n_proj; ++k)
    if (!(angles[k] > angles[k - 1])) return fail(ctx, MC_ERR_INVALID_ARG, "angles must increase");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)stream;
  const size_t img = (size_t)NU * NV, nall = img * n_proj;
  const size_t nvox = (size_t)P.nx * P.ny * P.nz;
  const size_t simg = (size_t)P.sim_nu * P.sim_nv;
  std::vector<float> sim_angles;
  for (int k = 0; k < n_proj; k += P.sim_angle_stride) sim_angles.push_back(angles[k]);
  const int n_sim = (int)sim_angles.size();
  // buffers
  std::vector<void*> bufs;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    return p;
  };
  auto release = [&](int code) {
    cudaStreamSynchronize(s);
    for (void* p : bufs) cudaFree(p);
    return code;
  };
  float* a = (float*)alloc(nall * 4);
  float* c = (float*)alloc(nall * 4);
  float* ip = (float*)alloc(nall * 4);
  float* is = (float*)alloc(nall * 4);
  float* vol = (float*)alloc(nvox * 4);
  uint8_t* mat = (uint8_t*)alloc(nvox);
  uint16_t* rho = (uint16_t*)alloc(nvox * 2);
  float* ip_sim = (float*)alloc((size_t)n_proj * simg * 4);
  float* is_sim = (float*)alloc((size_t)n_sim * simg * 4);
  unsigned int* hist = (unsigned int*)alloc(256 * 4);
  int* thr = (int*)alloc(2 * 4 + 3 * 4 + 6 * 4);
  const size_t nbin = binned ? nvox / 8 : 1;
  uint8_t* mat_b = (uint8_t*)alloc(nbin);
  uint16_t* rho_b = (uint16_t*)alloc(nbin * 2);
  float* d_murho = (float*)alloc((size_t)ctx->n_mat * 4);
  if (bufs.size() != 14) return release(fail(ctx, MC_ERR_OOM, "correction buffers"));
  const std::vector<float> murho_eff = murho_at(ctx, P.e_eff_keV);
  int* d_cls_mat = thr + 2;
  float* d_cls_murho = reinterpret_cast<float*>(thr + 5);
  float* d_cls_rho0 = d_cls_murho + 3;
  {
    int cm[3];
    float cmu[6];
    class_tables(ctx, P.classes, P.class_material, P.class_density0, P.e_eff_keV, cm, cmu);
    cudaError_t e = cudaMemcpyAsync(d_cls_mat, cm, sizeof(cm), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_cls_murho, cmu, sizeof(cmu), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_murho, murho_eff.data(), murho_eff.size() * 4, cudaMemcpyHostToDevice, s);
    // the host tables are locals: their copies must complete before they go out of scope
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return release(cuda_fail(ctx, e, "class tables"));
  }
  // geometry of the simulation grid over the same panel
  const float sod = ctx->sod, sdd = ctx->sdd, pu = ctx->pu, pv = ctx->pv;
  const int nu0 = ctx->nu, nv0 = ctx->nv;
  const float PU = pu * (float)nu0 / (float)NU, PV = pv * (float)nv0 / (float)NV;
  const float spu = PU * (float)NU / (float)P.sim_nu, spv = PV * (float)NV / (float)P.sim_nv;
  auto restore = [&]() { mc_set_geometry(ctx, sod, sdd, nu0, nv0, pu, pv); };
  cudaError_t e = recon_log_norm(raw_I, I0, img, nall, a, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c, a, nall * 4, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return release(cuda_fail(ctx, e, "line integrals"));
  const int saved_mode = ctx->opt.denoise_mode;
  for (int it = 0; it < n_iter; ++it) {
    const auto t0 = std::chrono::steady_clock::now();
    int rc = mc_fdk(ctx, c, n_proj, angles, NU, NV, P.nx, P.ny, P.nz, P.dx, P.dy, P.dz, vol, stream);
    if (rc) return release(rc);
    e = recon_otsu_segment(vol, nvox, P.mu_lo, P.mu_hi, P.classes, d_cls_mat, d_cls_murho, d_cls_rho0, 30.f, hist, thr,
                           mat, rho, s);
    if (e != cudaSuccess) return release(cuda_fail(ctx, e, "segmentation"));
    rc = mc_load_volume(ctx, mat, rho, P.nx, P.ny, P.nz, P.dx, P.dy, P.dz, 1, stream);
    if (rc) return release(rc);
    if (P.primary_full_res) {
      rc = mc_set_geometry(ctx, sod, sdd, NU, NV, PU, PV);
      if (rc == MC_OK) rc = mc_project(ctx, angles, n_proj, 1, P.step_mm, P.seed, ip, nullptr, nullptr, stream);
      if (rc) {
        restore();
        return release(rc);
      }
    }
    if (binned) {
      // the Monte Carlo step runs on the volume down-sampled by 2 per axis (Sec. II-C.2, II-E)
      e = recon_bin_volume(mat, rho, P.nx, P.ny, P.nz, d_murho, ctx->n_mat, mat_b, rho_b, s);
      if (e != cudaSuccess) return release(cuda_fail(ctx, e, "down-sampling"));
      rc = mc_load_volume(ctx, mat_b, rho_b, P.nx / 2, P.ny / 2, P.nz / 2, 2.f * P.dx, 2.f * P.dy, 2.f * P.dz, 1,
                          stream);
      if (rc) return release(rc);
    }
    rc = mc_set_geometry(ctx, sod, sdd, P.sim_nu, P.sim_nv, spu, spv);
    if (rc) return release(rc);
    if (!P.primary_full_res) rc = mc_project(ctx, angles, n_proj, 1, P.step_mm, P.seed, ip_sim, nullptr, nullptr, stream);
    if (rc == MC_OK)
      rc = mc_project(ctx, sim_angles.data(), n_sim, P.photons, P.step_mm, P.seed + 7919ull * (it + 1), nullptr,
                      is_sim, nullptr, stream);
    restore();
    if (rc && rc != MC_ERR_LIMIT) return release(rc);
    rc = mc_smooth_upsample(ctx, is_sim, n_sim, sim_angles.data(), P.sim_nu, P.sim_nv, is, n_proj, angles, NU, NV, stream);
    if (rc == MC_OK && !P.primary_full_res) {
      ctx->opt.denoise_mode = 2;  // the primary is noise free: interpolate only
      rc = mc_smooth_upsample(ctx, ip_sim, n_proj, angles, P.sim_nu, P.sim_nv, ip, n_proj, angles, NU, NV, stream);
      ctx->opt.denoise_mode = saved_mode;
    }
    if (rc) return release(rc);
    // per-pixel images scale with the pixel area: the scatter simulated on the
    // coarse grid is converted to the panel's pixels when the primary was
    // computed there (with the paper's up-sampled primary the factor cancels)
    const float area = P.primary_full_res ? (PU * PV) / (spu * spv) : 1.f;
    e = recon_correct(a, ip, is, area, nall, c, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return release(cuda_fail(ctx, e, "correction"));
    if (iter_seconds) iter_seconds[it] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  e = cudaMemcpyAsync(c_out, c, nall * 4, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return release(cuda_fail(ctx, e, "output"));
  if (vol_out) {
    const int rc = mc_fdk(ctx, c, n_proj, angles, NU, NV, P.nx, P.ny, P.nz, P.dx, P.dy, P.dz, vol_out, stream);
    if (rc) return release(rc);
  }
  return release(MC_OK);
}

// ---------------------------------------------------------------------------
// Learned denoiser
int mc_denoise_init(mc_ctx* ctx, int height, int width, int max_batch, uint64_t seed) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (height < 16 || width < 16 || height % 16 || width % 16 || max_batch < 1 || max_batch > 4096)
    return fail(ctx, MC_ERR_INVALID_ARG, "denoiser images must be multiples of 16 (>= 16) and 1 <= batch <= 4096");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  denoiser_destroy(ctx->denoiser);
  ctx->denoiser = nullptr;
  CK(denoiser_create(height, width, max_batch, seed, &ctx->denoiser), "denoiser creation");
  return MC_OK;
}

int mc_denoise_train_step(mc_ctx* ctx, const float* noisy, const float* clean, int n, float lr, float* loss_out,
                          void* stream) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!ctx->denoiser) return fail(ctx, MC_ERR_STATE, "denoiser not initialised");
  if (!noisy || !clean || !loss_out || !(lr >= 0.f)) return fail(ctx, MC_ERR_INVALID_ARG, "bad training arguments");
  int H, W, B;
  denoiser_size(ctx->denoiser, &H, &W, &B);
  if (n < 1 || n > B) return fail(ctx, MC_ERR_INVALID_ARG, "batch outside 1..max_batch");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  (void)cudaGetLastError();
  int err = 0;
  CK(denoiser_train_step(ctx->denoiser, noisy, clean, n, lr, loss_out, &err, (cudaStream_t)stream), "training step");
  if (err) return fail(ctx, MC_ERR_TIMEOUT, "a tensor-core wait gave up");
  return MC_OK;
}

int mc_denoise_infer(mc_ctx* ctx, const float* in, float* out, int n, void* stream) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!ctx->denoiser) return fail(ctx, MC_ERR_STATE, "denoiser not initialised");
  if (!in || !out || n < 1) return fail(ctx, MC_ERR_INVALID_ARG, "bad inference arguments");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  (void)cudaGetLastError();
  CK(denoiser_infer(ctx->denoiser, in, out, n, (cudaStream_t)stream), "inference");
  CK(cudaStreamSynchronize((cudaStream_t)stream), "inference");
  return MC_OK;
}

int mc_denoise_get_layer(mc_ctx* ctx, int layer, float* w, float* b, float* gw, float* gb, int* cin, int* cout) {
  if (!ctx || !cin || !cout) return MC_ERR_INVALID_ARG;
  if (!ctx->denoiser) return fail(ctx, MC_ERR_STATE, "denoiser not initialised");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  CK(cudaDeviceSynchronize(), "synchronize");
  if (!denoiser_get_layer(ctx->denoiser, layer, w, b, gw, gb, cin, cout))
    return fail(ctx, MC_ERR_INVALID_ARG, "layer index out of range");
  return MC_OK;
}

int mc_denoise_set_layer(mc_ctx* ctx, int layer, const float* w, const float* b) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!ctx->denoiser) return fail(ctx, MC_ERR_STATE, "denoiser not initialised");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (!denoiser_set_layer(ctx->denoiser, layer, w, b)) return fail(ctx, MC_ERR_INVALID_ARG, "bad layer or copy");
  return MC_OK;
}

int mc_denoise_save(mc_ctx* ctx, const char* path) {
  if (!ctx || !path) return MC_ERR_INVALID_ARG;
  if (!ctx->denoiser) return fail(ctx, MC_ERR_STATE, "denoiser not initialised");
  int H, W, B;
  const int nl = denoiser_size(ctx->denoiser, &H, &W, &B);
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(ctx, MC_ERR_IO, std::string("cannot write ") + path);
  const int32_t hdr[4] = {1, H, W, nl};
  bool ok = std::fwrite("MCXDEN01", 1, 8, f) == 8 && std::fwrite(hdr, 4, 4, f) == 4;
  for (int i = 0; i < nl && ok; ++i) {
    int ci = 0, co = 0;
    denoiser_get_layer(ctx->denoiser, i, nullptr, nullptr, nullptr, nullptr, &ci, &co);
    std::vector<float> w((size_t)co * 9 * ci), b(co);
    denoiser_get_layer(ctx->denoiser, i, w.data(), b.data(), nullptr, nullptr, &ci, &co);
    const int32_t dims[2] = {ci, co};
    ok = std::fwrite(dims, 4, 2, f) == 2 && std::fwrite(w.data(), 4, w.size(), f) == w.size() &&
         std::fwrite(b.data(), 4, b.size(), f) == b.size();
  }
  ok = (std::fclose(f) == 0) && ok;
  return ok ? MC_OK : fail(ctx, MC_ERR_IO, "write failed");
}

int mc_denoise_load(mc_ctx* ctx, const char* path, int max_batch) {
  if (!ctx || !path) return MC_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(ctx, MC_ERR_IO, std::string("cannot open ") + path);
  char magic[8];
  int32_t hdr[4];
  if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, "MCXDEN01", 8) || std::fread(hdr, 4, 4, f) != 4 ||
      hdr[0] != 1 || hdr[3] != denoiser_layer_count()) {
    std::fclose(f);
    return fail(ctx, MC_ERR_IO, "not a denoiser checkpoint");
  }
  int rc = mc_denoise_init(ctx, hdr[1], hdr[2], max_batch > 0 ? max_batch : 16, 0);
  if (rc) {
    std::fclose(f);
    return rc;
  }
  for (int i = 0; i < hdr[3]; ++i) {
    int ci = 0, co = 0;
    denoiser_get_layer(ctx->denoiser, i, nullptr, nullptr, nullptr, nullptr, &ci, &co);
    int32_t dims[2];
    std::vector<float> w((size_t)co * 9 * ci), b(co);
    if (std::fread(dims, 4, 2, f) != 2 || dims[0] != ci || dims[1] != co || std::fread(w.data(), 4, w.size(), f) != w.size() ||
        std::fread(b.data(), 4, b.size(), f) != b.size()) {
      std::fclose(f);
      return fail(ctx, MC_ERR_IO, "truncated or mismatched denoiser checkpoint");
    }
    denoiser_set_layer(ctx->denoiser, i, w.data(), b.data());
  }
  std::fclose(f);
  return MC_OK;
}

int mc_nn_conv3x3(const void* x, const void* w, const float* bias, void* y, int n, int h, int wd, int cin, int cout,
                  int relu, int out_f32, int* err, void* stream) {
  if (!x || !w || !y || !err || n < 1 || h < 1 || wd < 1 || cin < 16 || cin % 16 || cout < 16 || cout % 16 || cout > 256)
    return MC_ERR_INVALID_ARG;
  if ((uintptr_t)x & 15) return MC_ERR_INVALID_ARG;
  (void)cudaGetLastError();
  const cudaStream_t st = (cudaStream_t)stream;
  // the kernel reads the weights in tensor-core operand order: repack them
  // into a stream-ordered temporary
  __nv_bfloat16* wm = nullptr;
  if (cudaMallocAsync((void**)&wm, (size_t)cout * 9 * cin * 2, st) != cudaSuccess) return MC_ERR_OOM;
  cudaError_t e = nn::pack_weights_bf16((const __nv_bfloat16*)w, cout, cin, wm, st);
  if (e == cudaSuccess) {
    ConvParams p;
    p.x = (const __nv_bfloat16*)x;
    p.wt = wm;
    p.bias = bias;
    p.y = y;
    p.n = n; p.h = h; p.w = wd; p.cin = cin; p.cout = cout;
    p.co_total = cout; p.co0 = 0;
    p.relu = relu; p.out_f32 = out_f32;
    p.err = err;
    e = launch_conv3x3_fwd(p, st);
  }
  const cudaError_t ef = cudaFreeAsync(wm, st);
  if (e == cudaSuccess) e = ef;
  return e == cudaSuccess ? MC_OK : (e == cudaErrorInvalidValue ? MC_ERR_INVALID_ARG : MC_ERR_CUDA);
}

int mc_nn_conv3x3_wgrad(const void* x, const void* dy, float* dw, int n, int h, int wd, int cin, int cout, int splits,
                        int* err, void* stream) {
  if (!x || !dy || !dw || !err || n < 1 || h < 1 || wd < 1 || cin < 16 || cin % 16 || cout < 16 || cout % 16 ||
      cout > 256 || splits < 1 || splits > 65535)
    return MC_ERR_INVALID_ARG;
  WgradParams p;
  p.x = (const __nv_bfloat16*)x;
  p.dy = (const __nv_bfloat16*)dy;
  p.dw = dw;
  p.n = n; p.h = h; p.w = wd; p.cin = cin; p.cout = cout;
  p.err = err;
  (void)cudaGetLastError();
  const cudaError_t e = launch_conv3x3_wgrad(p, splits, (cudaStream_t)stream);
  return e == cudaSuccess ? MC_OK : MC_ERR_CUDA;
}

int mc_last_stats(const mc_ctx* ctx, double* out, int n) {
  if (!ctx || !out || n < 0 || n > MC_STAT_N) return MC_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) out[i] = ctx->stats[i];
  return MC_OK;
}

int mc_smooth_upsample(mc_ctx* ctx, const float* in, int n_in, const float* in_angles, int nu, int nv, float* out,
                       int n_out, const float* out_angles, int NU, int NV, void* stream) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  if (!in || !out || !in_angles || !out_angles || n_in < 1 || n_out < 1 || nu < 1 || nv < 1 || NU < 1 || NV < 1)
    return fail(ctx, MC_ERR_INVALID_ARG, "bad smooth_upsample arguments");
  const int win = ctx->opt.sg_window, ord = ctx->opt.sg_order;
  const bool smooth = ctx->opt.denoise_mode == 0;  // 1: learned denoiser, 2: none
  if (smooth && (nu < win || nv < win)) return fail(ctx, MC_ERR_INVALID_ARG, "image smaller than the smoothing window");
  const double two_pi = 6.283185307179586;
  for (int i = 0; i < n_in; ++i) {
    if (!std::isfinite(in_angles[i])) return fail(ctx, MC_ERR_INVALID_ARG, "angles must be finite");
    if (i > 0 && !(in_angles[i] > in_angles[i - 1])) return fail(ctx, MC_ERR_INVALID_ARG, "in_angles must increase");
  }
  if (n_in > 1 && !((double)in_angles[n_in - 1] - in_angles[0] < two_pi))
    return fail(ctx, MC_ERR_INVALID_ARG, "in_angles must span less than 2 pi");
  // bracketing simulated angles for each requested angle (periodic in 2 pi)
  std::vector<int> a0(n_out), a1(n_out);
  std::vector<float> fa(n_out);
  for (int o = 0; o < n_out; ++o) {
    if (!std::isfinite(out_angles[o])) return fail(ctx, MC_ERR_INVALID_ARG, "angles must be finite");
    if (n_in == 1) {
      a0[o] = a1[o] = 0;
      fa[o] = 0.f;
      continue;
    }
    double th = std::fmod((double)out_angles[o] - in_angles[0], two_pi);
    if (th < 0) th += two_pi;
    int k = n_in - 1;
    for (int i = 0; i + 1 < n_in; ++i)
      if (th < (double)in_angles[i + 1] - in_angles[0]) {
        k = i;
        break;
      }
    const double lo = (double)in_angles[k] - in_angles[0];
    const double hi = (k + 1 < n_in) ? (double)in_angles[k + 1] - in_angles[0] : two_pi;
    a0[o] = k;
    a1[o] = (k + 1) % n_in;
    fa[o] = (float)((th - lo) / (hi - lo));
  }
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nimg = (size_t)n_in * nu * nv;
  const size_t meta = (size_t)win * win + 3 * (size_t)n_out + 64;
  CK(ensure(ctx->d_post, ctx->post_cap, 2 * nimg + meta), "post-processing allocation");
  float* t0 = ctx->d_post;
  float* t1 = t0 + nimg;
  float* coef = t1 + nimg;
  int* d_a0 = reinterpret_cast<int*>(coef + win * win);
  int* d_a1 = d_a0 + n_out;
  float* d_fa = reinterpret_cast<float*>(d_a1 + n_out);
  std::vector<float> H;
  sg_hat(win, ord, H);
  std::vector<unsigned char> hostmeta((size_t)win * win * 4 + (size_t)n_out * 12);
  std::memcpy(hostmeta.data(), H.data(), (size_t)win * win * 4);
  std::memcpy(hostmeta.data() + (size_t)win * win * 4, a0.data(), (size_t)n_out * 4);
  std::memcpy(hostmeta.data() + (size_t)win * win * 4 + (size_t)n_out * 4, a1.data(), (size_t)n_out * 4);
  std::memcpy(hostmeta.data() + (size_t)win * win * 4 + (size_t)n_out * 8, fa.data(), (size_t)n_out * 4);
  CK(cudaMemcpyAsync(coef, hostmeta.data(), hostmeta.size(), cudaMemcpyHostToDevice, s), "coefficient upload");
  const float* src = in;
  if (smooth) {
    CK(launch_sg_rows(in, t0, n_in, nv, nu, coef, win, s), "smoothing launch");
    CK(launch_sg_cols(t0, t1, n_in, nv, nu, coef, win, s), "smoothing launch");
    src = t1;
  } else if (ctx->opt.denoise_mode == 1) {
    int dh = 0, dw = 0, db = 0;
    if (!ctx->denoiser) return fail(ctx, MC_ERR_STATE, "denoise_mode 1 needs mc_denoise_init or mc_denoise_load");
    denoiser_size(ctx->denoiser, &dh, &dw, &db);
    if (dh != nv || dw != nu) return fail(ctx, MC_ERR_INVALID_ARG, "image size differs from the denoiser's");
    CK(denoiser_infer(ctx->denoiser, in, t1, n_in, s), "denoiser inference");
    src = t1;
  }
  CK(launch_lerp_upsample(src, nv, nu, out, n_out, NV, NU, d_a0, d_a1, d_fa, ctx->opt.cubic_a, s), "upsample launch");
  CK(cudaStreamSynchronize(s), "stream synchronize");
  return MC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Read-only accessors for the static-scratch entry point (k_static.cu).  None
// of them allocates device or host heap memory: results go to caller buffers.
namespace mcx {

int static_check(mc_ctx* ctx, int* device, int* nu, int* nv) {
  const int rc = check_ready(ctx);
  if (rc) return rc;
  if (ctx->mesh_mode) return fail(ctx, MC_ERR_STATE, "the static-scratch entry point serves the voxel volume only");
  *device = ctx->device;
  *nu = ctx->nu;
  *nv = ctx->nv;
  return MC_OK;
}

int static_fail(mc_ctx* ctx, int code, const char* msg) { return fail(ctx, code, msg); }

int static_cuda_fail(mc_ctx* ctx, cudaError_t e, const char* where) { return cuda_fail(ctx, e, where); }

// FP32 shared-memory table blob for the nodes the spectrum reaches, written
// into dst (capacity cap bytes); same layout as the context's own blob.
int static_build_blob(mc_ctx* ctx, unsigned char* dst, int cap, int* bytes_out, int* n_stage_out) {
  const int ns = stage_nodes(ctx);
  const int bytes = tab_blob_bytes(ctx->n_mat, ns);
  if (bytes > cap) return fail(ctx, MC_ERR_INVALID_ARG, "the staged cross-section tables exceed MC_STATIC_MAX_TABLE_BYTES (65536): fewer materials or a spectrum "
                                        "reaching lower energies");
  write_blob(ctx, ns, dst);
  *bytes_out = bytes;
  *n_stage_out = ns;
  return MC_OK;
}

// Stratified counts (as in the main path) written as prefix sums, energies,
// S_n / M_n and S_n into caller arrays of MC_MAX_BINS (+1) entries.
int static_stratify(mc_ctx* ctx, uint64_t N, unsigned long long* pre, float* en, float* wb, float* sn, int* n_out) {
  const int n = (int)ctx->S.size();
  uint64_t M[MC_MAX_BINS];
  int elig[MC_MAX_BINS];
  double fr[MC_MAX_BINS];
  uint64_t sum = 0;
  for (int i = 0; i < n; ++i) {
    const double x = (double)N * ctx->S[i];
    const double fl = std::floor(x);
    elig[i] = 0;
    fr[i] = 0.0;
    if (ctx->S[i] <= 0) M[i] = 0;
    else if (fl < 1.0) M[i] = 1;
    else {
      M[i] = (uint64_t)fl;
      elig[i] = 1;
      fr[i] = x - fl;
    }
    sum += M[i];
  }
  if (sum > N) return fail(ctx, MC_ERR_INVALID_ARG, "n_photons is smaller than the number of non-empty energy bins");
  uint64_t rem = N - sum;
  while (rem > 0) {
    int best = -1;
    for (int i = 0; i < n; ++i)
      if (elig[i] == 1 && (best < 0 || fr[i] > fr[best])) best = i;
    if (best < 0) break;
    M[best] += 1;
    elig[best] = 2;
    --rem;
  }
  if (rem) return fail(ctx, MC_ERR_INTERNAL, "stratification did not place every photon");
  pre[0] = 0;
  for (int i = 0; i < n; ++i) {
    pre[i + 1] = pre[i] + M[i];
    en[i] = ctx->Ebin[i];
    wb[i] = M[i] ? (float)(ctx->S[i] / (double)M[i]) : 0.f;
    sn[i] = (float)ctx->S[i];
  }
  *n_out = n;
  return MC_OK;
}

void static_views(mc_ctx* ctx, TableView* t, VolumeView* v, GeomView* g, mc_options* opt, int* sm_count) {
  *t = table_view(ctx);
  *v = volume_view(ctx);
  *g = geom_view(ctx);
  *opt = ctx->opt;
  *sm_count = ctx->sm_count;
}

void static_set_stats(mc_ctx* ctx, const unsigned long long* st, float ms) {
  const int map[10] = {S_HIST, S_FLIGHT_STEPS, S_NEE_STEPS, S_NEE_RAYS, S_PHOTO, S_COMPTON, S_RAYLEIGH, S_ESCAPE, S_LIMIT, S_SAMPLER_FAIL};
  for (int i = 0; i < 10; ++i) ctx->stats[i] = (double)st[map[i]];
  ctx->stats[10] = ms;
  ctx->stats[11] = 0;
}

}  // namespace mcx
