// Scatter projection that allocates nothing: the transport and finalize kernels
// run with all their scratch (FP64 tally image, counters, staged tables,
// spectrum block and angles) in one file-scope __device__ array instead of
// buffers obtained from cudaMalloc.
//
// Some callers cannot allocate device memory once they are running: services
// that reserve the whole GPU at start-up for a fixed memory pool (a new
// cudaMalloc then fails or waits on the other streams), and real-time
// acquisition loops that must not pay for cudaMalloc's implicit device
// synchronisation on every projection.  They load tables, volume, spectrum
// and geometry once at start-up and then call mc_project_scatter_static.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "mc_device.cuh"
#include "mc_internal.h"

namespace mcx {

int static_check(mc_ctx* ctx, int* device, int* nu, int* nv);
int static_fail(mc_ctx* ctx, int code, const char* msg);
int static_cuda_fail(mc_ctx* ctx, cudaError_t e, const char* where);
int static_build_blob(mc_ctx* ctx, unsigned char* dst, int cap, int* bytes_out, int* n_stage_out);
int static_stratify(mc_ctx* ctx, uint64_t N, unsigned long long* pre, float* en, float* wb, float* sn, int* n_out);
void static_views(mc_ctx* ctx, TableView* t, VolumeView* v, GeomView* g, mc_options* opt, int* sm_count);
void static_set_stats(mc_ctx* ctx, const unsigned long long* st, float ms);

namespace {

// Layout of the static scratch (byte offsets, each a multiple of 256).
constexpr size_t kOffTally = 0;
constexpr size_t kTallyBytes = (size_t)MC_STATIC_MAX_TALLY * 8;
constexpr size_t kOffStats = kOffTally + kTallyBytes;
constexpr size_t kStatsBytes = 256;
constexpr size_t kOffBlob = kOffStats + kStatsBytes;
constexpr size_t kBlobBytes = MC_STATIC_MAX_TABLE_BYTES;
constexpr size_t kOffSpec = kOffBlob + kBlobBytes;
constexpr size_t kSpecBytes = ((size_t)(MC_MAX_BINS + 1) * 8 + (size_t)MC_MAX_BINS * 12 + 255) / 256 * 256;
constexpr size_t kOffAngles = kOffSpec + kSpecBytes;
constexpr size_t kAnglesBytes = (size_t)MC_STATIC_MAX_ANGLES * 4;
constexpr size_t kScratchBytes = kOffAngles + kAnglesBytes;

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Each CUDA context loads its own copy of this module, so the array's device
// address belongs to a context, not to a device number: the address is looked
// up (cudaGetSymbolAddress, which allocates nothing) the first time a call runs
// in a context and kept under that context's unique id.  Ids are never reused
// within a process, so a context created after cudaDeviceReset, or a second
// context on the same device, gets its own lookup.
constexpr int kMaxContexts = 64;
struct AddrEntry {
  unsigned long long ctx_id;
  unsigned char* addr;
};
AddrEntry g_addr[kMaxContexts] = {};
int g_addr_n = 0;
std::mutex g_addr_mutex;

typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

// Unique id of the CUDA context current on this thread (driver entry points
// fetched through the runtime, so the library needs no link to libcuda).
cudaError_t current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess)
      return cudaErrorNotSupported;
    get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  void* ctx = nullptr;
  if (get_current(&ctx) != 0 || ctx == nullptr) return cudaErrorDeviceUninitialized;
  if (get_id(ctx, id) != 0) return cudaErrorDeviceUninitialized;
  return cudaSuccess;
}

// Device address of g_scratch in the context current on this thread (the
// caller has made the context's device current with cudaSetDevice).
cudaError_t scratch_address(unsigned char** out) {
  unsigned long long id = 0;
  cudaError_t e = current_context_id(&id);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  for (int i = 0; i < g_addr_n; ++i)
    if (g_addr[i].ctx_id == id) {
      *out = g_addr[i].addr;
      return cudaSuccess;
    }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return e;
  // a full table reuses a slot; the context that held it looks its address up again on its next call
  const int slot = g_addr_n < kMaxContexts ? g_addr_n++ : (int)(id % kMaxContexts);
  g_addr[slot].ctx_id = id;
  g_addr[slot].addr = static_cast<unsigned char*>(p);
  *out = g_addr[slot].addr;
  return cudaSuccess;
}

}  // namespace
}  // namespace mcx

using namespace mcx;

extern "C" int mc_project_scatter_static(mc_ctx* ctx, const float* angles_rad, int n_angles, uint64_t n_photons,
                                         float step_mm, uint64_t seed, float* scatter_out, void* stream) {
  if (!ctx) return MC_ERR_INVALID_ARG;
  int device = 0, nu = 0, nv = 0;
  int rc = static_check(ctx, &device, &nu, &nv);
  if (rc) return rc;
  if (!scatter_out) return static_fail(ctx, MC_ERR_INVALID_ARG, "scatter_out is required");
  if (!angles_rad || n_angles < 1) return static_fail(ctx, MC_ERR_INVALID_ARG, "n_angles must be >= 1");
  if (n_angles > MC_STATIC_MAX_ANGLES)
    return static_fail(ctx, MC_ERR_INVALID_ARG, "n_angles exceeds MC_STATIC_MAX_ANGLES (4096)");
  const size_t img = (size_t)nu * nv;
  if (img * (size_t)n_angles > (size_t)MC_STATIC_MAX_TALLY)
    return static_fail(ctx, MC_ERR_INVALID_ARG,
                       "n_angles x nu x nv exceeds the static tally of MC_STATIC_MAX_TALLY (4194304) pixels");
  if (!(step_mm > 0.f) || !std::isfinite(step_mm)) return static_fail(ctx, MC_ERR_INVALID_ARG, "step_mm must be > 0");
  if (n_photons < 1) return static_fail(ctx, MC_ERR_INVALID_ARG, "n_photons must be >= 1");
  for (int i = 0; i < n_angles; ++i)
    if (!std::isfinite(angles_rad[i])) return static_fail(ctx, MC_ERR_INVALID_ARG, "angles must be finite");

  TableView tv;
  VolumeView vv;
  GeomView gv;
  mc_options opt;
  int sm_count = 0;
  static_views(ctx, &tv, &vv, &gv, &opt, &sm_count);
  if (opt.doppler && !tv.bound)
    return static_fail(ctx, MC_ERR_STATE, "Doppler broadening needs the bound-electron tables (version 2)");
  {
    const double diag = std::sqrt((double)vv.nx * vv.dx * vv.nx * vv.dx + (double)vv.ny * vv.dy * vv.ny * vv.dy +
                                  (double)vv.nz * vv.dz * vv.nz * vv.dz);
    if (diag / step_mm > 4.0e6)
      return static_fail(ctx, MC_ERR_INVALID_ARG, "step_mm too small: more than 4e6 steps per chord");
  }

  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return static_cuda_fail(ctx, e, "cudaSetDevice");
  unsigned char* base = nullptr;
  e = scratch_address(&base);
  if (e != cudaSuccess) return static_cuda_fail(ctx, e, "cudaGetSymbolAddress of the static scratch");
  cudaStream_t s = (cudaStream_t)stream;

  // host staging on the stack: tables, spectrum block
  unsigned char blob[kBlobBytes];
  int blob_bytes = 0, n_stage = 0;
  rc = static_build_blob(ctx, blob, (int)kBlobBytes, &blob_bytes, &n_stage);
  if (rc) return rc;
  unsigned char spec[kSpecBytes];
  int nb = 0;
  auto* pre = reinterpret_cast<unsigned long long*>(spec);
  float* en = reinterpret_cast<float*>(spec + (size_t)(MC_MAX_BINS + 1) * 8);
  float* wb = en + MC_MAX_BINS;
  float* sn = wb + MC_MAX_BINS;
  rc = static_stratify(ctx, n_photons, pre, en, wb, sn, &nb);
  if (rc) return rc;

  double* tally = reinterpret_cast<double*>(base + kOffTally);
  unsigned long long* stats = reinterpret_cast<unsigned long long*>(base + kOffStats);
  float* angles = reinterpret_cast<float*>(base + kOffAngles);
  const size_t n_img = img * n_angles;
  // everything the kernels read or accumulate is (re)written here: calls share the array
  e = cudaMemcpyAsync(base + kOffBlob, blob, blob_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + kOffSpec, spec, kSpecBytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(angles, angles_rad, (size_t)n_angles * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(tally, 0, n_img * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(stats, 0, S_NSTAT * 8, s);
  if (e != cudaSuccess) return static_cuda_fail(ctx, e, "static scratch staging");

  tv.blob = reinterpret_cast<const float2*>(base + kOffBlob);
  tv.n_stage = n_stage;
  tv.blob_bytes = blob_bytes;
  SpectrumView sv;
  sv.prefix = reinterpret_cast<const unsigned long long*>(base + kOffSpec);
  sv.energy = reinterpret_cast<const float*>(base + kOffSpec + (size_t)(MC_MAX_BINS + 1) * 8);
  sv.wbin = sv.energy + MC_MAX_BINS;
  sv.sn = sv.wbin + MC_MAX_BINS;
  sv.n_bins = nb;

  TransportParams tp;
  tp.tab = tv;
  tp.vol = vv;
  tp.geo = gv;
  tp.spec = sv;
  tp.angles = angles;
  tp.n_angles = n_angles;
  tp.n_photons = n_photons;
  tp.h_begin = 0;
  tp.h_count = n_photons;
  tp.step = step_mm;
  tp.seed = seed;
  tp.n_split = opt.n_split;
  tp.nee_mode = opt.nee_mode;
  tp.doppler = opt.doppler;
  tp.forced = opt.forced_detection;
  if (tp.forced && img > (size_t)MC_FORCED_MAX_PIXELS)
    return static_fail(ctx, MC_ERR_INVALID_ARG, "forced_detection needs at most MC_FORCED_MAX_PIXELS (65536) pixels");
  tp.rr_threshold = opt.rr_threshold;
  tp.max_order = opt.max_scatter_order;
  tp.n_batches = 1;
  tp.tally = tally;
  tp.stats = stats;
  tp.tally_mode = TALLY_GLOBAL;
  const int block = opt.block_size ? opt.block_size : 256;
  const int smem = transport_smem_bytes(tv, nb, block);
  int per_sm = opt.blocks_per_sm;
  if (per_sm == 0) {
    e = transport_occupancy(block, smem, &per_sm, false, vv.layout);
    if (e != cudaSuccess) return static_cuda_fail(ctx, e, "occupancy query");
    per_sm = per_sm > 0 ? per_sm : 1;
  }
  const unsigned long long work = (unsigned long long)n_angles * n_photons;
  const unsigned long long need = (work + block - 1) / block;
  const unsigned long long cap = (unsigned long long)sm_count * per_sm;
  const int grid = (int)(need < cap ? (need > 0 ? need : 1) : cap);
  e = launch_transport(tp, grid, block, s);
  if (e == cudaSuccess) e = launch_finalize(tally, 1, n_img, scatter_out, nullptr, s);
  if (e != cudaSuccess) return static_cuda_fail(ctx, e, "static transport launch");
  unsigned long long st[S_NSTAT] = {};
  e = cudaMemcpyAsync(st, stats, S_NSTAT * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return static_cuda_fail(ctx, e, "static transport");
  static_set_stats(ctx, st, 0.f);
  if (st[S_INTERNAL]) return static_fail(ctx, MC_ERR_TIMEOUT, "a block gave up waiting for its table copy");
  if (st[S_BAD_SMEM]) return static_fail(ctx, MC_ERR_INTERNAL, "transport launched with less shared memory than its layout");
  if (st[S_LIMIT] || st[S_SAMPLER_FAIL])
    return static_fail(ctx, MC_ERR_LIMIT, "histories hit the scatter-order or sampler cap (outputs valid)");
  return MC_OK;
}
