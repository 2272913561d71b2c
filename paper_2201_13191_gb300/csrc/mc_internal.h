// Internal interfaces of the GB300 library: parameter blocks passed by value to
// the kernels and the launch wrappers each translation unit exports to the API.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/mc.h"

namespace mcx {

constexpr int kMaxMat = MC_MAX_MATERIALS;
constexpr int kMaxComp = 8;
constexpr int kTabKinds = 6;  // tot, pe, incoh, coh, I_coh, I_incoh (bound model; zero otherwise)
enum TabKind { TAB_TOT = 0, TAB_PE = 1, TAB_IN = 2, TAB_CO = 3, TAB_ICOH = 4, TAB_IINC = 5 };

// Statistic slots (uint64 counters on the device, doubles at the ABI).
enum Stat {
  S_HIST = 0, S_FLIGHT_STEPS, S_NEE_STEPS, S_NEE_RAYS, S_PHOTO, S_COMPTON, S_RAYLEIGH, S_ESCAPE,
  S_LIMIT, S_SAMPLER_FAIL, S_INTERNAL,
  S_WORK,  // chunk counter of the tile-stratified tally (blocks take work from it)
  S_BAD_SMEM,  // blocks that found less dynamic shared memory than their layout needs (and did nothing)
  S_NSTAT
};

// Staged table blob (device global, copied per block into shared memory):
//   float2 tab[kTabKinds][n_mat][n_stage]   (v_i, v_{i+1} - v_i)
//   float2 jkn[n_stage]                      Klein-Nishina normalisation J(E)
//   float2 eta[n_stage]                      detector response
//   float2 comp[n_mat][kMaxComp]             (w Z^2, b) of the form factor
//   float  compz[n_mat][kMaxComp]            w Z (electrons, for the scattering function)
//   int    ncomp[n_mat] (padded to 16 bytes)
struct TableView {
  const float2* blob;  // device
  int n_mat;
  int n_stage;         // nodes staged (prefix of the file's nodes)
  int blob_bytes;      // multiple of 16
  float E0, inv_dE, dE;
  float mec2, inv_hc;
  int use_eta;         // the blob's detector-response row replaces eta(E) = E
  int bound;           // incoherent scattering with the scattering function S(x, Z)
};

// Voxel word: bits 0-15 the FP16 density (g/cm^3), bits 16-23 the material id.
// Layout LIN: x fastest.  Layout BRICK: 4x4x4 bricks (x fastest between
// bricks), Morton order inside a brick, so each 32-byte sector holds a 2x2x2
// cube and each 128-byte line a 4x4x2 slab whatever the ray direction.
enum VoxLayout { VOX_LIN = 0, VOX_BRICK = 1 };
// Transport geometry selector beside the two voxel layouts: closed triangle-
// mesh bodies (MeshView below) with exact flights instead of the march.
constexpr int GEO_MESH = 2;

// The packed volume carries a one-voxel border that repeats the edge voxels
// (padded dims px = nx + 2, ...), so a midpoint that rounding puts a hair
// outside the box reads the edge voxel, exactly as clamping would, and the
// march needs no per-axis clamps.
struct VolumeView {
  const uint32_t* vox;
  int layout;
  int nbx, nby;    // bricks along x, y (BRICK layout, padded dims)
  int px, py, pz;  // padded dims
  int words;       // words in the packed array (last index + 1)
  int pxy;         // px * py
  int lin_bias;    // 0x4B000000 (1 + px + px py) mod 2^32: folds the round-down floors' offsets into the index
  int nx, ny, nz;
  float dx, dy, dz;
  float inv_dx, inv_dy, inv_dz;
  float hx, hy, hz;  // half extents (mm)
};

struct GeomView {
  float sod, sdd, pu, pv;
  int nu, nv;
};

struct SpectrumView {
  const unsigned long long* prefix;  // [n_bins + 1] stratified history prefix sums
  const float* energy;               // [n_bins]
  const float* wbin;                 // [n_bins] S_n / M_n
  const float* sn;                   // [n_bins] S_n
  const float* eta;                  // [n_bins] detector response at each bin energy (primary)
  int n_bins;
};

// Triangle-mesh geometry (k_mesh.cu): BVH nodes as float4 pairs (lo.xyz + first,
// hi.xyz + count; count 0 = inner node with children first, first + 1),
// triangles as three float4 (xyz; the first's w carries the body id), bodies as
// int4 (material, parent or -1, parent material, density bits).
struct MeshView {
  const float4* nodes;
  const float4* tris;
  const int4* bodies;
  const float* body_rho;
  int n_nodes, n_tris, n_bodies;
};
struct TransportParams {
  TableView tab;
  VolumeView vol;
  GeomView geo;
  SpectrumView spec;
  const float* angles;  // device [n_angles]
  int n_angles;
  unsigned long long n_photons, h_begin, h_count;
  float step;
  unsigned long long seed;
  int n_split;
  int nee_mode;  // 0: sampled type's pdf; 1: expected value over the type (both terms, one march)
  int doppler;   // Doppler broadening of incoherent scatter (bound tables)
  int forced;    // forced detection: one pseudo-particle per pixel (of the panel or the history's tile)
  float rr_threshold;
  int max_order;
  int n_batches;
  double* tally;                 // [n_batches][n_angles][nv][nu]
  unsigned long long* stats;     // [S_NSTAT]
  int tally_mode = 0;            // TALLY_* below
  // when set, the Philox key is read from device memory at kernel start (a
  // captured graph then serves every seed); otherwise `seed` is used
  const unsigned long long* seed_dev = nullptr;
  // triangle-mesh geometry (geometry == GEO_MESH); `vol` then carries only the
  // half extents of a box around the bodies (hx, hy, hz)
  int geometry = 0;  // VOX_LIN / VOX_BRICK from vol.layout, or GEO_MESH
  MeshView mesh = {};
  // TALLY_TILED: tiles of tile_u x tile_v pixels, n_tu across, n_tiles in all;
  // work in chunks of up to tile_chunk histories of one (angle, tile), tile_k
  // chunks per (angle, tile), n_chunks in all, handed out by stats[S_WORK]
  int tile_u = 0, tile_v = 0, n_tu = 0, n_tiles = 0;
  unsigned long long tile_chunk = 0, tile_k = 0, n_chunks = 0;
};

// How pseudo-particle scores reach the FP64 image (eq. Is):
//   TALLY_GLOBAL  one FP64 atomic add per pseudo-particle;
//   TALLY_WARP    lanes of a warp that hit the same pixel first combine
//                 their scores (match + shuffle), one atomic per pixel group;
//   TALLY_SHARED  a per-block FP32 image in shared memory (warp-combined adds),
//                 flushed into the FP64 image once at the end of the block.
//   TALLY_TILED   tile-stratified point-detector pixels: history h aims at tile
//                 (h + o) mod T only (o uniform per run and angle, weight T); a
//                 block works through chunks of one (angle, tile) and tallies the
//                 tile in shared memory (warp-combined adds), flushing it into the
//                 FP64 image after each chunk.
enum TallyMode { TALLY_GLOBAL = 0, TALLY_WARP = 1, TALLY_SHARED = 2, TALLY_TILED = 3 };
constexpr int kSharedTallyMaxPixels = 12288;  // 48 KB of FP32 per block

struct PrimaryParams {
  TableView tab;
  VolumeView vol;
  GeomView geo;
  SpectrumView spec;
  const float* angles;
  int n_angles;
  float step;
  float* out;  // [n_angles][nv][nu]
  int shared_acc = 0;  // per-material totals in shared memory (volumes with frequent material changes)
};

// launch wrappers (return cudaError_t of the launch)
cudaError_t launch_transport(const TransportParams& p, int grid, int block, cudaStream_t s);
int transport_smem_bytes(const TableView& t, int n_bins, int block, int shared_pixels = 0);
// FP32 pixels of the shared tally image the kernel keeps for these parameters
int transport_shared_pixels(const TransportParams& p);
cudaError_t transport_occupancy(int block, int smem, int* blocks_per_sm, bool mesh = false, int layout = VOX_LIN);
cudaError_t launch_finalize(const double* tally, int n_batches, size_t n, float* out, float* var, cudaStream_t s);
cudaError_t launch_primary(const PrimaryParams& p, cudaStream_t s);
// Fraction of x-neighbour voxel pairs of a device material array whose materials differ (synchronises s).
cudaError_t material_change_fraction(const uint8_t* mat, int nx, int ny, int nz, cudaStream_t s, double* frac);

// Returns the depth of the deepest leaf (the device descent needs depth < 64).
int build_mesh_bvh(const float* v, const int* tris, const int* tri_body, int nt, std::vector<float4>& nodes,
                   std::vector<float4>& out_tris);
cudaError_t launch_primary_mesh(const PrimaryParams& p, const MeshView& m, cudaStream_t s);
// Checks a device-resident volume (ids < n_mat, finite non-negative binary16
// densities); *bad_host = 1 if any voxel fails.  Synchronises s.
cudaError_t validate_volume_device(const uint8_t* mat, const uint16_t* rho, size_t n, int n_mat, cudaStream_t s,
                                   int* bad_host);
// Packs material + density into voxel words in the given layout.
cudaError_t pack_volume(const uint8_t* mat, const uint16_t* rho, int nx, int ny, int nz, int layout, uint32_t* out,
                        size_t out_words, cudaStream_t s);
size_t packed_words(int nx, int ny, int nz, int layout);
// Padded dimensions, brick counts and word count of a packed volume.
void padded_dims(int nx, int ny, int nz, int layout, VolumeView* v);

// post-processing
cudaError_t launch_sg_rows(const float* in, float* out, int n_img, int h, int w, const float* coef, int win,
                           cudaStream_t s);
cudaError_t launch_sg_cols(const float* in, float* out, int n_img, int h, int w, const float* coef, int win,
                           cudaStream_t s);
cudaError_t launch_lerp_upsample(const float* in, int nv, int nu, float* out, int n_out, int NV, int NU,
                                 const int* a0, const int* a1, const float* fa, float cubic_a, cudaStream_t s);

// ---------------------------------------------------------------------------
// Denoiser convolutions (k_conv.cu): NHWC BF16, channels multiples of 16.
struct ConvParams {
  const __nv_bfloat16* x;   // [n][h][w][cin], 16-byte aligned
  const __nv_bfloat16* wt;  // packed [cin/8][9][co_total][8], tap = 3 * (dy + 1) + (dx + 1)
  const float* bias;        // [cout] or null
  void* y;                  // [n][h][w][cout], BF16 or FP32
  int n, h, w, cin, cout;   // cout: output channels of this launch, rows co0 .. co0 + cout of wt
  int co_total, co0;
  int relu, out_f32;
  int* err;                 // set to 1 if a bounded wait gave up
};
struct WgradParams {
  const __nv_bfloat16* x;   // [n][h][w][cin] layer input
  const __nv_bfloat16* dy;  // [n][h][w][cout] gradient at the layer output (pre-activation)
  float* dw;                // [cout][9 * cin] FP32, accumulated (zero it first)
  int n, h, w, cin, cout;
  int* err;
};
cudaError_t launch_conv3x3_fwd(const ConvParams& p, cudaStream_t s);
cudaError_t launch_conv3x3_wgrad(const WgradParams& p, int splits, cudaStream_t s);

// Correction plumbing (k_recon.cu)
cudaError_t recon_log_norm(const float* I, const float* I0, size_t img, size_t n, float* a, cudaStream_t s);
cudaError_t recon_fdk(const float* p, int n_proj, const float* d_cos, const float* d_sin, int nu, int nv, float pu,
                      float pv, float sod, float sdd, int nx, int ny, int nz, float dx, float dy, float dz, float* q_tmp,
                      float* vol, cudaStream_t s);
cudaError_t recon_otsu_segment(const float* vol, size_t n, float lo, float hi, int classes, const int* d_cls_mat,
                               const float* d_cls_murho, const float* d_cls_rho0, float rho_max, unsigned int* d_hist,
                               int* d_thr, uint8_t* mat, uint16_t* rho, cudaStream_t s);
// 2x2x2 down-sampling of a segmented volume (even dims): largest-mass material, attenuation-conserving density
// at the effective energy (murho: device [n_mat] mass attenuation there).
cudaError_t recon_bin_volume(const uint8_t* mat, const uint16_t* rho, int nx, int ny, int nz, const float* murho,
                             int n_mat, uint8_t* mat_b, uint16_t* rho_b, cudaStream_t s);
// c = a - ln(ip / (ip + is_scale * is)): is_scale converts the scatter image's
// per-pixel values to the panel's pixel area when it was simulated on another grid.
cudaError_t recon_correct(const float* a, const float* ip, const float* is, float is_scale, size_t n, float* c,
                          cudaStream_t s);

// Learned denoiser (denoiser.cu)
struct Denoiser;
cudaError_t denoiser_create(int H, int W, int B, unsigned long long seed, Denoiser** out);
void denoiser_destroy(Denoiser* d);
cudaError_t denoiser_infer(Denoiser* d, const float* img, float* out, int n, cudaStream_t s);
cudaError_t denoiser_train_step(Denoiser* d, const float* noisy, const float* clean, int n, float lr, float* loss_out,
                                int* err_out, cudaStream_t s);
int denoiser_size(const Denoiser* d, int* H, int* W, int* B);
bool denoiser_get_layer(const Denoiser* d, int i, float* w, float* b, float* gw, float* gb, int* cin, int* cout);
bool denoiser_set_layer(Denoiser* d, int i, const float* w, const float* b);
int denoiser_layer_count();

}  // namespace mcx
