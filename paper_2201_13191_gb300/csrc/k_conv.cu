// 3x3 convolutions of the learned scatter denoiser on the tcgen05 tensor cores.
//
// Tensors are NHWC, BF16, with channel counts that are multiples of 16.
//  - forward: implicit GEMM over shifted views of a halo tile fetched by the
//    tensor memory accelerator (description at k_conv3x3_fwd); FP32
//    accumulators in tensor memory; epilogue bias, optional ReLU, BF16 or FP32.
//  - input gradient: the same kernel with the adjoint weights (flipped in space,
//    transposed in channels: a 3x3 'same' convolution's adjoint).
//  - weight gradient: dW[co][k] = sum_p dY[p][co] Xcol[p][k]; the tile is 128
//    rows of k by N = C_out, the reduction over pixels runs in stages of 64
//    pixels staged transposed into the K-major layout; CTAs split the pixels and
//    add their FP32 partial tiles into dW.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>

#include "mc_internal.h"
#include "mc_tc.cuh"

namespace mcx {
namespace {

constexpr int kM = 128;        // pixels (forward) or K rows (weight gradient) per CTA
constexpr int kStageK = 64;    // reduction elements per stage
constexpr int kKG = kStageK / 8;
constexpr int kThreads = 128;  // four warps: one per 32 tensor-memory lanes

// Weight-gradient operand tiles: the K-major no-swizzle canonical layout (core
// matrices of 8 rows x 16 bytes) with padded strides, core matrices kLbo bytes
// apart along K and 8-row groups kSbo apart, so that eight lanes storing the
// same row of eight different core matrices hit eight different 16-byte bank
// slots (the unpadded 128 / 1024-byte strides put them all on one).
constexpr int kLbo = 128 + 16;
constexpr int kSbo = kKG * kLbo + 16;
template <int N>
struct ConvSmem {
  static constexpr int a_bytes = (kM / 8) * kSbo;
  static constexpr int b_bytes = (N / 8) * kSbo;
  static constexpr int stage_bytes = a_bytes + b_bytes;
  static constexpr int bytes = 2 * stage_bytes + 1024;  // + alignment slack
};
__device__ __forceinline__ uint32_t wg_off(int row, int k) {
  return (uint32_t)((row >> 3) * kSbo + (k >> 3) * kLbo + (row & 7) * 16 + (k & 7) * 2);
}

// ---------------------------------------------------------------------------
// Forward (and input-gradient) convolution.
//
// Tiling.  The image is cut into column strips of width ws = min(w, MC_CONV_WS); a
// strip with its one-pixel border (the neighbouring strips' columns, or zeros
// at the image edge) and a zero row above and below is the "padded strip", of
// width wp = ws + 2, linearised row-major.  A CTA computes A x 128 consecutive
// positions q of one padded strip (A accumulators of 128 rows x N output
// channels in tensor memory); positions on the border are computed and
// discarded.  For tap (dy, dx) the input of position q sits at q + dy*wp + dx,
// so with the input tile ("halo": the rows of the padded strip that cover
// [q0 - wp - 1, q0 + 128A + wp]) stored position-major -- one row of CC
// channels (2 CC bytes, swizzled 32/64/128B) per position, the canonical
// K-major swizzled layout -- every tap's A operand is the same tile seen from
// a start address shifted by (dy*wp + dx) rows.  Each input chunk is fetched
// once per CTA instead of nine times, by one tiled 4-D tensor copy per stage
// (zero-filled outside the image).
//
// Pipeline.  The reduction runs over the input channels in chunks of CC; a
// chunk's stage holds its halo and its weights for all nine taps (the packed
// operand order wm[ci/8][tap][co][ci%8] makes that one contiguous block).
// Warp 0 lane 0 fills a ring of `stages` stages (mbarrier `full`), warp 1
// lane 0 issues the MMAs (9 taps x CC/16 k-steps x A accumulators per stage)
// and frees each stage with tcgen05.commit (mbarrier `empty`); after the last
// stage all four warps read their accumulator rows (tensor-memory lanes) and
// store bias + optional ReLU, BF16 or FP32.
// ---------------------------------------------------------------------------
constexpr int kMaxStages = 8;
constexpr int kSmemBudget = 225 * 1024;  // the most one CTA may take
// Shared memory the planner lets one forward CTA take: the whole budget (one
// CTA per SM, the deepest ring) or less, so that several CTAs share an SM and
// one's pipeline fill and epilogue overlap another's MMAs.
#ifndef MC_CONV_PLAN_KB
#define MC_CONV_PLAN_KB 110
#endif
constexpr int kPlanBudget = MC_CONV_PLAN_KB * 1024;
// Output-channel tiles narrower than C_out when the grid would not cover the
// SMs (1), or always C_out rounded up (0).
#ifndef MC_CONV_SPLIT_N
#define MC_CONV_SPLIT_N 1
#endif
// Widest strip (columns) the forward tiles cut an image into: narrower strips
// cut the halo rows a tile fetches (measured 301.6 / 307.9 / 312.3 TFLOP/s
// FLOP-weighted at 128 / 64 / 32 over the denoiser's layers).
#ifndef MC_CONV_WS
#define MC_CONV_WS 32
#endif

struct FwdArgs {
  const __nv_bfloat16* wm;  // packed weights [cin/8][9][co_total][8]
  const float* bias;        // [cout] or null
  void* y;                  // [n][h][w][cout]
  int n, h, w, cin, cout, co_total, co0;
  int ws, strips, wp, tiles;  // strip width, strips per row, padded width, tiles per strip
  int A, CC, stages, rbox;    // accumulators, channels per stage, ring depth, halo rows per copy
  uint32_t halo_bytes, stage_bytes;
  int rb;                     // halo bytes per position row (2 CC), swizzled in 8-row groups
  int relu, out_f32;
  int* err;
};

__device__ __forceinline__ uint32_t tmem_cols(int n) {
  uint32_t c = 32;
  while (c < (uint32_t)n) c <<= 1;
  return c;
}

// Tap folding (FOLD, for C_out tiles with 3N <= 256).  The three taps of one
// kernel row (dy, dx = -1, 0, +1) share one MMA: the A operand is the halo seen
// from the row shift dy*wp - 1 alone and B holds the three taps' weights side by
// side (N_mma = 3N, contiguous in the packed [tap][co] order), so accumulator
// row r collects, in column block dx, the contributions that output position
// r - 1 - dx ... needs; the epilogue adds block -1 of row r, block 0 of row
// r + 1 and block +1 of row r + 2.  That is 3 instead of 9 MMAs per k-step,
// each three times wider (narrow-N MMAs are bound by their A operand reads),
// and 126 instead of 128 output positions per accumulator.
#ifndef MC_CONV_FOLD
#define MC_CONV_FOLD 1
#endif
constexpr int kFoldRows = 126;

template <int N, bool FOLD>
__global__ void __launch_bounds__(kThreads, 1) k_conv3x3_fwd(const __grid_constant__ CUtensorMap xmap, const FwdArgs a) {
  extern __shared__ unsigned char dyn_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)dyn_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], done;
  __shared__ uint32_t tmem_holder;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  int tile = blockIdx.x;
  const int t = tile % a.tiles;
  tile /= a.tiles;
  const int strip = tile % a.strips;
  const int img = tile / a.strips;
  const int nb = blockIdx.y * N;  // first output channel of this CTA (within the launch's cout)
  constexpr int NA = FOLD ? 3 * N : N;         // accumulator columns
  constexpr int RA = FOLD ? kFoldRows : 128;   // output positions per accumulator
  const int Mt = RA * a.A;
  const int q0 = a.wp + 1 + t * Mt;           // first position: row 1, column 1 of the padded strip
  const int vr_lo = (q0 - a.wp - 1) / a.wp;   // first halo row (padded-strip row index)
  const int o0 = q0 - vr_lo * a.wp;           // halo index of q0
  const int n_chunks = a.cin / a.CC;
  const uint32_t ncols = tmem_cols(a.A * NA);

  if (warp == 0) tc::tmem_alloc(&tmem_holder, ncols);
  if (tid == 0) {
    for (int i = 0; i < a.stages; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(&done, 1);
    abort_flag = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer: halo by tensor copies, weights by one bulk copy per chunk
      const int rows = min(N, a.cout - nb);  // weight rows this CTA needs
      const int r0 = a.co0 + nb;
      const bool one_block = rows == N && N == a.co_total;
      const uint32_t w_tx = (uint32_t)(a.CC / 8) * 9u * (uint32_t)rows * 16u;
      const uint32_t halo_tx = (uint32_t)(a.CC / 8) * 16u * (uint32_t)a.wp * (uint32_t)a.rbox;
      int issued = 0;
      for (int st = 0; st < n_chunks; ++st) {
        const int slot = st % a.stages;
        if (st >= a.stages && !tc::mbar_wait(&empty[slot], (uint32_t)((st / a.stages) - 1) & 1u)) {
          abort_flag = 1;
          break;
        }
        if (abort_flag) break;
        unsigned char* hs = sm + (size_t)slot * a.stage_bytes;
        unsigned char* wsm = hs + a.halo_bytes;
        tc::mbar_expect_tx(&full[slot], halo_tx + w_tx);
        const int g0 = st * (a.CC / 8);  // first 8-channel group of the chunk
        tc::tma_load_4d(hs, &xmap, &full[slot], g0 * 8, strip * a.ws - 1, vr_lo - 1, img);
        if (one_block) {
          tc::bulk_load(wsm, a.wm + (size_t)g0 * 9 * a.co_total * 8, w_tx, &full[slot]);
        } else {
          for (int kc = 0; kc < a.CC / 8; ++kc)
            for (int tap = 0; tap < 9; ++tap)
              tc::bulk_load(wsm + (size_t)((kc * 9 + tap) * N) * 16,
                            a.wm + ((size_t)((g0 + kc) * 9 + tap) * a.co_total + r0) * 8, (uint32_t)rows * 16u,
                            &full[slot]);
        }
        ++issued;
      }
      if (abort_flag) {
        // let the copies still in flight land before the CTA can exit
        for (int st = max(0, issued - a.stages); st < issued; ++st)
          tc::mbar_wait(&full[st % a.stages], (uint32_t)(st / a.stages) & 1u);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      const uint32_t idesc = tc::idesc_bf16(128, NA);
      const uint32_t lbo_b = 9u * N * 16u;
      constexpr int kGroups = FOLD ? 3 : 9;  // MMAs per k-step and accumulator: kernel rows or taps
      for (int st = 0; st < n_chunks; ++st) {
        const int slot = st % a.stages;
        if (!tc::mbar_wait(&full[slot], (uint32_t)(st / a.stages) & 1u)) {
          abort_flag = 1;
          break;
        }
        tc::fence_after();
        const uint32_t hb = tc::saddr(sm + (size_t)slot * a.stage_bytes);
        const uint32_t wb = hb + a.halo_bytes;
        for (int g = 0; g < kGroups; ++g) {
          // first tap of the group and the row shift of its A operand
          const int tap = FOLD ? 3 * g : g;
          const int shift = FOLD ? (g - 1) * a.wp - 1 : (tap / 3 - 1) * a.wp + (tap % 3 - 1);
          for (int ks = 0; ks < a.CC / 16; ++ks) {
            const uint64_t db = tc::sdesc(wb + (uint32_t)((2 * ks * 9 + tap) * N) * 16u, lbo_b, 128);
            for (int acc = 0; acc < a.A; ++acc) {
              // rows of 2 CC bytes, 8-row groups 8 rb apart; k-step = 32 bytes within the row.  The
              // tensor core applies the swizzle on absolute shared-memory address bits, like the TMA
              // that wrote the tile, so a start shifted by any number of rows needs no phase field.
              const uint32_t sa = hb + (uint32_t)(o0 + RA * acc + shift) * (uint32_t)a.rb + (uint32_t)ks * 32u;
              const uint64_t da = tc::sdesc_swz(sa, 8u * (uint32_t)a.rb, a.rb);
              tc::mma_bf16(tmem + (uint32_t)(acc * NA), da, db, idesc, (st | g | ks) ? 1u : 0u);
            }
          }
        }
        tc::commit(&empty[slot]);
      }
      tc::commit(&done);
    }
    __syncwarp();
  }
  bool ok = tc::mbar_wait(&done, 0);
  tc::fence_after();
  // one decision for the whole CTA: the folded epilogue synchronises its threads
  ok = __syncthreads_and(ok && !abort_flag) != 0;
  if (!ok && tid == 0) atomicOr(a.err, 1);
  if (ok) {
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    // exchange rows of the folded epilogue: the ring is idle once `done` has completed
    constexpr int kX = 20;  // floats per row (16 used; 80-byte rows keep float4 reads conflict-free)
    float* xch = reinterpret_cast<float*>(sm);
    for (int acc = 0; acc < a.A; ++acc) {
      const int q = q0 + RA * acc + tid;
      const int vr = q / a.wp, vc = q - vr * a.wp;
      const int y = vr - 1, x = strip * a.ws + vc - 1;
      const bool valid = (!FOLD || tid < kFoldRows) && vr >= 1 && vr <= a.h && vc >= 1 && vc <= a.ws && x < a.w;
      const long long pix = ((long long)img * a.h + y) * a.w + x;
#pragma unroll 1
      for (int c0 = 0; c0 < N; c0 += 8) {
        float v[8];
        tc::tmem_ld8(lane_base + (uint32_t)(acc * NA + c0), v);
        if (FOLD) {
          float v0[8], vp[8];
          tc::tmem_ld8(lane_base + (uint32_t)(acc * NA + N + c0), v0);
          tc::tmem_ld8(lane_base + (uint32_t)(acc * NA + 2 * N + c0), vp);
          __syncthreads();  // the previous chunk's reads of xch are done
          float4* mine = reinterpret_cast<float4*>(xch + tid * kX);
          mine[0] = make_float4(v0[0], v0[1], v0[2], v0[3]);
          mine[1] = make_float4(v0[4], v0[5], v0[6], v0[7]);
          mine[2] = make_float4(vp[0], vp[1], vp[2], vp[3]);
          mine[3] = make_float4(vp[4], vp[5], vp[6], vp[7]);
          __syncthreads();
          if (tid < kFoldRows) {
            const float4* r1 = reinterpret_cast<const float4*>(xch + (tid + 1) * kX);
            const float4* r2 = reinterpret_cast<const float4*>(xch + (tid + 2) * kX);
            const float4 a0 = r1[0], a1 = r1[1], b0 = r2[2], b1 = r2[3];
            v[0] += a0.x + b0.x; v[1] += a0.y + b0.y; v[2] += a0.z + b0.z; v[3] += a0.w + b0.w;
            v[4] += a1.x + b1.x; v[5] += a1.y + b1.y; v[6] += a1.z + b1.z; v[7] += a1.w + b1.w;
          }
        }
        const int co = nb + c0;
        if (valid && co < a.cout) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            if (a.bias) v[j] += __ldg(a.bias + co + j);
            if (a.relu) v[j] = fmaxf(v[j], 0.f);
          }
          if (a.out_f32) {
            float* dst = reinterpret_cast<float*>(a.y) + pix * a.cout + co;
            *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<float4*>(dst + 4) = make_float4(v[4], v[5], v[6], v[7]);
          } else {
            __nv_bfloat162 b[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
            *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.y) + pix * a.cout + co) =
                *reinterpret_cast<uint4*>(b);
          }
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, ncols);
}

// Weight gradient.  CTA (blockIdx.x = k tile, blockIdx.y = pixel split).
// Transpose of an 8 x 8 block of 16-bit values held as 8 rows of 16 bytes:
// out[i] word m = (v[2m] element i, v[2m+1] element i).
__device__ __forceinline__ void transpose8x8(const uint4 (&v)[8], uint4 (&o)[8]) {
#pragma unroll
  for (int pr = 0; pr < 4; ++pr) {
    uint32_t lo[4], hi[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const uint32_t a = pr == 0 ? v[2 * m].x : pr == 1 ? v[2 * m].y : pr == 2 ? v[2 * m].z : v[2 * m].w;
      const uint32_t b = pr == 0 ? v[2 * m + 1].x : pr == 1 ? v[2 * m + 1].y : pr == 2 ? v[2 * m + 1].z : v[2 * m + 1].w;
      lo[m] = __byte_perm(a, b, 0x5410);  // element 2 pr of both rows
      hi[m] = __byte_perm(a, b, 0x7632);  // element 2 pr + 1 of both rows
    }
    o[2 * pr] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    o[2 * pr + 1] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  }
}

// Weight gradient dW[co][k] = sum_q dY[q][co] X(q shifted by tap(k))[c(k)],
// k = tap * C_in + c.  GEMM rows = 128 values of k (blockIdx.x), columns =
// C_out (N), reduction over the pixels [pbeg, pend) of this CTA (blockIdx.y of
// `splits`), 64 pixels per stage.  Both operands are K-major (pixels along K)
// while the tensors are channel-minor, so each thread turns one 8 x 8 block
// (8 pixels x 8 channels, eight 16-byte loads) into one core matrix (8 rows of
// 8 pixels) by a register transpose and one 16-byte store per row.  A stage's
// loads go out before the previous stage's MMAs are waited on (two buffers,
// one mbarrier each); thread 0 issues the MMAs.  The partial tile is added
// into dW (FP32 atomics).
template <int N>
__global__ void __launch_bounds__(kThreads) k_conv3x3_wgrad(const WgradParams p) {
  extern __shared__ unsigned char dyn_raw[];
  unsigned char* dyn = reinterpret_cast<unsigned char*>(((uintptr_t)dyn_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_holder;
  __shared__ __align__(8) uint64_t mbar[2];
  constexpr int kBUnits = (N / 8) * (kStageK / 8);          // 8 x 8 blocks of the dY operand per stage
  constexpr int kBPer = (kBUnits + kThreads - 1) / kThreads;  // per thread
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = 9 * p.cin;
  const int krow0 = blockIdx.x * kM;
  const long long npix = (long long)p.n * p.h * p.w;
  const long long chunk = (npix + gridDim.y - 1) / gridDim.y;
  const long long pbeg = (long long)blockIdx.y * chunk;
  const long long pend = min(npix, pbeg + chunk);
  const int n_stages = pend > pbeg ? (int)((pend - pbeg + kStageK - 1) / kStageK) : 0;

  // this thread's A block: rows rg*8 .. rg*8+7 (one tap, channels c .. c+7), pixels pg*8 .. pg*8+7
  const int rg = tid & 15, pg = tid >> 4;
  const int k_a = krow0 + rg * 8;
  const int tap = k_a / p.cin, c_a = k_a - tap * p.cin;
  const int ddy = tap / 3 - 1, ddx = tap % 3 - 1;
  const bool row_ok = k_a < K;

  auto load_a = [&](int st, uint4 (&v)[8]) {
    const long long qs = pbeg + (long long)st * kStageK + pg * 8;
    long long t = qs / p.w;
    int qx = (int)(qs - t * p.w);
    int qy = (int)(t % p.h);
    long long qn = t / p.h;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      v[jj] = make_uint4(0u, 0u, 0u, 0u);
      const int yy = qy + ddy, xx = qx + ddx;
      if (row_ok && qs + jj < pend && yy >= 0 && yy < p.h && xx >= 0 && xx < p.w)
        v[jj] = __ldg(reinterpret_cast<const uint4*>(p.x + ((qn * p.h + yy) * p.w + xx) * p.cin + c_a));
      if (++qx == p.w) {
        qx = 0;
        if (++qy == p.h) {
          qy = 0;
          ++qn;
        }
      }
    }
  };
  auto load_b = [&](int st, int u, uint4 (&v)[8]) {
    const int cg = u % (N / 8), bp = u / (N / 8);
    const long long qs = pbeg + (long long)st * kStageK + bp * 8;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      v[jj] = make_uint4(0u, 0u, 0u, 0u);
      if (qs + jj < pend && cg * 8 < p.cout)
        v[jj] = __ldg(reinterpret_cast<const uint4*>(p.dy + (qs + jj) * p.cout + cg * 8));
    }
  };

  if (warp == 0) tc::tmem_alloc(&tmem_holder, tmem_cols(N));
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_holder;
  bool ok = true;
  uint4 ra[8], rb[kBPer][8];
  if (n_stages > 0) {
    load_a(0, ra);
#pragma unroll
    for (int i = 0; i < kBPer; ++i)
      if (tid + i * kThreads < kBUnits) load_b(0, tid + i * kThreads, rb[i]);
  }
  for (int st = 0; st < n_stages; ++st) {
    const int buf = st & 1;
    unsigned char* sA = dyn + buf * ConvSmem<N>::stage_bytes;
    unsigned char* sB = sA + ConvSmem<N>::a_bytes;
    if (st >= 2) ok &= tc::mbar_wait(&mbar[buf], (uint32_t)((st >> 1) - 1) & 1u);
    {
      uint4 o[8];
      transpose8x8(ra, o);
#pragma unroll
      for (int i = 0; i < 8; ++i)
        *reinterpret_cast<uint4*>(sA + wg_off(rg * 8 + i, pg * 8)) = o[i];
    }
#pragma unroll
    for (int i = 0; i < kBPer; ++i) {
      const int u = tid + i * kThreads;
      if (u < kBUnits) {
        const int cg = u % (N / 8), bp = u / (N / 8);
        uint4 o[8];
        transpose8x8(rb[i], o);
#pragma unroll
        for (int r = 0; r < 8; ++r) *reinterpret_cast<uint4*>(sB + wg_off(cg * 8 + r, bp * 8)) = o[r];
      }
    }
    // the next stage's loads overlap the barrier and this stage's MMAs
    if (st + 1 < n_stages) {
      load_a(st + 1, ra);
#pragma unroll
      for (int i = 0; i < kBPer; ++i)
        if (tid + i * kThreads < kBUnits) load_b(st + 1, tid + i * kThreads, rb[i]);
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t idesc = tc::idesc_bf16(kM, N);
      for (int ks = 0; ks < kStageK / 16; ++ks) {
        // k-step ks covers core-matrix columns 2 ks, 2 ks + 1
        const uint64_t da = tc::sdesc(tc::saddr(sA) + ks * 2 * kLbo, kLbo, kSbo);
        const uint64_t db = tc::sdesc(tc::saddr(sB) + ks * 2 * kLbo, kLbo, kSbo);
        tc::mma_bf16(tmem, da, db, idesc, (st > 0 || ks > 0) ? 1u : 0u);
      }
      tc::commit(&mbar[buf]);
    }
  }
  if (n_stages > 0) {
    const int last = n_stages - 1;
    ok &= tc::mbar_wait(&mbar[last & 1], (uint32_t)(last >> 1) & 1u);
    if (n_stages > 1) ok &= tc::mbar_wait(&mbar[(last - 1) & 1], (uint32_t)((last - 1) >> 1) & 1u);
  }
  tc::fence_after();
  if (!ok && tid == 0) atomicOr(p.err, 1);
  if (ok && n_stages > 0) {
    const int k = krow0 + warp * 32 + lane;  // this lane's accumulator row
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 8) {
      float v[8];
      tc::tmem_ld8(lane_base + (uint32_t)c0, v);
      if (k < K)
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (c0 + j < p.cout) atomicAdd(p.dw + (long long)(c0 + j) * K + k, v[j]);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, tmem_cols(N));
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  });
  return fn;
}

// Tiling of one launch.  For each accumulator count A (A x N tensor-memory
// columns <= 512): the channel chunk CC and ring depth that fit shared memory
// (prefer >= 3 stages or every chunk resident, then larger chunks); then the A
// with the smallest estimated time, waves x (positions per CTA + halo rows +
// a fixed per-CTA cost), waves counted with the CTAs that fit on one SM.
// Shared memory of one stage's halo: swizzled rows of 2 CC bytes per position,
// one 1024-byte-aligned region.
uint32_t halo_bytes_for(int CC, int rbox, int wp) {
  return ((uint32_t)rbox * (uint32_t)wp * (uint32_t)(2 * CC) + 1023u) & ~1023u;
}

bool plan_fwd_budget(const ConvParams& p, int N, bool fold, int sms, int budget, FwdArgs& a, int& grid_x,
                     int& grid_y, int& smem);

// The plan within the planning budget, or within the whole budget when no tile fits the smaller one.
bool plan_fwd(const ConvParams& p, int N, bool fold, int sms, FwdArgs& a, int& grid_x, int& grid_y, int& smem) {
  return plan_fwd_budget(p, N, fold, sms, kPlanBudget, a, grid_x, grid_y, smem) ||
         plan_fwd_budget(p, N, fold, sms, kSmemBudget, a, grid_x, grid_y, smem);
}

int tmem_cols_host(int n) {
  int c = 32;
  while (c < n) c <<= 1;
  return c;
}

bool plan_fwd_budget(const ConvParams& p, int N, bool fold, int sms, int budget, FwdArgs& a, int& grid_x,
                     int& grid_y, int& smem) {
  a.ws = p.w < MC_CONV_WS ? p.w : MC_CONV_WS;
  a.strips = (p.w + a.ws - 1) / a.ws;
  a.wp = a.ws + 2;
  grid_y = (p.cout + N - 1) / N;
  const int NA = fold ? 3 * N : N;             // accumulator columns
  const int RA = fold ? kFoldRows : 128;       // output positions per accumulator
  const int min_bytes = 128 * 20 * 4 + 1024;   // the folded epilogue's exchange rows
  double best_cost = -1.0;
  for (int A = 8; A >= 1; A >>= 1) {
    if (A * NA > 512) continue;
    const int Mt = RA * A;
    const int rbox = (Mt + 2 * a.wp + 1) / a.wp + 2;
    if (rbox > 256) continue;
    const int tiles = ((p.h - 1) * a.wp + a.ws + Mt - 1) / Mt;
    const long long grid = (long long)p.n * a.strips * tiles * grid_y;
    if (grid / grid_y > 0x7FFFFFFF) continue;
    int bestCC = 0, bestStages = 0, bestScore = -1;
    uint32_t bestStage = 0;
    for (int CC = 64; CC >= 16; CC >>= 1) {
      if (p.cin % CC) continue;
      const uint32_t halo = halo_bytes_for(CC, rbox, a.wp);
      const uint32_t stage = ((halo + (uint32_t)CC * 9u * N * 2u) + 1023u) & ~1023u;
      const int chunks = p.cin / CC;
      int stages = (int)((budget - 1024) / stage);
      if (stages > kMaxStages) stages = kMaxStages;
      if (stages > chunks) stages = chunks;
      if (stages < 1 || (stages < 2 && chunks > 1)) continue;
      const int score = (stages >= 3 || stages == chunks ? 100 : 0) + CC;
      if (score > bestScore) {
        bestScore = score;
        bestCC = CC;
        bestStages = stages;
        bestStage = stage;
      }
    }
    if (bestScore < 0) continue;
    int bytes = (int)(bestStage * bestStages) + 1024;
    if (fold && bytes < min_bytes) bytes = min_bytes;
    int per_sm = (228 * 1024) / (bytes + 1024);
    const int by_tmem = 512 / tmem_cols_host(A * NA);
    if (per_sm > by_tmem) per_sm = by_tmem;
    if (per_sm < 1) per_sm = 1;
    const long long slots = (long long)sms * per_sm;
    const double waves = (double)((grid + slots - 1) / slots);
    const double cost = waves * (Mt + 2.0 * a.wp + 256.0);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      a.A = A;
      a.CC = bestCC;
      a.stages = bestStages;
      a.rbox = rbox;
      a.tiles = tiles;
      a.halo_bytes = halo_bytes_for(bestCC, rbox, a.wp);
      a.rb = 2 * bestCC;
      a.stage_bytes = bestStage;
      grid_x = (int)(grid / grid_y);
      smem = bytes;
    }
  }
  return best_cost >= 0;
}

template <int N, bool FOLD>
cudaError_t launch_fwd_kernel(const CUtensorMap& map, const FwdArgs& a, int gx, int gy, int smem, cudaStream_t s) {
  static unsigned long long smem_set = 0;  // devices on which the attribute was raised
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(smem_set & bit)) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_conv3x3_fwd<N, FOLD>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget + 1024);
    if (e != cudaSuccess) return e;
    smem_set |= bit;
  }
  k_conv3x3_fwd<N, FOLD><<<dim3((unsigned)gx, (unsigned)gy), kThreads, smem, s>>>(map, a);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_fwd_n(const ConvParams& p, cudaStream_t s) {
  int dev0 = 0, sms = 0;
  cudaGetDevice(&dev0);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev0);
  if (sms < 1) sms = 1;
  constexpr bool fold = MC_CONV_FOLD && N == 16;  // measured: a gain at N = 16 only
  FwdArgs a{};
  int gx = 0, gy = 0, smem = 0;
  if (!plan_fwd(p, N, fold, sms, a, gx, gy, smem)) return cudaErrorInvalidValue;
  a.wm = p.wt;
  a.bias = p.bias;
  a.y = p.y;
  a.n = p.n;
  a.h = p.h;
  a.w = p.w;
  a.cin = p.cin;
  a.cout = p.cout;
  a.co_total = p.co_total;
  a.co0 = p.co0;
  a.relu = p.relu;
  a.out_f32 = p.out_f32;
  a.err = p.err;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t dims[4] = {(cuuint64_t)p.cin, (cuuint64_t)p.w, (cuuint64_t)p.h, (cuuint64_t)p.n};
  const cuuint64_t strides[3] = {(cuuint64_t)p.cin * 2, (cuuint64_t)p.cin * 2 * p.w, (cuuint64_t)p.cin * 2 * p.w * p.h};
  const cuuint32_t box[4] = {(cuuint32_t)a.CC, (cuuint32_t)a.wp, (cuuint32_t)a.rbox, 1u};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  const CUtensorMapSwizzle swz = a.rb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                 : a.rb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                              : CU_TENSOR_MAP_SWIZZLE_32B;
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)p.x, dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  if constexpr (fold)
    return launch_fwd_kernel<N, true>(map, a, gx, gy, smem, s);
  else
    return launch_fwd_kernel<N, false>(map, a, gx, gy, smem, s);
}

template <int N>
cudaError_t launch_wgrad_n(const WgradParams& p, int splits, cudaStream_t s) {
  const int smem = ConvSmem<N>::bytes;
  cudaError_t e = cudaFuncSetAttribute(k_conv3x3_wgrad<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int ktiles = (9 * p.cin + kM - 1) / kM;
  k_conv3x3_wgrad<N><<<dim3(ktiles, splits), kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

// N = the launch's cout rounded up to the tile widths 16/32/64/128/256 (cout a
// multiple of 16; wider outputs are split over blockIdx.y).  x must be 16-byte
// aligned; wt is the packed operand order [cin/8][9][co_total][8].
cudaError_t launch_conv3x3_fwd(const ConvParams& p, cudaStream_t s) {
  if (p.cin % 16 || p.cout % 16 || p.cin < 16 || p.cout < 16 || p.co_total < p.co0 + p.cout || p.n < 1 || p.h < 1 ||
      p.w < 1 || ((uintptr_t)p.x & 15) || ((uintptr_t)p.wt & 15))
    return cudaErrorInvalidValue;
  int N = p.cout <= 16 ? 16 : p.cout <= 32 ? 32 : p.cout <= 64 ? 64 : p.cout <= 128 ? 128 : 256;
  if (MC_CONV_SPLIT_N) {
    // small images: narrower output-channel tiles (more CTAs, each reading the same input tile) until the
    // grid covers the SMs
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    while (N > 64) {
      FwdArgs a{};
      int gx = 0, gy = 0, smem = 0;
      if (!plan_fwd(p, N, false, sms, a, gx, gy, smem) || (long long)gx * gy >= sms) break;
      N >>= 1;
    }
  }
  switch (N) {
    case 16: return launch_fwd_n<16>(p, s);
    case 32: return launch_fwd_n<32>(p, s);
    case 64: return launch_fwd_n<64>(p, s);
    case 128: return launch_fwd_n<128>(p, s);
    default: return launch_fwd_n<256>(p, s);
  }
}

cudaError_t launch_conv3x3_wgrad(const WgradParams& p, int splits, cudaStream_t s) {
  if (p.cin % 16 || p.cout % 16 || p.cout > 256 || p.cin < 16 || splits < 1) return cudaErrorInvalidValue;
  if (p.cout <= 16) return launch_wgrad_n<16>(p, splits, s);
  if (p.cout <= 32) return launch_wgrad_n<32>(p, splits, s);
  if (p.cout <= 64) return launch_wgrad_n<64>(p, splits, s);
  if (p.cout <= 128) return launch_wgrad_n<128>(p, splits, s);
  return launch_wgrad_n<256>(p, splits, s);
}

}  // namespace mcx
