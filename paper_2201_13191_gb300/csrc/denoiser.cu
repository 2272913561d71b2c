// Learned scatter denoiser: a residual U-Net (4 levels, 32 base channels, 3x3
// convolutions, 2x2 max pooling, nearest up-sampling, concatenated skips),
// BF16 weights and activations with FP32 accumulation in tensor memory, trained
// with Adam on pairs of low-photon / high-photon scatter images produced by the
// Monte Carlo of this library.  It replaces the Savitzky-Golay smoothing of
// Sec. II-C.4 at low photon counts; plain high-photon Monte Carlo remains the
// reference that judges it.
//
// Images are normalised per image by their mean s: the network sees x / s and
// predicts a residual r, the output is s (x / s + r).  All convolutions run on
// the tcgen05 kernels of k_conv.cu; every other step on the kernels of k_nn.cu;
// the host only sequences launches.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <set>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "mc_internal.h"
#include "mc_nn.h"

namespace mcx {

namespace {

struct Layer {
  int cin = 0, cout = 0;
  bool relu = true;
  float *w = nullptr, *b = nullptr;    // FP32 master [cout][9][cin], [cout]
  float *gw = nullptr, *gb = nullptr;  // gradients
  float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;  // Adam moments
  __nv_bfloat16* wb = nullptr;  // forward weights, tensor-core order [cin/8][9][cout][8]
  __nv_bfloat16* wt = nullptr;  // adjoint weights, tensor-core order [cout/8][9][cin][8]
  size_t nw() const { return (size_t)cout * 9 * cin; }
};

constexpr int kLayers = 15;
// (cin, cout) of the 15 convolutions; level resolution index in kLevel
constexpr int kCin[kLayers] = {16, 32, 32, 64, 64, 128, 128, 256, 384, 128, 192, 64, 96, 32, 32};
constexpr int kCout[kLayers] = {32, 32, 64, 64, 128, 128, 256, 256, 128, 128, 64, 64, 32, 32, 16};
constexpr int kLevel[kLayers] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0, 0};

}  // namespace

struct Denoiser {
  int H = 0, W = 0, B = 0;
  int step = 0;
  Layer L[kLayers];
  // activations, BF16
  __nv_bfloat16 *in0, *a0a, *s0, *p0, *a1a, *s1, *p1, *a2a, *s2, *p2, *a3a, *a3b, *cat2, *u2a, *u2b, *cat1, *u1a,
      *u1b, *cat0, *u0a, *u0b, *gbuf;
  float* out;  // FP32 [B][H][W][16]
  // gradients, FP32
  float *g_out, *g_u0b, *g_u0a, *g_cat0up, *g_s0, *g_u1b, *g_u1a, *g_cat1up, *g_s1, *g_u2b, *g_u2a, *g_cat2up, *g_s2,
      *g_a3b, *g_a3a, *g_p2, *g_a2a, *g_p1, *g_a1a, *g_p0, *g_a0a;
  float* scale;  // [B]
  double* loss;  // [1]
  int* err;      // [1]
  // inference replay: input/output staging and one CUDA graph per batch size
  float *stage_in = nullptr, *stage_out = nullptr;  // [B][H][W]
  cudaStream_t cap = nullptr;
  std::map<int, cudaGraphExec_t> graphs;
  std::set<int> warmed;
  std::vector<void*> allocs;
};

namespace {

template <class T>
cudaError_t dalloc(Denoiser* d, T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T) + 16);
  if (e == cudaSuccess) {
    d->allocs.push_back((void*)*p);
    e = cudaMemset(*p, 0, count * sizeof(T) + 16);
  }
  return e;
}

size_t npix(const Denoiser* d, int n, int level) { return (size_t)n * (d->H >> level) * (d->W >> level); }

// Output channels co0 .. co0 + cout of the operator whose packed weights `wts`
// hold co_total output channels.
cudaError_t conv(const Denoiser* d, const Layer& l, const __nv_bfloat16* x, const __nv_bfloat16* wts, const float* bias,
                 void* y, int n, int level, int cin, int cout, int co_total, int co0, bool relu, bool out_f32,
                 cudaStream_t s) {
  ConvParams p;
  p.x = x;
  p.wt = wts;
  p.bias = bias;
  p.y = y;
  p.n = n;
  p.h = d->H >> level;
  p.w = d->W >> level;
  p.cin = cin;
  p.cout = cout;
  p.co_total = co_total;
  p.co0 = co0;
  p.relu = relu ? 1 : 0;
  p.out_f32 = out_f32 ? 1 : 0;
  p.err = d->err;
  (void)l;
  return launch_conv3x3_fwd(p, s);
}

cudaError_t forward(Denoiser* d, const float* img, int n, cudaStream_t s) {
  cudaError_t e;
#define TRY(x)                     \
  do {                             \
    e = (x);                       \
    if (e != cudaSuccess) return e; \
  } while (0)
  const int hw = d->H * d->W;
  TRY(nn::image_mean(img, n, hw, d->scale, s));
  TRY(nn::pack_input(img, d->scale, n, hw, d->in0, s));
  const Layer* L = d->L;
  auto c = [&](int i, const __nv_bfloat16* x, void* y, bool f32 = false) {
    return conv(d, L[i], x, L[i].wb, L[i].b, y, n, kLevel[i], L[i].cin, L[i].cout, L[i].cout, 0, L[i].relu, f32, s);
  };
  TRY(c(0, d->in0, d->a0a));
  TRY(c(1, d->a0a, d->s0));
  TRY(nn::pool_fwd(d->s0, n, d->H, d->W, 32, d->p0, s));
  TRY(c(2, d->p0, d->a1a));
  TRY(c(3, d->a1a, d->s1));
  TRY(nn::pool_fwd(d->s1, n, d->H >> 1, d->W >> 1, 64, d->p1, s));
  TRY(c(4, d->p1, d->a2a));
  TRY(c(5, d->a2a, d->s2));
  TRY(nn::pool_fwd(d->s2, n, d->H >> 2, d->W >> 2, 128, d->p2, s));
  TRY(c(6, d->p2, d->a3a));
  TRY(c(7, d->a3a, d->a3b));
  TRY(nn::up_fwd(d->a3b, n, d->H >> 3, d->W >> 3, 256, d->cat2, 384, 0, s));
  TRY(nn::copy_channels(d->s2, npix(d, n, 2), 128, d->cat2, 384, 256, s));
  TRY(c(8, d->cat2, d->u2a));
  TRY(c(9, d->u2a, d->u2b));
  TRY(nn::up_fwd(d->u2b, n, d->H >> 2, d->W >> 2, 128, d->cat1, 192, 0, s));
  TRY(nn::copy_channels(d->s1, npix(d, n, 1), 64, d->cat1, 192, 128, s));
  TRY(c(10, d->cat1, d->u1a));
  TRY(c(11, d->u1a, d->u1b));
  TRY(nn::up_fwd(d->u1b, n, d->H >> 1, d->W >> 1, 64, d->cat0, 96, 0, s));
  TRY(nn::copy_channels(d->s0, npix(d, n, 0), 32, d->cat0, 96, 64, s));
  TRY(c(12, d->cat0, d->u0a));
  TRY(c(13, d->u0a, d->u0b));
  TRY(c(14, d->u0b, d->out, true));
  return cudaSuccess;
}

// Backward through layer i: gradient g_y (FP32) at its output y (BF16, ReLU
// mask when the layer has one), input x.  Accumulates the weight and bias
// gradients; writes the input gradient into gx (rows [0, split)) and gx2
// (rows [split, cin)) when those are non-null.
cudaError_t back(Denoiser* d, int i, int n, const __nv_bfloat16* x, const __nv_bfloat16* y, const float* g_y, float* gx,
                 float* gx2, int split, cudaStream_t s) {
  cudaError_t e;
  Layer& l = d->L[i];
  const int lev = kLevel[i];
  const size_t np = npix(d, n, lev);
  TRY(nn::relu_mask(g_y, l.relu ? y : nullptr, np * l.cout, d->gbuf, s));
  TRY(nn::bias_grad(d->gbuf, np, l.cout, l.gb, s));
  WgradParams wp;
  wp.x = x;
  wp.dy = d->gbuf;
  wp.dw = l.gw;
  wp.n = n;
  wp.h = d->H >> lev;
  wp.w = d->W >> lev;
  wp.cin = l.cin;
  wp.cout = l.cout;
  wp.err = d->err;
  const int ktiles = (9 * l.cin + 127) / 128;
  int splits = (int)std::max<size_t>(1, std::min<size_t>(np / 256, (size_t)(4 * 152 / ktiles + 1)));
  TRY(launch_conv3x3_wgrad(wp, splits, s));
  if (gx) {
    const int c1 = split > 0 ? split : l.cin;
    TRY(conv(d, l, d->gbuf, l.wt, nullptr, gx, n, lev, l.cout, c1, l.cin, 0, false, true, s));
    if (gx2) TRY(conv(d, l, d->gbuf, l.wt, nullptr, gx2, n, lev, l.cout, l.cin - c1, l.cin, c1, false, true, s));
  }
  return cudaSuccess;
}

cudaError_t backward(Denoiser* d, int n, cudaStream_t s) {
  cudaError_t e;
  const int H = d->H, W = d->W;
  TRY(back(d, 14, n, d->u0b, nullptr, d->g_out, d->g_u0b, nullptr, 0, s));
  TRY(back(d, 13, n, d->u0a, d->u0b, d->g_u0b, d->g_u0a, nullptr, 0, s));
  TRY(back(d, 12, n, d->cat0, d->u0a, d->g_u0a, d->g_cat0up, d->g_s0, 64, s));
  TRY(nn::up_bwd(d->g_cat0up, n, H >> 1, W >> 1, 64, 64, 0, d->g_u1b, s));
  TRY(back(d, 11, n, d->u1a, d->u1b, d->g_u1b, d->g_u1a, nullptr, 0, s));
  TRY(back(d, 10, n, d->cat1, d->u1a, d->g_u1a, d->g_cat1up, d->g_s1, 128, s));
  TRY(nn::up_bwd(d->g_cat1up, n, H >> 2, W >> 2, 128, 128, 0, d->g_u2b, s));
  TRY(back(d, 9, n, d->u2a, d->u2b, d->g_u2b, d->g_u2a, nullptr, 0, s));
  TRY(back(d, 8, n, d->cat2, d->u2a, d->g_u2a, d->g_cat2up, d->g_s2, 256, s));
  TRY(nn::up_bwd(d->g_cat2up, n, H >> 3, W >> 3, 256, 256, 0, d->g_a3b, s));
  TRY(back(d, 7, n, d->a3a, d->a3b, d->g_a3b, d->g_a3a, nullptr, 0, s));
  TRY(back(d, 6, n, d->p2, d->a3a, d->g_a3a, d->g_p2, nullptr, 0, s));
  TRY(nn::pool_bwd(d->s2, d->g_p2, n, H >> 2, W >> 2, 128, d->g_s2, s));
  TRY(back(d, 5, n, d->a2a, d->s2, d->g_s2, d->g_a2a, nullptr, 0, s));
  TRY(back(d, 4, n, d->p1, d->a2a, d->g_a2a, d->g_p1, nullptr, 0, s));
  TRY(nn::pool_bwd(d->s1, d->g_p1, n, H >> 1, W >> 1, 64, d->g_s1, s));
  TRY(back(d, 3, n, d->a1a, d->s1, d->g_s1, d->g_a1a, nullptr, 0, s));
  TRY(back(d, 2, n, d->p0, d->a1a, d->g_a1a, d->g_p0, nullptr, 0, s));
  TRY(nn::pool_bwd(d->s0, d->g_p0, n, H, W, 32, d->g_s0, s));
  TRY(back(d, 1, n, d->a0a, d->s0, d->g_s0, d->g_a0a, nullptr, 0, s));
  TRY(back(d, 0, n, d->in0, d->a0a, d->g_a0a, nullptr, nullptr, 0, s));
  return cudaSuccess;
}

cudaError_t refresh_weights(Denoiser* d, cudaStream_t s) {
  cudaError_t e;
  for (auto& l : d->L) TRY(nn::pack_weights(l.w, l.cout, l.cin, l.wb, l.wt, s));
  return cudaSuccess;
}

}  // namespace

void denoiser_destroy(Denoiser* d) {
  if (!d) return;
  cudaDeviceSynchronize();
  for (auto& g : d->graphs) cudaGraphExecDestroy(g.second);
  if (d->cap) cudaStreamDestroy(d->cap);
  for (void* p : d->allocs) cudaFree(p);
  delete d;
}

cudaError_t denoiser_create(int H, int W, int B, unsigned long long seed, Denoiser** out) {
  *out = nullptr;
  if (H < 16 || W < 16 || H % 16 || W % 16 || B < 1) return cudaErrorInvalidValue;
  Denoiser* d = new Denoiser();
  d->H = H;
  d->W = W;
  d->B = B;
  cudaError_t e = cudaSuccess;
#define A(ptr, count)                         \
  do {                                        \
    if (e == cudaSuccess) e = dalloc(d, &(ptr), (count)); \
  } while (0)
  const size_t n0 = (size_t)B * H * W, n1 = n0 / 4, n2 = n0 / 16, n3 = n0 / 64;
  A(d->in0, n0 * 16); A(d->a0a, n0 * 32); A(d->s0, n0 * 32); A(d->p0, n1 * 32);
  A(d->a1a, n1 * 64); A(d->s1, n1 * 64); A(d->p1, n2 * 64);
  A(d->a2a, n2 * 128); A(d->s2, n2 * 128); A(d->p2, n3 * 128);
  A(d->a3a, n3 * 256); A(d->a3b, n3 * 256);
  A(d->cat2, n2 * 384); A(d->u2a, n2 * 128); A(d->u2b, n2 * 128);
  A(d->cat1, n1 * 192); A(d->u1a, n1 * 64); A(d->u1b, n1 * 64);
  A(d->cat0, n0 * 96); A(d->u0a, n0 * 32); A(d->u0b, n0 * 32);
  A(d->out, n0 * 16);
  A(d->stage_in, n0);
  A(d->stage_out, n0);
  A(d->gbuf, std::max(std::max(n0 * 32, n1 * 64), std::max(n2 * 128, n3 * 256)));
  A(d->g_out, n0 * 16); A(d->g_u0b, n0 * 32); A(d->g_u0a, n0 * 32); A(d->g_cat0up, n0 * 64); A(d->g_s0, n0 * 32);
  A(d->g_u1b, n1 * 64); A(d->g_u1a, n1 * 64); A(d->g_cat1up, n1 * 128); A(d->g_s1, n1 * 64);
  A(d->g_u2b, n2 * 128); A(d->g_u2a, n2 * 128); A(d->g_cat2up, n2 * 256); A(d->g_s2, n2 * 128);
  A(d->g_a3b, n3 * 256); A(d->g_a3a, n3 * 256); A(d->g_p2, n3 * 128);
  A(d->g_a2a, n2 * 128); A(d->g_p1, n2 * 64); A(d->g_a1a, n1 * 64); A(d->g_p0, n1 * 32); A(d->g_a0a, n0 * 32);
  A(d->scale, (size_t)B);
  A(d->loss, (size_t)1);
  A(d->err, (size_t)1);
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.f, 1.f);
  for (int i = 0; i < kLayers && e == cudaSuccess; ++i) {
    Layer& l = d->L[i];
    l.cin = kCin[i];
    l.cout = kCout[i];
    l.relu = i != kLayers - 1;
    const size_t nw = l.nw();
    A(l.w, nw); A(l.gw, nw); A(l.mw, nw); A(l.vw, nw); A(l.wb, nw); A(l.wt, nw);
    A(l.b, (size_t)l.cout); A(l.gb, (size_t)l.cout); A(l.mb, (size_t)l.cout); A(l.vb, (size_t)l.cout);
    if (e != cudaSuccess) break;
    // He initialisation over the real fan-in (the first layer sees one channel);
    // the output layer starts small so the initial residual is close to zero
    const int fan_in = 9 * (i == 0 ? 1 : l.cin);
    const float sd = std::sqrt(2.f / (float)fan_in) * (i == kLayers - 1 ? 0.1f : 1.f);
    std::vector<float> hw(nw);
    for (size_t k = 0; k < nw; ++k) hw[k] = sd * nd(rng);
    e = cudaMemcpy(l.w, hw.data(), nw * 4, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = refresh_weights(d, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    denoiser_destroy(d);
    return e;
  }
  *out = d;
  return cudaSuccess;
#undef A
}

// Inference of one staged batch: forward pass and residual output.
cudaError_t infer_staged(Denoiser* d, int nb, cudaStream_t s) {
  cudaError_t e;
  TRY(forward(d, d->stage_in, nb, s));
  TRY(nn::unpack_output(d->stage_in, d->scale, d->out, nb, d->H * d->W, d->stage_out, s));
  return cudaSuccess;
}

// Inference replays one captured CUDA graph per batch size: the batch is
// staged into a fixed buffer (the graph's input), the ~30 launches of the
// network go out as one graph launch, and the result is copied out.  The
// first call for a batch size runs the launches directly (it also sets the
// kernels' attributes), the second captures them on a private stream.
cudaError_t denoiser_infer(Denoiser* d, const float* img, float* out, int n, cudaStream_t s) {
  cudaError_t e;
  const size_t hw = (size_t)d->H * d->W;
  for (int b0 = 0; b0 < n; b0 += d->B) {
    const int nb = std::min(d->B, n - b0);
    const size_t off = (size_t)b0 * hw;
    TRY(cudaMemcpyAsync(d->stage_in, img + off, nb * hw * 4, cudaMemcpyDeviceToDevice, s));
    auto it = d->graphs.find(nb);
    if (it == d->graphs.end() && d->warmed.count(nb)) {
      if (!d->cap) TRY(cudaStreamCreateWithFlags(&d->cap, cudaStreamNonBlocking));
      cudaGraph_t g = nullptr;
      TRY(cudaStreamBeginCapture(d->cap, cudaStreamCaptureModeThreadLocal));
      const cudaError_t ec = infer_staged(d, nb, d->cap);
      const cudaError_t ee = cudaStreamEndCapture(d->cap, &g);
      if (ec != cudaSuccess) return ec;
      if (ee != cudaSuccess) return ee;
      cudaGraphExec_t x = nullptr;
      e = cudaGraphInstantiate(&x, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return e;
      it = d->graphs.emplace(nb, x).first;
    }
    if (it != d->graphs.end()) {
      TRY(cudaGraphLaunch(it->second, s));
    } else {
      TRY(infer_staged(d, nb, s));
      d->warmed.insert(nb);
    }
    TRY(cudaMemcpyAsync(out + off, d->stage_out, nb * hw * 4, cudaMemcpyDeviceToDevice, s));
  }
  return cudaSuccess;
}

// One optimiser step on a batch; *loss_out receives the batch loss (mean
// squared error in normalised units) of the forward pass before the update.
cudaError_t denoiser_train_step(Denoiser* d, const float* noisy, const float* clean, int n, float lr, float* loss_out,
                                int* err_out, cudaStream_t s) {
  cudaError_t e;
  if (n < 1 || n > d->B) return cudaErrorInvalidValue;
  TRY(cudaMemsetAsync(d->loss, 0, 8, s));
  TRY(cudaMemsetAsync(d->err, 0, 4, s));
  TRY(forward(d, noisy, n, s));
  TRY(nn::mse(noisy, clean, d->scale, d->out, n, d->H * d->W, d->g_out, d->loss, s));
  for (auto& l : d->L) {
    TRY(cudaMemsetAsync(l.gw, 0, l.nw() * 4, s));
    TRY(cudaMemsetAsync(l.gb, 0, (size_t)l.cout * 4, s));
  }
  TRY(backward(d, n, s));
  d->step += 1;
  if (lr > 0.f) {
    for (auto& l : d->L) {
      TRY(nn::adam(l.w, l.gw, l.mw, l.vw, l.nw(), lr, d->step, nullptr, s));
      TRY(nn::adam(l.b, l.gb, l.mb, l.vb, (size_t)l.cout, lr, d->step, nullptr, s));
      TRY(nn::pack_weights(l.w, l.cout, l.cin, l.wb, l.wt, s));
    }
  }
  double loss = 0;
  TRY(cudaMemcpyAsync(&loss, d->loss, 8, cudaMemcpyDeviceToHost, s));
  TRY(cudaMemcpyAsync(err_out, d->err, 4, cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  *loss_out = (float)loss;
  return cudaSuccess;
}

int denoiser_size(const Denoiser* d, int* H, int* W, int* B) {
  *H = d->H;
  *W = d->W;
  *B = d->B;
  return kLayers;
}

// Copy layer i's weights, bias and last gradients to host (nullable outputs);
// returns false for a bad index.
bool denoiser_get_layer(const Denoiser* d, int i, float* w, float* b, float* gw, float* gb, int* cin, int* cout) {
  if (i < 0 || i >= kLayers) return false;
  const Layer& l = d->L[i];
  *cin = l.cin;
  *cout = l.cout;
  if (w) cudaMemcpy(w, l.w, l.nw() * 4, cudaMemcpyDeviceToHost);
  if (b) cudaMemcpy(b, l.b, (size_t)l.cout * 4, cudaMemcpyDeviceToHost);
  if (gw) cudaMemcpy(gw, l.gw, l.nw() * 4, cudaMemcpyDeviceToHost);
  if (gb) cudaMemcpy(gb, l.gb, (size_t)l.cout * 4, cudaMemcpyDeviceToHost);
  return true;
}

bool denoiser_set_layer(Denoiser* d, int i, const float* w, const float* b) {
  if (i < 0 || i >= kLayers) return false;
  Layer& l = d->L[i];
  if (w) cudaMemcpy(l.w, w, l.nw() * 4, cudaMemcpyHostToDevice);
  if (b) cudaMemcpy(l.b, b, (size_t)l.cout * 4, cudaMemcpyHostToDevice);
  nn::pack_weights(l.w, l.cout, l.cin, l.wb, l.wt, 0);
  return cudaDeviceSynchronize() == cudaSuccess;
}

int denoiser_layer_count() { return kLayers; }

}  // namespace mcx
