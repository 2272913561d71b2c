/*
 * mc.h -- C ABI of the GB300 Monte Carlo X-ray scatter forward projection.
 *
 * Method: "Computational Scatter Correction for High-Resolution Flat-Panel CT
 * Based on a Fast Monte Carlo Photon Transport Model" (arXiv 2201.13191),
 * Sec. II-A (photon transport model, eqs. KleinNishina, Thomson, Th,
 * pmueforIncoherent, pmueforcoherent, Is, Ip), Sec. II-C (variance
 * reduction, controllable ray-tracing step, dual interpolation, smoothing)
 * and Sec. II-E (iterative correction, eq. Correction).
 *
 * Conventions shared by every entry point
 *   - lengths in mm, energies in keV, angles in radians;
 *   - the volume is centred on the isocentre, stored [nz][ny][nx] with x
 *     fastest; the source turns about z: s(b) = SOD (cos b, sin b, 0); the
 *     flat panel is centred on (SOD - SDD)(cos b, sin b, 0) with axes
 *     e_u = (-sin b, cos b, 0), e_v = (0, 0, 1); images are [nv][nu] row
 *     major, pixel (i, j) centred at (i - (nu-1)/2) pu e_u + (j - (nv-1)/2) pv e_v
 *     from the panel centre;
 *   - detector response eta(E) = E (energy integrating) unless
 *     mc_set_detector_response sets another; both images are the expected
 *     detector signal per pixel per source photon emitted into 4 pi (keV for
 *     eta = E), the source being collimated to the detector pyramid;
 *   - the object is a voxel volume (mc_load_volume) or closed triangulated
 *     bodies (mc_load_mesh), whichever was loaded last;
 *   - device pointers belong to the caller, who keeps ownership; the library
 *     copies what it needs at load time and owns only its internal buffers;
 *   - every call returns MC_OK or a negative status; mc_last_error() gives
 *     detail.  No C++ exception crosses the ABI.  A context is not thread
 *     safe: use one context per host thread.  All GPU work is enqueued on the
 *     caller's stream (a cudaStream_t passed as void*, NULL = legacy default).
 */
#ifndef MC_H
#define MC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MC_OK 0
#define MC_ERR_INVALID_ARG -1 /* argument out of range or inconsistent */
#define MC_ERR_STATE -2       /* call made before the data it needs was loaded */
#define MC_ERR_CUDA -3        /* a CUDA runtime call failed */
#define MC_ERR_OOM -4         /* device allocation failed */
#define MC_ERR_TIMEOUT -5     /* a bounded device wait gave up */
#define MC_ERR_LIMIT -6       /* a history hit the scatter-order or sampler cap; outputs valid */
#define MC_ERR_INTERNAL -7    /* a device-side consistency check failed */
#define MC_ERR_IO -8          /* table file missing or malformed */

#define MC_MAX_MATERIALS 8
#define MC_MAX_BINS 512
#define MC_MAX_BODIES 64

typedef struct mc_ctx mc_ctx;

/* Tally modes for the scatter image (Sec. II-A, eq. Is). */
#define MC_TALLY_AUTO 0   /* the fastest measured mode: currently GLOBAL on every workload */
#define MC_TALLY_GLOBAL 1 /* every pseudo-particle adds straight into the FP64 image */
#define MC_TALLY_SHARED 2 /* per-block FP32 shared-memory image (warp-combined adds), flushed into
                             FP64 at block end; needs n_batches x n_angles x nu x nv <= 12288 */
#define MC_TALLY_WARP 3   /* lanes of a warp hitting the same pixel combine (match + shuffle) first */
#define MC_TALLY_TILED 4  /* tile-stratified point-detector pixels: the panel is cut into tiles of
                             tile_u x tile_v pixels (T tiles); history h aims every pseudo-particle at
                             tile (h + o) mod T only, o uniform on [0, T) per run and angle (Philox
                             block (2^32-1, angle, 2^32-1, 2^32-1)), at a pixel uniform in the tile, with
                             weight T (unbiased); each block works through chunks of one (angle, tile)
                             and tallies the tile in shared memory, flushed into FP64 per chunk; needs
                             n_batches x tile_u x tile_v <= 12288 */

typedef struct mc_options {
  int n_split;           /* pseudo-particles per scatter interaction (Sec. II-C.1), default 10 */
  float rr_threshold;    /* Russian roulette on the pseudo-particle weight x0 (Sec. II-C.1); 0 = off */
  int max_scatter_order; /* a history ends after this many scatters (energy deposited), default 64 */
  int n_batches;         /* >1: histories h mod n_batches form batches for scatter_var_out (with
                            MC_TALLY_TILED: floor(h / T) mod n_batches, T the number of tiles) */
  int block_size;        /* transport threads per block; 0 = default (256) */
  int blocks_per_sm;     /* persistent grid = SMs x blocks_per_sm; 0 = default (occupancy) */
  int tally_mode;        /* MC_TALLY_* */
  int sg_window;         /* Savitzky-Golay window (odd, >= order + 2), default 9 (Sec. II-C.4) */
  int sg_order;          /* Savitzky-Golay polynomial order, default 3 (Sec. II-C.4) */
  float cubic_a;         /* Keys cubic parameter of the spatial up-sampling, default -0.5 (Sec. II-C.3) */
  int denoise_mode;      /* 0 = Savitzky-Golay, 1 = learned denoiser (mc_denoise_*), 2 = none */
  int voxel_layout;      /* device volume layout: 1 = x fastest, 2 = 4x4x4 Morton bricks, 0 = default:
                            x fastest while the packed volume fits in 3/4 of L2, bricks beyond */
  int use_graph;         /* 1: mc_project replays one captured CUDA graph while its launch shape is unchanged */
  int nee_mode;          /* point-detector scoring (Sec. II-C.1): 0 = the sampled scatter type's pdf (the
                            paper's, default); 1 = expected value over the interaction type: every
                            interaction, absorptions included, scores (mu_incoh/mu) x Compton term at E'
                            + (mu_coh/mu) x Rayleigh term at E, both attenuations from one shared march;
                            same mean, less variance */
  int doppler;           /* 1: Doppler broadening of incoherent scatter (impulse approximation with the
                            orbital model of the bound tables; needs tables of version 2), 0 = off (default) */
  int tile_u, tile_v;    /* tile size in pixels of MC_TALLY_TILED, default 64 x 64 */
  int forced_detection;  /* 1: forced detection (Sec. I names it among the variance-reduction techniques):
                            every scatter interaction sends exactly one pseudo-particle to every pixel of
                            the panel (of the history's tile under MC_TALLY_TILED), at a uniform point in
                            it, with weight 1 instead of P / n_split: the paper's split estimator with the
                            pixel choice stratified, so it adds no variance; n_split is ignored.  Needs
                            at most MC_FORCED_MAX_PIXELS such pixels.  0 = off (default) */
} mc_options;
#define MC_FORCED_MAX_PIXELS 65536

/* Fill *opt with the defaults listed above. */
void mc_default_options(mc_options *opt);

/* Create a context on CUDA device `cuda_device`; opt may be NULL (defaults).
 * *out receives the context.  Errors: INVALID_ARG (bad option), CUDA. */
int mc_create(mc_ctx **out, int cuda_device, const mc_options *opt);
/* Free the context and every device buffer it owns (after a device sync). */
void mc_destroy(mc_ctx *ctx);
/* Replace the options (validated as in mc_create). */
int mc_set_options(mc_ctx *ctx, const mc_options *opt);
/* Detail of the last failing call on this context (never NULL). */
const char *mc_last_error(const mc_ctx *ctx);

/* Load the per-material cross-section tables (1 keV nodes; format described
 * in mc_inputs/tables.py): mu_pe, mu_incoh, mu_coh in cm^2/g and the Rayleigh
 * pdf normalisation I_coh(E), plus each material's form-factor components.
 * These stand in for the Hubbell data of Sec. II-A.  Values between nodes are
 * linear in E.  Errors: IO (missing/malformed file), INVALID_ARG (more than
 * MC_MAX_MATERIALS materials), CUDA/OOM. */
int mc_load_tables(mc_ctx *ctx, const char *path);

/* Load the voxelised object (Sec. II-A last paragraph; Sec. II-E: segmented
 * materials converted to densities): mat[nz][ny][nx] material ids (uint8,
 * each < n_materials), rho_fp16[nz][ny][nx] densities in g/cm^3 as IEEE
 * binary16 bit patterns (finite, >= 0), voxel size dx, dy, dz in mm.  The
 * arrays are host memory (is_device_ptr = 0) or device memory (1); they are
 * copied (on `stream`) and the caller keeps ownership.  Errors: STATE (no
 * tables), INVALID_ARG (sizes, ids, densities), CUDA/OOM. */
int mc_load_volume(mc_ctx *ctx, const uint8_t *mat, const uint16_t *rho_fp16, int nx, int ny, int nz, float dx,
                   float dy, float dz, int is_device_ptr, void *stream);

/* Polychromatic source as discrete bins (Sec. II-A, eq. Is: N bins, M photons
 * per bin): host arrays weights[n] >= 0 (normalised here to sum 1) and
 * energies_keV[n] inside the table range; 1 <= n <= MC_MAX_BINS.  Photons are
 * stratified over bins: M_n = max(1, floor(N S_n)) for S_n > 0 plus the
 * remainder by largest fractional part.  Errors: STATE (no tables), INVALID_ARG. */
int mc_set_spectrum(mc_ctx *ctx, const double *weights, const float *energies_keV, int n_bins);

/* Cone-beam geometry: source-isocentre sod, source-detector sdd (mm), flat
 * panel of nu x nv pixels of pu x pv mm.  The volume must lie strictly
 * between source and panel (checked at projection time).  Errors: INVALID_ARG. */
int mc_set_geometry(mc_ctx *ctx, float sod, float sdd, int nu, int nv, float pu, float pv);

/* Forward projection at n_angles source angles (host array angles_rad), all in
 * one launch per kernel (Sec. II-B projection parallelism).
 *   primary_out  device [n_angles][nv][nu] FP32: eq. (Ip), deterministic line
 *                integral sampled at pixel centres with the fixed-step march;
 *   scatter_out  device [n_angles][nv][nu] FP32: eq. (Is), n_photons histories
 *                per angle, point-detector scoring (eq. Th) split n_split ways;
 *   scatter_var_out (nullable) device, same shape: variance of scatter_out
 *                from n_batches >= 2 batches.
 * Either image pointer may be NULL to skip that image.  step_mm is the
 * controllable ray-tracing step (Sec. II-C.2): each chord is cut into
 * ceil(L/step) equal steps sampled at their midpoints.  Histories are keyed by
 * (seed, angle index, history index) through Philox4x32-10, so results are
 * deterministic up to the order of the FP64 tally sums.  The call returns once
 * the work is enqueued and its status read back (it synchronises `stream`).
 * Errors: STATE, INVALID_ARG, CUDA/OOM, LIMIT (outputs still valid), INTERNAL. */
int mc_project(mc_ctx *ctx, const float *angles_rad, int n_angles, uint64_t n_photons, float step_mm, uint64_t seed,
               float *primary_out, float *scatter_out, float *scatter_var_out, void *stream);

/* As mc_project's scatter image, restricted to histories
 * [h_begin, h_begin + h_count) of an n_photons run: the same histories, the
 * same random numbers and the same weights as in the full run, so any
 * subset can be checked history for history.  scatter_out is FP32
 * [n_angles][nv][nu] on the device.  Errors as mc_project. */
int mc_project_histories(mc_ctx *ctx, const float *angles_rad, int n_angles, uint64_t n_photons, uint64_t h_begin,
                         uint64_t h_count, float step_mm, uint64_t seed, float *scatter_out, void *stream);

/* Counters of the last projection (double[n], n <= MC_STAT_N): histories,
 * flight steps, pseudo-particle steps, pseudo-particles, photoelectric,
 * Compton, Rayleigh, escapes, limit hits, sampler failures, transport kernel
 * milliseconds, primary kernel milliseconds. */
#define MC_STAT_N 12
int mc_last_stats(const mc_ctx *ctx, double *out, int n);

/* Smoothing and dual interpolation of simulated scatter (Sec. II-C.3, II-C.4):
 *   1. Savitzky-Golay smoothing of each input image, separable, polynomial
 *      order opt.sg_order over opt.sg_window points per axis, edges fitted by
 *      the same least-squares polynomial over the first/last window
 *      (denoise_mode 0; mode 2 skips it);
 *   2. linear interpolation in angle, periodic in 2 pi, from the n_in sorted
 *      simulated angles in_angles (host, radians) to out_angles (host);
 *   3. separable Keys cubic up-sampling (parameter opt.cubic_a) from nv x nu
 *      to NV x NU with half-pixel centre alignment and clamped edges.
 * in: device FP32 [n_in][nv][nu]; out: device FP32 [n_out][NV][NU].
 * Values are interpolated as given (no pixel-area rescaling).
 * Errors: INVALID_ARG (sizes, window, unsorted angles), CUDA/OOM. */
int mc_smooth_upsample(mc_ctx *ctx, const float *in, int n_in, const float *in_angles, int nu, int nv, float *out,
                       int n_out, const float *out_angles, int NU, int NV, void *stream);

/* Iterative scatter correction (Sec. II-E and its flowchart; eq. Correction).
 * Measured intensities raw_I (device [n_proj][NV][NU], the panel set by
 * mc_set_geometry at NU x NV pixels) and the flat field I0 (device [NV][NU])
 * give a = -ln(I/I0).  Each of n_iter iterations:
 *   1. FDK reconstruction of the current projections c (c = a at first) on
 *      the nx x ny x nz grid (Ram-Lak ramp, cosine pre-weighting, voxel-driven
 *      backprojection with bilinear interpolation);
 *   2. Otsu segmentation into `classes` (2 or 3) classes of the histogram over
 *      [mu_lo, mu_hi) mm^-1; class 0 becomes class_material[0] at density
 *      class_density0, class k >= 1 becomes class_material[k] with density
 *      mu / (mu_rho(class_material[k], e_eff_keV) x 0.1);
 *   3. Monte Carlo on a sim_nu x sim_nv grid over the same panel: scatter
 *      (photons histories each) at every sim_angle_stride-th angle; the
 *      primary at every angle, on the same grid or (primary_full_res) on the
 *      NU x NV panel; with mc_bin = 2 the Monte Carlo (and the primary on the
 *      simulation grid) runs on the segmented volume down-sampled by 2 per
 *      axis (mc_bin_volume), the full-panel primary on the full volume;
 *   4. smoothing (options.denoise_mode) of the scatter, linear interpolation
 *      to every angle and cubic up-sampling to NU x NV (of the primary too
 *      unless it was computed at full resolution);
 *   5. c = a - ln(Ip / (Ip + Is)); images are per pixel, so with the primary
 *      on the panel the up-sampled scatter is scaled by the pixel-area ratio
 *      (panel pixel / simulation pixel) first.
 * corrected_a_out (device, like raw_I) receives the final c; volume_out
 * (device [nz][ny][nx] FP32, nullable) the last reconstruction (of the last
 * corrected projections when n_iter >= 1); iter_seconds (host [n_iter],
 * nullable) the wall time of each iteration.  angles_rad (host) must cover a
 * full orbit in increasing order.  The context's volume is replaced by the
 * segmented reconstruction (its down-sampled form with mc_bin = 2).
 * Allocates temporary device buffers.
 * Errors: STATE, INVALID_ARG, CUDA/OOM, and those of mc_project. */
typedef struct mc_correct_params {
  int nx, ny, nz;
  float dx, dy, dz;
  int sim_nu, sim_nv;
  int sim_angle_stride;
  uint64_t photons;
  float step_mm;
  uint64_t seed;
  int classes;
  int class_material[3];
  float class_density0;
  float e_eff_keV;
  float mu_lo, mu_hi;
  int primary_full_res; /* 1: primary computed on the NU x NV panel itself (exact, cheap); 0: on the
                           simulation grid and up-sampled with the scatter, as the paper does */
  int mc_bin;           /* 2: the Monte Carlo scatter (and the low-resolution primary) runs on the segmented
                           volume down-sampled by 2 per axis (mc_bin_volume; even nx, ny, nz), as the paper
                           does to cut the ray-tracing time; 0 or 1: on the full volume */
} mc_correct_params;
int mc_correct_iter(mc_ctx *ctx, const float *raw_I, const float *I0, int n_proj, const float *angles_rad, int NU,
                    int NV, int n_iter, const mc_correct_params *prm, float *corrected_a_out, float *volume_out,
                    double *iter_seconds, void *stream);

/* The steps of mc_correct_iter as separate calls (Sec. II-E and its
 * flowchart), so each can be run and checked on its own; mc_correct_iter runs
 * the same kernels.
 *
 * mc_line_integrals: a = -ln(I / I0) per pixel (Sec. II-E: the measured
 *   intensities become line integrals); I device FP32 [n_proj][NV][NU], I0
 *   device FP32 [NV][NU] (one flat field for all projections), a_out device
 *   FP32 like I.  Values below 1e-30 are clamped to 1e-30 first.
 * mc_segment: segmentation of a reconstruction vol (device FP32
 *   [nz][ny][nx], mm^-1) into `classes` (2 or 3) classes by multi-level Otsu
 *   (exhaustive search of the thresholds maximising the between-class
 *   variance, ties to the smallest) over a 256-bin histogram of [mu_lo, mu_hi):
 *   bin b = (int)((mu - mu_lo) * (256 / (mu_hi - mu_lo))) in FP32, clamped to
 *   [0, 255]; thresholds t0 < t1 are bin indices (t1 = 256 for 2 classes) and
 *   a voxel in bin b has class 0 if b < t0, 1 if b < t1, else 2.  Class 0
 *   becomes class_material[0] at density class_density0; class k >= 1 becomes
 *   class_material[k] at rho = mu / (0.1 mu_rho(class_material[k], e_eff_keV))
 *   (FP32, tables linear between nodes), clamped to [0, 30] g/cm^3.  Outputs:
 *   mat_out (device uint8) and rho_out (device binary16 bits) [nz][ny][nx];
 *   hist_out (host uint32 [256], nullable) and thresholds_out (host int [2],
 *   nullable).  Synchronises `stream`.
 * mc_correct_images: eq. (Correction), c = a - ln(Ip / (Ip + s Is)) per
 *   element, with Ip clamped below at 1e-30, Is at 0, s = is_scale (the
 *   pixel-area ratio when Is was simulated on coarser pixels; 1 otherwise);
 *   a, ip, is, c_out device FP32 [n].
 * Errors: STATE (no tables, for mc_segment), INVALID_ARG, CUDA/OOM. */
int mc_line_integrals(mc_ctx *ctx, const float *I, const float *I0, int n_proj, int NU, int NV, float *a_out,
                      void *stream);
int mc_segment(mc_ctx *ctx, const float *vol, int nx, int ny, int nz, int classes, const int *class_material,
               float class_density0, float e_eff_keV, float mu_lo, float mu_hi, uint32_t *hist_out,
               int *thresholds_out, uint8_t *mat_out, uint16_t *rho_out, void *stream);
int mc_correct_images(mc_ctx *ctx, const float *a, const float *ip, const float *is, float is_scale, size_t n,
                      float *c_out, void *stream);

/* Down-sampling of a segmented volume for the Monte Carlo step (Sec. II-C.2:
 * the number of voxels is down-sampled to cut the ray-tracing time; Sec.
 * II-E).  Device mat [nz][ny][nx] (ids < the table's materials) and rho
 * (binary16 g/cm^3), even dimensions -> mat_out, rho_out [nz/2][ny/2][nx/2]
 * (device, caller-owned): each 2x2x2 block becomes one voxel of the material
 * holding the block's largest mass (ties to the lower id), with the density
 * that keeps the block's summed attenuation at e_eff_keV (tables linear
 * between nodes): rho = sum_v mu/rho(m_v) rho_v / (8 mu/rho(m)).  Enqueued on
 * `stream`.  Errors: STATE (no tables), INVALID_ARG (odd dimension, energy
 * outside the table), CUDA/OOM. */
int mc_bin_volume(mc_ctx *ctx, const uint8_t *mat, const uint16_t *rho, int nx, int ny, int nz, float e_eff_keV,
                  uint8_t *mat_out, uint16_t *rho_out, void *stream);

/* Plain FDK reconstruction (step 1 above) of line-integral projections p
 * (device [n_proj][NV][NU], the context's panel geometry) into vol (device
 * [nz][ny][nx], mm^-1).  Errors: STATE (no geometry), INVALID_ARG, CUDA/OOM. */
int mc_fdk(mc_ctx *ctx, const float *p, int n_proj, const float *angles_rad, int NU, int NV, int nx, int ny, int nz,
           float dx, float dy, float dz, float *vol, void *stream);

/* Learned scatter denoiser (replaces the Savitzky-Golay smoothing of
 * Sec. II-C.4 at low photon counts; no counterpart network in the paper): a
 * residual U-Net, 4 levels, 32 base channels, 3x3 convolutions, 2x2 max
 * pooling, nearest up-sampling with concatenated skips, BF16 weights and
 * activations, FP32 accumulation on the tcgen05 tensor cores, Adam.  Images
 * are normalised by their mean; the network predicts a residual.
 *   mc_denoise_init: allocate for height x width images (multiples of 16) and
 *     up to max_batch images per call; seeded He initialisation.
 *   mc_denoise_train_step: one Adam step (lr; lr = 0 computes gradients only)
 *     on n device FP32 image pairs [n][height][width]; *loss = mean squared
 *     error of the normalised images before the step.
 *   mc_denoise_infer: n device FP32 images in, denoised images out (any n).
 *   mc_denoise_get_layer / set_layer: host FP32 weights [cout][9][cin], biases
 *     [cout] and last gradients of layer 0..14 (nullable pointers).
 *   mc_denoise_save / load: FP32 checkpoint file.
 * Errors: STATE (not initialised), INVALID_ARG, CUDA/OOM, TIMEOUT, IO. */
int mc_denoise_init(mc_ctx *ctx, int height, int width, int max_batch, uint64_t seed);
int mc_denoise_train_step(mc_ctx *ctx, const float *noisy, const float *clean, int n, float lr, float *loss,
                          void *stream);
int mc_denoise_infer(mc_ctx *ctx, const float *in, float *out, int n, void *stream);
int mc_denoise_get_layer(mc_ctx *ctx, int layer, float *w, float *b, float *gw, float *gb, int *cin, int *cout);
int mc_denoise_set_layer(mc_ctx *ctx, int layer, const float *w, const float *b);
int mc_denoise_save(mc_ctx *ctx, const char *path);
int mc_denoise_load(mc_ctx *ctx, const char *path, int max_batch);

/* Denoiser convolution primitives on the tcgen05 tensor cores (device
 * pointers, NHWC, BF16 stored as uint16, cin and cout multiples of 16,
 * cout <= 256), enqueued on `stream` without synchronising:
 *   mc_nn_conv3x3: y = relu?(conv3x3_same(x, w) + bias); w [cout][9][cin]
 *     (tap = 3 (dy+1) + (dx+1)), bias FP32 [cout] or NULL, y BF16 or FP32
 *     (out_f32) [n][h][w][cout];
 *   mc_nn_conv3x3_wgrad: dw[cout][9][cin] (FP32, accumulated: zero it first)
 *     += sum over pixels of dy[p][co] x[p shifted by tap][ci], pixels split
 *     over `splits` CTA groups.
 * *err (device int) is set to 1 if a bounded wait gave up. */
int mc_nn_conv3x3(const void *x, const void *w, const float *bias, void *y, int n, int h, int wd, int cin, int cout,
                  int relu, int out_f32, int *err, void *stream);
int mc_nn_conv3x3_wgrad(const void *x, const void *dy, float *dw, int n, int h, int wd, int cin, int cout, int splits,
                        int *err, void *stream);

/* Autotuner of the projection (Sec. II-C.2 controllable step; launch shape).
 * 1. Ray step: primary images (eq. Ip) at step_min and at candidate steps
 *    between step_max and step_min are compared; the largest step whose image
 *    stays within step_tol relative L2 of the step_min image is chosen (the
 *    deterministic primary measures the fixed-step discretisation error).
 * 2. Launch shape: short transport runs of probe_photons histories per angle
 *    at the chosen step, over block size {128, 192, 256}, blocks per SM
 *    {1 .. occupancy} and tally mode {global, warp}; the fastest is kept.
 * 3. Russian roulette (Sec. II-C.1): thresholds of 0.3, 1, 3 and 10 times
 *    the mean attenuated pseudo-particle score of a run without roulette are
 *    compared by figure of merit 1 / (noise^2 x time), the noise being the
 *    8-batch estimate of the scatter image's relative L2 error; the best
 *    (or none) is kept.
 * 4. Tally pixels (tile-stratified point-detector pixels change the noise as
 *    well as the speed): MC_TALLY_TILED with tiles of 16 x 16 and 32 x 32
 *    pixels is compared with the configuration of steps 2-3 by the same
 *    figure of merit; a tile shape is kept only if it beats it.
 * The chosen block_size, blocks_per_sm, tally_mode (and tile_u, tile_v) and
 * rr_threshold are written into the context's options; *out receives them
 * with the step, the measured histories/s and the figure-of-merit gains of the
 * roulette and of the tiles.
 * Allocates temporary device buffers.  Errors as mc_project. */
typedef struct mc_tuning {
  float step_mm;
  int block_size;
  int blocks_per_sm;
  int tally_mode;      /* the mode written into the options: MC_TALLY_TILED when step 4 kept a tile shape */
  double histories_per_s;
  double step_error;   /* relative L2 of the chosen step's primary vs step_min */
  float rr_threshold;  /* chosen Russian-roulette threshold (0: off) */
  double rr_fom_gain;  /* figure of merit with it / without roulette */
  int tile_u, tile_v;  /* chosen tile of MC_TALLY_TILED (0, 0: not tiled) */
  double tile_fom_gain; /* best figure of merit of the tiled trials / that of steps 2-3 */
} mc_tuning;
int mc_autotune(mc_ctx *ctx, const float *angles_rad, int n_angles, uint64_t probe_photons, float step_min,
                float step_max, float step_tol, mc_tuning *out, void *stream);

/* Scatter projection that allocates nothing (no counterpart in the paper: an
 * integration aid).  Some callers cannot allocate device memory once running:
 * services that reserve the whole GPU for a fixed memory pool at start-up (a
 * later cudaMalloc fails or stalls their other streams) and real-time
 * acquisition loops that cannot afford cudaMalloc's implicit device
 * synchronisation per projection.  Such a caller loads tables, volume,
 * spectrum and geometry once at start-up (those calls allocate), then calls
 * this entry point, which computes the same scatter image as mc_project
 * (scatter_out only, n_batches ignored) while keeping its scratch -- FP64
 * tally image, counters, staged tables, spectrum block, angles -- in one
 * file-scope __device__ array of about 32.4 MiB, held on every GPU that loads
 * the library until the process exits.  It calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *   - Limits (larger requests return MC_ERR_INVALID_ARG):
 *       n_angles <= MC_STATIC_MAX_ANGLES;
 *       n_angles * nu * nv <= MC_STATIC_MAX_TALLY;
 *       the cross-section tables staged for the spectrum fit in
 *       MC_STATIC_MAX_TABLE_BYTES: 8 n_s (6 n_mat + 2) + 100 n_mat bytes
 *       (rounded up to 16), n_mat the table's materials and n_s the energy
 *       nodes from the table's first up to one past the spectrum's highest
 *       energy (e.g. 8 materials reach the limit near 160 keV at 1 keV
 *       nodes), where mc_project has no such limit.
 *   - Each CUDA context holds its own copy of the array.  The first call in a
 *     context looks up the array's device address there (cudaGetSymbolAddress,
 *     with the context's device current) and keeps it for that context; make
 *     that first call before any stream capture.  Every call synchronises
 *     `stream` before it returns.
 *   - Every call re-stages and zeroes what it uses, so it never sees an
 *     earlier call's contents; but calls in one context share the one array,
 *     so calls that overlap on the GPU (several streams, several host threads
 *     of one context) race: serialise them.
 *   - Uses about 80 KB of the calling thread's stack for host staging.
 * Inputs: angles_rad host [n_angles]; scatter_out device FP32
 * [n_angles][nv][nu].  Errors: as mc_project. */
#define MC_STATIC_MAX_TALLY 4194304
#define MC_STATIC_MAX_ANGLES 4096
#define MC_STATIC_MAX_TABLE_BYTES 65536
int mc_project_scatter_static(mc_ctx *ctx, const float *angles_rad, int n_angles, uint64_t n_photons, float step_mm,
                              uint64_t seed, float *scatter_out, void *stream);

/* Triangle-mesh geometry (the paper's CAD surface model, Sec. II-A: closed
 * triangulated surfaces).  Host arrays: vertices FP32 [n_vertices][3] (mm, the
 * volume frame: rotation axis z), triangles int32 [n_triangles][3] (counter-
 * clockwise seen from outside), tri_body int32 [n_triangles], and per body
 * material (table index), density (g/cm^3, >= 0) and parent (-1: in vacuum,
 * else an earlier body inside which this one replaces the parent's
 * material); up to MC_MAX_BODIES bodies.  Each body's surface must be closed.
 * The library copies the data, builds a bounding-volume hierarchy and switches
 * the context to this geometry until mc_load_volume is called again.  With a
 * mesh, mc_project and mc_project_histories compute primary images (eq. Ip) by
 * exact ray casting (watertight ray/triangle tests, a body's path length as the
 * signed sum of its crossings) and scatter images (eq. Is) from photon
 * histories with exact free flights through the bodies and exact point-
 * detector attenuation; step_mm is validated but unused, and the warp-combined
 * and shared tally modes act as the global one.  mc_autotune and
 * mc_project_scatter_static serve the voxel volume only (MC_ERR_STATE).
 * Errors: STATE (no tables), INVALID_ARG (indices, bodies, non-finite
 * vertices), INTERNAL (hierarchy deeper than the device stack), CUDA/OOM. */
int mc_load_mesh(mc_ctx *ctx, const float *vertices, int n_vertices, const int *triangles, const int *tri_body,
                 int n_triangles, const int *body_material, const float *body_density, const int *body_parent,
                 int n_bodies);

/* Detector response (Sec. II-D.2: the model maps each detected photon energy
 * through the panel's energy-response curve).  eta[n]: the expected signal
 * (keV) of a photon of energy E reaching the panel, at the table's n_E energy
 * nodes E0 + i dE (host FP64, n == n_E, finite, >= 0), linear between nodes.
 * It replaces the default eta(E) = E (energy integrating) in eq. (Ip) --
 * S(E_n) eta(E_n) per bin -- and in the point-detector score of eq. (Is) at the
 * scattered energy E'.  eta == NULL restores the default; loading tables
 * clears it.  Errors: STATE (no tables), INVALID_ARG. */
int mc_set_detector_response(mc_ctx *ctx, const double *eta, int n);

#ifdef __cplusplus
}
#endif
#endif /* MC_H */
