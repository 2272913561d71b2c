/*
 * ORACLE -- test infrastructure only.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * A plain, slow, single-threaded FP64 restatement of the Monte Carlo X-ray
 * scatter forward projection of "Computational Scatter Correction for
 * High-Resolution Flat-Panel CT Based on a Fast Monte Carlo Photon Transport
 * Model" (arXiv 2201.13191), Sec. II-A and II-C:
 *
 *   - primary image by the deterministic line integral, eq. (Ip);
 *   - photon histories from a binned polychromatic source (Sec. II-A, last
 *     paragraph), free flight by a fixed-step ray march with a controllable
 *     step (Sec. II-C.2), photoelectric absorption, Compton scattering
 *     sampled by Kahn's method from eq. (KleinNishina) with S = 1, Rayleigh
 *     scattering sampled by inversion on F^2 plus rejection on the Thomson
 *     factor, eq. (Thomson);
 *   - scatter scoring by the point-detector estimator eq. (Th) with the
 *     scatter-toward-detector pdfs eqs. (pmueforIncoherent) and
 *     (pmueforcoherent), split into N_split pseudo-particles aimed at
 *     randomly selected pixels (Sec. II-A and II-C.1), optional Russian
 *     roulette, summed per eq. (Is);
 *   - the same histories through closed triangulated bodies (the CAD surface
 *     model of Sec. II-A) with exact path lengths: free flights over the
 *     sorted surface crossings, point-detector attenuation by exact chords;
 *   - options: a detector response table (Sec. II-D.2), expected-value
 *     scoring over the interaction type (Sec. II-C.1), forced detection (one
 *     pseudo-particle per pixel; Sec. I names the technique), the
 *     bound-electron scattering function and Doppler broadening (Sec. II-A),
 *     and tile-stratified point-detector pixels.
 *
 * Readings of the paper that it implements (all listed in the design notes):
 * lengths in mm, energies in keV, eta(E) = E unless a detector response
 * table is set (orc_set_detector_response, Sec. II-D.2), images in expected
 * detector signal per pixel per source photon emitted into 4 pi; step rule = equal
 * subdivision of the clipped chord, nearest voxel at each step midpoint;
 * cross-section tables linear in E between their 1 keV nodes; counter-based
 * Philox4x32-10 random numbers (Salmon et al., SC'11) with a fixed draw order.
 *
 * Parity pins: see the -m "not gpu" tests (chord lengths, Beer-Lambert,
 * chi-square tests of both samplers, pdf normalisation, energy conservation,
 * single-scatter quadrature, NEE vs analog tally, Philox known answers).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ESTATE -2
#define ORC_EIO -8
#define ORC_MAXMAT 16
#define ORC_MAXCOMP 8
#define ORC_MAXBODY 64

static const double PI = 3.14159265358979323846;

typedef struct {
  /* tables */
  int have_tables, n_mat, n_E;
  double E0, dE, r0, mec2, hc, NA, cF, Kpe;
  double density[ORC_MAXMAT];
  int n_comp[ORC_MAXMAT];
  double comp[ORC_MAXMAT][ORC_MAXCOMP][3]; /* Z, w (mol/g), b (A^2) */
  double *mu_pe, *mu_in, *mu_co, *icoh;    /* [n_mat][n_E] */
  int bound;                               /* incoherent scattering function S(x,Z) in use (table version 2) */
  double *iincoh;                          /* [n_mat][n_E] its normalisation (version 2) */
  /* volume */
  int have_volume, nx, ny, nz;
  double dx, dy, dz;
  uint8_t *mat;
  double *rho;
  /* spectrum */
  int have_spectrum, n_bins;
  double *S, *Ebin;
  /* detector response eta(E) at the table nodes (NULL: eta(E) = E) */
  double *eta;
  /* triangle-mesh geometry (CAD bodies); replaces the volume while loaded */
  int have_mesh, n_tri, n_body;
  double *tri;   /* [n_tri][9] vertex coordinates */
  int *tri_body; /* [n_tri] */
  int body_mat[ORC_MAXBODY], body_parent[ORC_MAXBODY];
  double body_rho[ORC_MAXBODY];
  int mesh_active; /* photon histories run in the mesh (set by orc_load_mesh, cleared by orc_load_volume) */
  double mesh_rxy; /* largest distance of a vertex from the rotation axis */
  /* geometry */
  int have_geometry, nu, nv;
  double sod, sdd, pu, pv;
  /* options */
  int n_split, max_order;
  int nee_mode; /* 0: score the sampled scatter type; 1: expected value over both types */
  int forced;   /* forced detection: one pseudo-particle per pixel of the panel (or of the history's tile) */
  int doppler;  /* Doppler broadening of incoherent scatter (needs the bound tables) */
  double rr_threshold, eps_face;
  int tile_u, tile_v; /* > 0: tile-stratified point-detector pixels (see orc_set_tiles) */
} orc_ctx;

/* ------------------------------------------------------------------ */
/* Philox4x32-10, from the published description (Salmon, Moraes, Dror,
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of
 * two 32x32->64 multiplies with a Weyl key schedule. */
void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Per-history random stream: key = seed, counter = (block, angle, h_lo, h_hi).
 * Values are consumed four per block, in order. */
typedef struct {
  uint32_t key[2], ctr[4], buf[4];
  int idx;
  uint64_t draws;
} rng_t;

static void rng_init(rng_t *g, uint64_t h, uint32_t angle_index, uint64_t seed) {
  g->key[0] = (uint32_t)seed;
  g->key[1] = (uint32_t)(seed >> 32);
  g->ctr[0] = 0;
  g->ctr[1] = angle_index;
  g->ctr[2] = (uint32_t)h;
  g->ctr[3] = (uint32_t)(h >> 32);
  g->idx = 4;
  g->draws = 0;
}
static uint32_t rng_next(rng_t *g) {
  if (g->idx == 4) {
    orc_philox(g->ctr, g->key, g->buf);
    g->ctr[0] += 1;
    g->idx = 0;
  }
  g->draws++;
  return g->buf[g->idx++];
}
/* Skip to the start of the next block of four. */
static void rng_align(rng_t *g) { g->idx = 4; }
/* Uniform on (0,1): the top 23 bits plus one half, scaled by 2^-23; exact in FP32. */
static double u01(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }
static double rng_u(rng_t *g) { return u01(rng_next(g)); }

/* ------------------------------------------------------------------ */
/* context */
int orc_create(orc_ctx **out) {
  orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
  if (!c) return ORC_EINVAL;
  c->n_split = 10;
  c->max_order = 64;
  c->rr_threshold = 0.0;
  c->eps_face = 2e-4;
  *out = c;
  return ORC_OK;
}
void orc_destroy(orc_ctx *c) {
  if (!c) return;
  free(c->mu_pe); free(c->mu_in); free(c->mu_co); free(c->icoh); free(c->iincoh);
  free(c->mat); free(c->rho); free(c->S); free(c->Ebin); free(c->eta);
  free(c->tri); free(c->tri_body);
  free(c);
}

int orc_load_tables(orc_ctx *c, const char *path) {
  free(c->eta); /* a response belongs to the previous tables' nodes */
  c->eta = NULL;
  FILE *f = fopen(path, "rb");
  if (!f) return ORC_EIO;
  char magic[8];
  int32_t hdr[4];
  double e[2], k[6];
  if (fread(magic, 1, 8, f) != 8 || memcmp(magic, "MCXTAB01", 8) != 0 || fread(hdr, 4, 4, f) != 4 ||
      fread(e, 8, 2, f) != 2 || fread(k, 8, 6, f) != 6) {
    fclose(f);
    return ORC_EIO;
  }
  int n_mat = hdr[1], n_E = hdr[2], maxc = hdr[3];
  if ((hdr[0] != 1 && hdr[0] != 2) || n_mat < 1 || n_mat > ORC_MAXMAT || n_E < 2 || maxc != ORC_MAXCOMP) {
    fclose(f);
    return ORC_EIO;
  }
  c->n_mat = n_mat; c->n_E = n_E; c->E0 = e[0]; c->dE = e[1];
  c->r0 = k[0]; c->mec2 = k[1]; c->hc = k[2]; c->NA = k[3]; c->cF = k[4]; c->Kpe = k[5];
  for (int m = 0; m < n_mat; ++m) {
    char name[16];
    double dens;
    int32_t nc[2];
    double buf[ORC_MAXCOMP * 3];
    if (fread(name, 1, 16, f) != 16 || fread(&dens, 8, 1, f) != 1 || fread(nc, 4, 2, f) != 2 ||
        fread(buf, 8, ORC_MAXCOMP * 3, f) != ORC_MAXCOMP * 3 || nc[0] < 1 || nc[0] > ORC_MAXCOMP) {
      fclose(f);
      return ORC_EIO;
    }
    c->density[m] = dens;
    c->n_comp[m] = nc[0];
    for (int i = 0; i < ORC_MAXCOMP; ++i)
      for (int j = 0; j < 3; ++j) c->comp[m][i][j] = buf[i * 3 + j];
  }
  size_t n = (size_t)n_mat * n_E;
  free(c->mu_pe); free(c->mu_in); free(c->mu_co); free(c->icoh);
  c->mu_pe = malloc(n * 8); c->mu_in = malloc(n * 8); c->mu_co = malloc(n * 8); c->icoh = malloc(n * 8);
  if (fread(c->mu_pe, 8, n, f) != n || fread(c->mu_in, 8, n, f) != n || fread(c->mu_co, 8, n, f) != n ||
      fread(c->icoh, 8, n, f) != n) {
    fclose(f);
    return ORC_EIO;
  }
  free(c->iincoh);
  c->iincoh = NULL;
  c->bound = hdr[0] == 2;
  if (c->bound) {
    c->iincoh = malloc(n * 8);
    if (fread(c->iincoh, 8, n, f) != n) {
      fclose(f);
      c->bound = 0;
      return ORC_EIO;
    }
  }
  fclose(f);
  c->have_tables = 1;
  return ORC_OK;
}

int orc_load_volume(orc_ctx *c, const uint8_t *mat, const uint16_t *rho16, int nx, int ny, int nz, double dx,
                    double dy, double dz) {
  if (!c->have_tables) return ORC_ESTATE;
  if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0) || !(dz > 0)) return ORC_EINVAL;
  size_t n = (size_t)nx * ny * nz;
  uint8_t *m = malloc(n);
  double *r = malloc(n * 8);
  for (size_t i = 0; i < n; ++i) {
    if (mat[i] >= c->n_mat) {
      free(m); free(r);
      return ORC_EINVAL;
    }
    m[i] = mat[i];
    /* IEEE binary16 -> double, exactly */
    uint16_t hbits = rho16[i];
    int s = hbits >> 15, ex = (hbits >> 10) & 31, fr = hbits & 1023;
    double v;
    if (ex == 0) v = ldexp((double)fr, -24);
    else if (ex == 31) v = NAN;
    else v = ldexp((double)(fr | 1024), ex - 25);
    if (s) v = -v;
    if (!(v >= 0.0) || isinf(v)) {
      free(m); free(r);
      return ORC_EINVAL;
    }
    r[i] = v;
  }
  free(c->mat); free(c->rho);
  c->mat = m; c->rho = r;
  c->nx = nx; c->ny = ny; c->nz = nz; c->dx = dx; c->dy = dy; c->dz = dz;
  c->have_volume = 1;
  c->mesh_active = 0;
  return ORC_OK;
}

int orc_set_spectrum(orc_ctx *c, const double *w, const float *E, int n) {
  if (!c->have_tables) return ORC_ESTATE;
  if (n < 1) return ORC_EINVAL;
  double sum = 0;
  double Emax = c->E0 + c->dE * (c->n_E - 1);
  for (int i = 0; i < n; ++i) {
    if (!(w[i] >= 0.0) || !((double)E[i] >= c->E0) || !((double)E[i] <= Emax)) return ORC_EINVAL;
    sum += w[i];
  }
  if (!(sum > 0)) return ORC_EINVAL;
  free(c->S); free(c->Ebin);
  c->S = malloc(n * 8); c->Ebin = malloc(n * 8);
  for (int i = 0; i < n; ++i) {
    c->S[i] = w[i] / sum;
    c->Ebin[i] = (double)E[i];
  }
  c->n_bins = n;
  c->have_spectrum = 1;
  return ORC_OK;
}

/* eta[n_E]: detector response at the table's energy nodes (keV per photon), or
 * NULL for eta(E) = E.  Values must be finite and >= 0. */
int orc_set_detector_response(orc_ctx *c, const double *eta, int n) {
  if (!c->have_tables) return ORC_ESTATE;
  if (!eta) {
    free(c->eta);
    c->eta = NULL;
    return ORC_OK;
  }
  if (n != c->n_E) return ORC_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!(eta[i] >= 0.0) || !isfinite(eta[i])) return ORC_EINVAL;
  double *e = malloc((size_t)n * sizeof(double));
  if (!e) return ORC_EINVAL;
  memcpy(e, eta, (size_t)n * sizeof(double));
  free(c->eta);
  c->eta = e;
  return ORC_OK;
}

int orc_set_geometry(orc_ctx *c, double sod, double sdd, int nu, int nv, double pu, double pv) {
  if (!(sod > 0) || !(sdd > sod) || nu < 1 || nv < 1 || !(pu > 0) || !(pv > 0)) return ORC_EINVAL;
  c->sod = sod; c->sdd = sdd; c->nu = nu; c->nv = nv; c->pu = pu; c->pv = pv;
  c->have_geometry = 1;
  return ORC_OK;
}

/* Point-detector scoring mode.  0 (the paper's): at a Compton or Rayleigh
 * interaction, score that type's scatter-toward-detector pdf.  1 (expected
 * value over the interaction type): at every interaction, whatever type is
 * then sampled for the photon's own continuation, score
 * (mu_incoh/mu) x Compton term at E' + (mu_coh/mu) x Rayleigh term at E --
 * the expectation of mode 0's score over the type draw, so the same mean with
 * less variance. */
/* Doppler broadening of incoherent scatter on (1) or off (0); it needs the
 * bound-electron tables (their orbital model). */
int orc_set_doppler(orc_ctx *c, int on) {
  if (on != 0 && on != 1) return ORC_EINVAL;
  if (on && (!c->have_tables || !c->bound)) return ORC_ESTATE;
  c->doppler = on;
  return ORC_OK;
}

static double sample_doppler(const orc_ctx *c, rng_t *g, int m, double E, double cos_t, int *fail);

/* E'/E of one Doppler-broadened incoherent scatter of energy E through cos_t
 * in material m (stream h = i, for the sampler tests). */
int orc_sample_doppler(const orc_ctx *c, int m, double E, double cos_t, uint64_t n, uint64_t seed, double *out) {
  if (!c->have_tables || !c->bound || m < 0 || m >= c->n_mat) return ORC_ESTATE;
  for (uint64_t i = 0; i < n; ++i) {
    rng_t g;
    rng_init(&g, i, 0, seed);
    int fail = 0;
    out[i] = sample_doppler(c, &g, m, E, cos_t, &fail);
    if (fail) return ORC_EINVAL;
  }
  return ORC_OK;
}

int orc_set_nee_mode(orc_ctx *c, int mode) {
  if (mode != 0 && mode != 1) return ORC_EINVAL;
  c->nee_mode = mode;
  return ORC_OK;
}

/* Forced detection (named among the variance-reduction techniques in Sec. I):
 * every scatter interaction scores every pixel of the panel -- or of the
 * history's tile under tile-stratified scoring -- exactly once, pixel s taking
 * the s-th pseudo-particle's counter block (its first word unused) for a
 * uniform point inside the pixel, with weight 1 in place of P / n_split.  It is
 * the split estimator of eq. (Th) with the pixel choice stratified instead of
 * drawn, so each pixel receives the same expected score and the pixel choice
 * adds no variance. */
int orc_set_forced(orc_ctx *c, int on) {
  if (on != 0 && on != 1) return ORC_EINVAL;
  c->forced = on;
  return ORC_OK;
}

/* Tile-stratified point-detector scoring: the panel is cut into tiles of
 * tile_u x tile_v pixels (ragged at the far edges), T tiles in all; history h
 * aims all its pseudo-particles at tile t = (h + o) mod T, at pixels drawn
 * uniformly within it (probability 1/P_t instead of 1/P), and its scores
 * carry the factor T.  The offset o is uniform on [0, T), one per run and
 * angle, from the Philox block (2^32 - 1, angle, 2^32 - 1, 2^32 - 1) (above
 * every history's blocks), so each energy bin's consecutive histories start
 * at a uniformly random tile: a tile receives M_n / T of bin n's histories in
 * expectation, whatever M_n, and every pixel receives in expectation what the
 * unstratified estimator gives it.  tile_u = tile_v = 0 turns it off; one tile
 * covering the panel reduces exactly to the unstratified estimator. */
int orc_set_tiles(orc_ctx *c, int tile_u, int tile_v) {
  if (tile_u < 0 || tile_v < 0 || (tile_u == 0) != (tile_v == 0)) return ORC_EINVAL;
  c->tile_u = tile_u;
  c->tile_v = tile_v;
  return ORC_OK;
}

int orc_set_options(orc_ctx *c, int n_split, double rr_threshold, int max_order, double eps_face) {
  if (n_split < 1 || max_order < 1 || rr_threshold < 0) return ORC_EINVAL;
  c->n_split = n_split;
  c->rr_threshold = rr_threshold;
  c->max_order = max_order;
  if (eps_face > 0) c->eps_face = eps_face;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* tables: linear in E between nodes */
static void interp_idx(const orc_ctx *c, double E, int *i, double *f) {
  double x = (E - c->E0) / c->dE;
  int k = (int)floor(x);
  if (k < 0) k = 0;
  if (k > c->n_E - 2) k = c->n_E - 2;
  *i = k;
  *f = x - k;
}
static double tab(const orc_ctx *c, const double *a, int m, double E) {
  int i;
  double f;
  interp_idx(c, E, &i, &f);
  const double *row = a + (size_t)m * c->n_E;
  return row[i] + f * (row[i + 1] - row[i]);
}
/* Detector response (Sec. II-D.2): the signal of a photon of energy E reaching
 * the panel; eta(E) = E (energy integrating) unless a response table was set,
 * which is then interpolated linearly between the table's nodes. */
static double det_eta(const orc_ctx *c, double E) {
  if (!c->eta) return E;
  int i;
  double f;
  interp_idx(c, E, &i, &f);
  return c->eta[i] + f * (c->eta[i + 1] - c->eta[i]);
}

/* total mass attenuation, cm^2/g */
static double mu_rho_tot(const orc_ctx *c, int m, double E) {
  return tab(c, c->mu_pe, m, E) + tab(c, c->mu_in, m, E) + tab(c, c->mu_co, m, E);
}

/* Klein-Nishina total cross section per electron divided by pi r0^2
 * (closed form of int_{-1}^{1} (a'/a)^2 (a'/a + a/a' - sin^2) dmu), with
 * its Taylor series where the closed form cancels. */
double orc_kn_norm(double E, double mec2) {
  double k = E / mec2;
  if (k < 1e-3) {
    /* 8/3 (1 - 2k + 26/5 k^2 - 133/10 k^3 + 1144/35 k^4) */
    return 8.0 / 3.0 * (1.0 - 2.0 * k + 5.2 * k * k - 13.3 * k * k * k + 1144.0 / 35.0 * k * k * k * k);
  }
  double l = log1p(2.0 * k);
  double a = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / (1.0 + 2.0 * k) - l / k);
  double b = l / (2.0 * k);
  double d = (1.0 + 3.0 * k) / ((1.0 + 2.0 * k) * (1.0 + 2.0 * k));
  return 2.0 * (a + b - d);
}

/* Molecular F^2 = sum_i w_i Z_i^2 / (1 + b_i x^2)^4 at x^2 = u (A^-2). */
static double ff2(const orc_ctx *c, int m, double u) {
  double s = 0;
  for (int i = 0; i < c->n_comp[m]; ++i) {
    double Z = c->comp[m][i][0], w = c->comp[m][i][1], b = c->comp[m][i][2];
    double q = 1.0 + b * u;
    double q2 = q * q;
    s += w * Z * Z / (q2 * q2);
  }
  return s;
}

/* Molecular incoherent scattering function at x^2 = u (A^-2), per gram in
 * moles of electrons: sum_i w_i Z_i (1 - (1 + b_i u)^-4) -- the Waller-Hartree
 * form for Z_i electrons sharing the orbital factor of the form factor above.
 * Its large-u limit is sum_i w_i Z_i. */
static double smol(const orc_ctx *c, int m, double u) {
  double s = 0;
  for (int i = 0; i < c->n_comp[m]; ++i) {
    double Z = c->comp[m][i][0], w = c->comp[m][i][1], b = c->comp[m][i][2];
    double q = 1.0 + b * u;
    double q2 = q * q;
    s += w * Z * (1.0 - 1.0 / (q2 * q2));
  }
  return s;
}
static double smol_max(const orc_ctx *c, int m) {
  double s = 0;
  for (int i = 0; i < c->n_comp[m]; ++i) s += c->comp[m][i][1] * c->comp[m][i][0];
  return s;
}

/* Scatter-toward-detector pdf over lambda in [-1, 1] (integrates to one):
 * type 1 Compton, eq. (pmueforIncoherent) with S = 1, normalised by the KN total;
 * type 2 Rayleigh, eq. (pmueforcoherent), normalised by the tabulated I_coh(E).
 * Returns p and, for Compton, the scattered energy in *Eout. */
double orc_nee_pdf(const orc_ctx *c, int type, int m, double E, double lam, double *Eout) {
  if (type == 1) {
    double a = E / c->mec2;
    double ratio = 1.0 / (1.0 + a * (1.0 - lam));
    if (Eout) *Eout = E * ratio;
    double shape = ratio * ratio * (ratio + 1.0 / ratio - 1.0 + lam * lam);
    if (c->bound) { /* KN x S_mol, normalised by I_incoh(E) */
      double K = (E / c->hc) * (E / c->hc);
      return shape * smol(c, m, 0.5 * K * (1.0 - lam)) / tab(c, c->iincoh, m, E);
    }
    return shape / orc_kn_norm(E, c->mec2);
  }
  if (Eout) *Eout = E;
  double K = (E / c->hc) * (E / c->hc);
  double u = 0.5 * K * (1.0 - lam);
  return (1.0 + lam * lam) * ff2(c, m, u) / tab(c, c->icoh, m, E);
}

/* Kahn's rejection method for the Klein-Nishina distribution (S = 1).
 * r = E/E' in [1, 1 + 2a].  Returns cos(theta); *ratio = r. */
static double sample_compton(rng_t *g, double E, double mec2, double *ratio, int *fail) {
  double a = E / mec2;
  for (int it = 0; it < 100000; ++it) {
    double u1 = rng_u(g), u2 = rng_u(g), u3 = rng_u(g);
    double r;
    int acc;
    if (u1 <= (1.0 + 2.0 * a) / (9.0 + 2.0 * a)) {
      r = 1.0 + 2.0 * a * u2;
      acc = u3 <= 4.0 * (1.0 / r - 1.0 / (r * r));
    } else {
      r = (1.0 + 2.0 * a) / (1.0 + 2.0 * a * u2);
      double mu = 1.0 - (r - 1.0) / a;
      acc = u3 <= 0.5 * (mu * mu + 1.0 / r);
    }
    if (acc) {
      *ratio = r;
      return 1.0 - (r - 1.0) / a;
    }
  }
  *fail = 1;
  *ratio = 1.0;
  return 1.0;
}

/* Doppler broadening of incoherent scattering (impulse approximation).  Each
 * element's electrons share the hydrogen-like orbital behind the form factor
 * F_i = Z_i (1 + b_i x^2)^-2, whose exponent is zeta_i = 2 pi a0 / sqrt(b_i)
 * (atomic units) and whose Compton profile is
 * J_i(p_z) = 8 / (3 pi zeta_i) (1 + (p_z / zeta_i)^2)^-3.  A scatter through
 * cos(theta) = c picks element i with probability w_i S_i(x) / S_mol(x), draws
 * p_z from J_i (Cauchy proposal t = tan(pi (u - 1/2)), accepted with
 * probability (1 + t^2)^-2) and solves the impulse-approximation relation
 * P sqrt(1 + tau^2 - 2 tau c) = tau (1 + kappa (1 - c)) - 1 for tau = E'/E
 * (P = p_z / (m_e c), kappa = E / m_e c^2); a draw without a root in
 * 0 < tau <= 1 is redrawn (the profile is truncated to physical energies). */
static const double ALPHA_FS = 1.0 / 137.035999084; /* CODATA 2018 */
static const double A0_ANGSTROM = 0.529177210903;   /* Bohr radius, CODATA 2018 */

static double doppler_tau(double kappa, double c, double P) {
  const double a = 1.0 + kappa * (1.0 - c);
  const double P2 = P * P;
  const double den = a * a - P2;
  if (!(den > 0)) return 0;
  const double B = a - P2 * c;
  const double D = B * B - den * (1.0 - P2);
  if (!(D >= 0)) return 0;
  const double t = (B + (P >= 0 ? 1.0 : -1.0) * sqrt(D)) / den;
  if (!(t > 0 && t <= 1.0)) return 0;
  if (P != 0 && (a * t - 1.0) * P < 0) return 0; /* root of the squared equation only */
  return t;
}

static double sample_doppler(const orc_ctx *c, rng_t *g, int m, double E, double cos_t, int *fail) {
  const double K = (E / c->hc) * (E / c->hc);
  const double u = 0.5 * K * (1.0 - cos_t);
  const double kappa = E / c->mec2;
  const double smax = smol(c, m, u);
  for (int it = 0; it < 256; ++it) {
    const double ue = rng_u(g) * smax, uc = rng_u(g), ua = rng_u(g);
    int el = c->n_comp[m] - 1;
    double cum = 0;
    for (int i = 0; i < c->n_comp[m]; ++i) {
      const double Z = c->comp[m][i][0], w = c->comp[m][i][1], b = c->comp[m][i][2];
      const double q = 1.0 + b * u, q2 = q * q;
      cum += w * Z * (1.0 - 1.0 / (q2 * q2));
      if (ue < cum) {
        el = i;
        break;
      }
    }
    const double t = tan(PI * (uc - 0.5));
    const double w1 = 1.0 + t * t;
    if (ua * w1 * w1 > 1.0) continue; /* Cauchy -> (1 + t^2)^-3 */
    const double zeta = 2.0 * PI * A0_ANGSTROM / sqrt(c->comp[m][el][2]);
    const double tau = doppler_tau(kappa, cos_t, t * zeta * ALPHA_FS);
    if (tau > 0) return tau;
  }
  *fail = 1;
  return 1.0 / (1.0 + kappa * (1.0 - cos_t));
}

/* Side stream of pseudo-particle s of an interaction whose pseudo-particle
 * blocks start at k0: counter (2^31 | (k0 + s) << 6 | j, angle, h_lo, h_hi),
 * j = 0, 1, ... (disjoint from every history's own blocks). */
static void rng_side(rng_t *d, const rng_t *g, uint32_t k0s) {
  *d = *g;
  d->ctr[0] = 0x80000000u | (k0s << 6);
  d->idx = 4;
}

/* Incoherent scattering with the scattering function: Kahn's method for the
 * Klein-Nishina factor, then acceptance with probability S_mol(x)/S_mol(inf)
 * (one more draw per try); a rejected angle restarts Kahn's method. */
static double sample_incoherent(const orc_ctx *c, rng_t *g, int m, double E, double *ratio, int *fail) {
  if (!c->bound) return sample_compton(g, E, c->mec2, ratio, fail);
  const double K = (E / c->hc) * (E / c->hc);
  const double smax = smol_max(c, m);
  for (int it = 0; it < 100000; ++it) {
    double mu = sample_compton(g, E, c->mec2, ratio, fail);
    if (*fail) return mu;
    if (rng_u(g) * smax <= smol(c, m, 0.5 * K * (1.0 - mu))) return mu;
  }
  *fail = 1;
  *ratio = 1.0;
  return 1.0;
}

/* Rayleigh: pick a form-factor component with probability proportional to
 * w_i Z_i^2 G_i(K), invert u = x^2 on (1 + b_i u)^-4 over [0, K], take
 * mu = 1 - 2u/K and accept with probability (1 + mu^2)/2. */
static double sample_rayleigh(const orc_ctx *c, rng_t *g, int m, double E, int *fail) {
  double K = (E / c->hc) * (E / c->hc);
  double G[ORC_MAXCOMP], tot = 0;
  int nc = c->n_comp[m];
  for (int i = 0; i < nc; ++i) {
    double Z = c->comp[m][i][0], w = c->comp[m][i][1], b = c->comp[m][i][2];
    double T = 1.0 + b * K;
    G[i] = w * Z * Z * (1.0 - 1.0 / (T * T * T)) / (3.0 * b);
    tot += G[i];
  }
  for (int it = 0; it < 100000; ++it) {
    double u1 = rng_u(g), u2 = rng_u(g), u3 = rng_u(g);
    int i = 0;
    double acc = G[0];
    while (i < nc - 1 && !(u1 * tot < acc)) {
      ++i;
      acc += G[i];
    }
    double b = c->comp[m][i][2];
    double T = 1.0 + b * K;
    double q = 1.0 - u2 * (1.0 - 1.0 / (T * T * T));
    double u = (pow(q, -1.0 / 3.0) - 1.0) / b;
    double mu = 1.0 - 2.0 * u / K;
    if (mu < -1.0) mu = -1.0;
    if (u3 <= 0.5 * (1.0 + mu * mu)) return mu;
  }
  *fail = 1;
  return 1.0;
}

/* Rotate unit vector w by polar cosine ct and azimuth phi. */
static void rotate(double w[3], double ct, double phi) {
  double st = sqrt(fmax(0.0, 1.0 - ct * ct));
  double cp = cos(phi), sp = sin(phi);
  double x = w[0], y = w[1], z = w[2], nx, ny, nz;
  if (fabs(z) > 0.99999) {
    nx = st * cp;
    ny = st * sp;
    nz = (z > 0 ? ct : -ct);
  } else {
    double s = sqrt(1.0 - z * z);
    nx = x * ct + st * (x * z * cp - y * sp) / s;
    ny = y * ct + st * (y * z * cp + x * sp) / s;
    nz = z * ct - st * s * cp;
  }
  double n = sqrt(nx * nx + ny * ny + nz * nz);
  w[0] = nx / n; w[1] = ny / n; w[2] = nz / n;
}

/* ------------------------------------------------------------------ */
/* geometry */
typedef struct {
  double s[3], c[3], eu[3], ev[3], n[3];
} pose_t;
static void pose(const orc_ctx *c, double beta, pose_t *p) {
  double cb = cos(beta), sb = sin(beta);
  p->s[0] = c->sod * cb; p->s[1] = c->sod * sb; p->s[2] = 0;
  p->c[0] = (c->sod - c->sdd) * cb; p->c[1] = (c->sod - c->sdd) * sb; p->c[2] = 0;
  p->eu[0] = -sb; p->eu[1] = cb; p->eu[2] = 0;
  p->ev[0] = 0; p->ev[1] = 0; p->ev[2] = 1;
  p->n[0] = cb; p->n[1] = sb; p->n[2] = 0;
}
/* Detector point at continuous pixel coordinates (a, b), pixel (i, j) spanning [i, i+1) x [j, j+1). */
static void det_point(const orc_ctx *c, const pose_t *p, double a, double b, double out[3]) {
  double ou = (a - 0.5 * c->nu) * c->pu, ov = (b - 0.5 * c->nv) * c->pv;
  for (int k = 0; k < 3; ++k) out[k] = p->c[k] + ou * p->eu[k] + ov * p->ev[k];
}

/* Slab clip of p0 + t w, t in [t0, t1], to the volume box. */
static int clip_box(const orc_ctx *c, const double p0[3], const double w[3], double t0, double t1, double *ta,
                    double *tb) {
  double half[3] = {0.5 * c->nx * c->dx, 0.5 * c->ny * c->dy, 0.5 * c->nz * c->dz};
  double a = t0, b = t1;
  for (int k = 0; k < 3; ++k) {
    if (w[k] == 0.0) {
      if (p0[k] < -half[k] || p0[k] > half[k]) return 0;
    } else {
      double u = (-half[k] - p0[k]) / w[k], v = (half[k] - p0[k]) / w[k];
      if (u > v) { double t = u; u = v; v = t; }
      if (u > a) a = u;
      if (v < b) b = v;
    }
  }
  *ta = a;
  *tb = b;
  return b > a;
}

static size_t voxel_of(const orc_ctx *c, const double p[3], int ijk[3]) {
  double lo[3] = {-0.5 * c->nx * c->dx, -0.5 * c->ny * c->dy, -0.5 * c->nz * c->dz};
  double d[3] = {c->dx, c->dy, c->dz};
  int n[3] = {c->nx, c->ny, c->nz};
  for (int k = 0; k < 3; ++k) {
    int i = (int)floor((p[k] - lo[k]) / d[k]);
    if (i < 0) i = 0;
    if (i > n[k] - 1) i = n[k] - 1;
    ijk[k] = i;
  }
  return ((size_t)ijk[2] * c->ny + ijk[1]) * c->nx + ijk[0];
}

/* Fixed-step march (Sec. II-C.2): the clipped chord [ta, tb] is cut into
 * n = ceil(L/step) equal steps of length h = L/n; each step takes the
 * material and density of the voxel holding its midpoint.  Accumulates
 * rho*h per material into rhoL (g/cm^3 * mm).  If bound != NULL, adds for
 * every midpoint within eps_face*voxel of a face, edge or corner whose other
 * voxels differ the largest possible change of rho*mu_rho*h at energy Eb (an
 * ambiguity bound for FP32 re-evaluation); sets *namb if L/step is within 1e-5
 * of an integer.
 * Returns the number of steps. */
static long march_rhoL_n(const orc_ctx *c, const double p0[3], const double w[3], double t0, double t1, double step,
                         double *rhoL, double *bound, double Eb, int *namb, long n_force) {
  double ta, tb;
  if (!clip_box(c, p0, w, t0, t1, &ta, &tb)) return 0;
  double L = tb - ta;
  double q = L / step;
  long n = (long)ceil(q);
  if (n < 1) n = 1;
  if (n_force > 0) n = n_force;
  if (namb) {
    double fr = q - floor(q + 0.5);
    if (fabs(fr) < 1e-5 * (q > 1 ? q : 1)) *namb = 1;
  }
  double h = L / n;
  double lo[3] = {-0.5 * c->nx * c->dx, -0.5 * c->ny * c->dy, -0.5 * c->nz * c->dz};
  double dv[3] = {c->dx, c->dy, c->dz};
  int nn[3] = {c->nx, c->ny, c->nz};
  for (long k = 0; k < n; ++k) {
    double t = ta + (k + 0.5) * h;
    double p[3] = {p0[0] + t * w[0], p0[1] + t * w[1], p0[2] + t * w[2]};
    int ijk[3];
    size_t v = voxel_of(c, p, ijk);
    rhoL[c->mat[v]] += c->rho[v] * h;
    if (bound) {
      /* the voxels an FP32 re-evaluation may pick instead: those reached by
       * stepping across any subset of the faces this midpoint lies within
       * eps_face of (a face, an edge or a corner neighbour); the largest change
       * of rho mu h among them that differs from this voxel */
      double mu_here = c->rho[v] * mu_rho_tot(c, c->mat[v], Eb) * 0.1;
      int nb[3];
      for (int a = 0; a < 3; ++a) {
        double x = (p[a] - lo[a]) / dv[a];
        double fr = x - floor(x);
        nb[a] = -1;
        if (fr < c->eps_face) nb[a] = ijk[a] - 1;
        else if (fr > 1.0 - c->eps_face) nb[a] = ijk[a] + 1;
        /* a neighbour index outside the volume, or equal to the clamped index, is no other voxel */
        if (nb[a] < 0 || nb[a] >= nn[a] || nb[a] == ijk[a]) nb[a] = -1;
      }
      double worst = 0;
      for (int sub = 1; sub < 8; ++sub) {
        int j2[3] = {ijk[0], ijk[1], ijk[2]}, ok = 1;
        for (int a = 0; a < 3; ++a)
          if (sub >> a & 1) {
            if (nb[a] < 0) ok = 0;
            else j2[a] = nb[a];
          }
        if (!ok) continue;
        size_t v2 = ((size_t)j2[2] * c->ny + j2[1]) * c->nx + j2[0];
        if (c->mat[v2] != c->mat[v] || c->rho[v2] != c->rho[v]) {
          double mu2 = c->rho[v2] * mu_rho_tot(c, c->mat[v2], Eb) * 0.1;
          double dlt = fabs(mu2 - mu_here) * h;
          if (dlt > worst) worst = dlt;
        }
      }
      *bound += worst;
    }
  }
  return n;
}

static long march_rhoL(const orc_ctx *c, const double p0[3], const double w[3], double t0, double t1, double step,
                       double *rhoL, double *bound, double Eb, int *namb) {
  return march_rhoL_n(c, p0, w, t0, t1, step, rhoL, bound, Eb, namb, 0);
}

/* Optical depth tau at energy E along the march (mm^-1 * mm). */
static double march_tau(const orc_ctx *c, const double p0[3], const double w[3], double t0, double t1, double step,
                        double E, long *nsteps) {
  double rhoL[ORC_MAXMAT] = {0};
  long n = march_rhoL(c, p0, w, t0, t1, step, rhoL, NULL, 0, NULL);
  if (nsteps) *nsteps += n;
  double tau = 0;
  for (int m = 0; m < c->n_mat; ++m)
    if (rhoL[m] != 0) tau += mu_rho_tot(c, m, E) * 0.1 * rhoL[m];
  return tau;
}

/* Exported march for tests: tau at energy E and per-material rho*L. */
int orc_march(const orc_ctx *c, const double p0[3], const double w[3], double t0, double t1, double step, double E,
              double *tau, double *rhoL_out, double *bound, long *nsteps) {
  if (!c->have_volume) return ORC_ESTATE;
  double rhoL[ORC_MAXMAT] = {0};
  double b = 0;
  int namb = 0;
  long n = march_rhoL(c, p0, w, t0, t1, step, rhoL, &b, E, &namb);
  double t = 0;
  for (int m = 0; m < c->n_mat; ++m) {
    if (rhoL[m] != 0) t += mu_rho_tot(c, m, E) * 0.1 * rhoL[m];
    if (rhoL_out) rhoL_out[m] = rhoL[m];
  }
  *tau = t;
  if (bound) *bound = namb ? INFINITY : b;
  if (nsteps) *nsteps = n;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Spectrum sum of eq. (Ip) for per-material column masses rhoL; also the
 * transmitted-energy-weighted mean optical depth. */
static double primary_sum(const orc_ctx *c, const double *rhoL, double *tau_mean) {
  double sum = 0, wtau = 0;
  for (int n = 0; n < c->n_bins; ++n) {
    if (c->S[n] == 0) continue;
    double tau = 0;
    for (int m = 0; m < c->n_mat; ++m)
      if (rhoL[m] != 0) tau += mu_rho_tot(c, m, c->Ebin[n]) * 0.1 * rhoL[m];
    double e = c->S[n] * det_eta(c, c->Ebin[n]) * exp(-tau);
    sum += e;
    wtau += e * tau;
  }
  if (tau_mean) *tau_mean = sum > 0 ? wtau / sum : 0;
  return sum;
}

/* Primary image, eq. (Ip), one angle.  Ip[j*nu + i] in keV per pixel per source
 * photon into 4 pi.  bound[] (nullable) is, as an optical depth, what a
 * re-evaluation in FP32 may legitimately change: midpoints within eps_face of
 * a face between different voxels may fall on either side (largest optical
 * depth change at the lowest spectrum energy); the chord length carries an FP32
 * rounding of a few units in the last place of the larger ray parameter; and
 * where ceil(L/step) itself is within rounding of an integer, either
 * neighbouring step count is a valid evaluation (largest |ln| ratio of the
 * images they give). */
/* ------------------------------------------------------------------ */
/* Triangle-mesh geometry (the paper's CAD model of closed triangulated
 * surfaces).  Bodies are closed, outward-oriented surfaces with a material
 * and density, optionally inside a parent body whose material they replace;
 * outside every body is vacuum. */
int orc_load_mesh(orc_ctx *c, const float *v, int nv, const int *tris, const int *tri_body, int nt,
                  const int *body_mat, const float *body_rho, const int *body_parent, int nb) {
  if (!c->have_tables) return ORC_ESTATE;
  if (!v || !tris || !tri_body || nv < 3 || nt < 1 || nb < 1 || nb > ORC_MAXBODY) return ORC_EINVAL;
  for (int b = 0; b < nb; ++b)
    if (body_mat[b] < 0 || body_mat[b] >= c->n_mat || !(body_rho[b] >= 0) || body_parent[b] >= b ||
        body_parent[b] < -1)
      return ORC_EINVAL;
  double *t = malloc((size_t)nt * 9 * sizeof(double));
  int *tb = malloc((size_t)nt * sizeof(int));
  if (!t || !tb) {
    free(t); free(tb);
    return ORC_EINVAL;
  }
  for (int k = 0; k < nt; ++k) {
    if (tri_body[k] < 0 || tri_body[k] >= nb) {
      free(t); free(tb);
      return ORC_EINVAL;
    }
    tb[k] = tri_body[k];
    for (int q = 0; q < 3; ++q) {
      int i = tris[3 * k + q];
      if (i < 0 || i >= nv) {
        free(t); free(tb);
        return ORC_EINVAL;
      }
      for (int a = 0; a < 3; ++a) t[9 * k + 3 * q + a] = (double)v[3 * i + a];
    }
  }
  free(c->tri); free(c->tri_body);
  c->tri = t;
  c->tri_body = tb;
  c->n_tri = nt;
  c->n_body = nb;
  for (int b = 0; b < nb; ++b) {
    c->body_mat[b] = body_mat[b];
    c->body_rho[b] = (double)body_rho[b];
    c->body_parent[b] = body_parent[b];
  }
  double r2 = 0;
  for (int i = 0; i < nv; ++i) {
    const double q = (double)v[3 * i] * v[3 * i] + (double)v[3 * i + 1] * v[3 * i + 1];
    if (q > r2) r2 = q;
  }
  c->mesh_rxy = sqrt(r2);
  c->have_mesh = 1;
  c->mesh_active = 1;
  return ORC_OK;
}

/* Watertight ray/triangle test (Woop, Benthin and Wald, JCGT 2013): the
 * triangle is sheared into the ray's frame (kz the dominant axis of dir) and
 * the three edge functions U, V, W of the origin are evaluated; an edge
 * function exactly zero counts as inside for only one of the two triangles
 * that share the edge (half-open rule on the edge's projected direction,
 * normalised by the triangle's facing), so a ray through an edge or a vertex
 * crosses the surface exactly once.  Returns 1 and the ray parameter *t on a
 * hit. */
static int edge_incl(double ex, double ey) { return ey > 0 || (ey == 0 && ex < 0); }
typedef struct {
  int kx, ky, kz;
  double Sx, Sy, Sz;
} shear_t;
static void shear_of(const double dir[3], shear_t *h) {
  int kz = 0;
  if (fabs(dir[1]) > fabs(dir[kz])) kz = 1;
  if (fabs(dir[2]) > fabs(dir[kz])) kz = 2;
  int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
  if (dir[kz] < 0) { int tmp = kx; kx = ky; ky = tmp; }
  h->kx = kx; h->ky = ky; h->kz = kz;
  h->Sx = dir[kx] / dir[kz];
  h->Sy = dir[ky] / dir[kz];
  h->Sz = 1.0 / dir[kz];
}
static int ray_tri(const double org[3], const shear_t *h, const double *tv, double *t) {
  double A[3], B[3], C[3];
  for (int i = 0; i < 3; ++i) {
    A[i] = tv[i] - org[i];
    B[i] = tv[3 + i] - org[i];
    C[i] = tv[6 + i] - org[i];
  }
  const double Ax = A[h->kx] - h->Sx * A[h->kz], Ay = A[h->ky] - h->Sy * A[h->kz];
  const double Bx = B[h->kx] - h->Sx * B[h->kz], By = B[h->ky] - h->Sy * B[h->kz];
  const double Cx = C[h->kx] - h->Sx * C[h->kz], Cy = C[h->ky] - h->Sy * C[h->kz];
  const double U = Cx * By - Cy * Bx, V = Ax * Cy - Ay * Cx, W = Bx * Ay - By * Ax;
  const double det = U + V + W;
  if (det == 0) return 0;
  const double sg = det > 0 ? 1.0 : -1.0;
  if (!(sg * U > 0 || (U == 0 && edge_incl(sg * (Cx - Bx), sg * (Cy - By))))) return 0;
  if (!(sg * V > 0 || (V == 0 && edge_incl(sg * (Ax - Cx), sg * (Ay - Cy))))) return 0;
  if (!(sg * W > 0 || (W == 0 && edge_incl(sg * (Bx - Ax), sg * (By - Ay))))) return 0;
  const double T = h->Sz * (U * A[h->kz] + V * B[h->kz] + W * C[h->kz]);
  *t = T / det;
  return 1;
}

/* Per-material column masses rho*L (g/cm^3 x mm) along x + t w, t in (0, t1):
 * every crossing of body b's surface adds sign x t to its inside length
 * (+ on leaving, - on entering, t measured from x: crossings of a closed
 * surface alternate, so the sum is the length inside it, also when x itself
 * is inside), and the body's material replaces its parent's there.  The ray
 * is tested from the point closest to the origin, which keeps the
 * parameters small. */
static long mesh_rhoL(const orc_ctx *c, const double x[3], const double w[3], double t1, double *rhoL) {
  long ncross = 0;
  double t0 = -(x[0] * w[0] + x[1] * w[1] + x[2] * w[2]);
  double org[3] = {x[0] + t0 * w[0], x[1] + t0 * w[1], x[2] + t0 * w[2]};
  shear_t h;
  shear_of(w, &h);
  double Lb[ORC_MAXBODY] = {0};
  for (int k = 0; k < c->n_tri; ++k) {
    double t;
    const double *tv = c->tri + 9 * k;
    if (!ray_tri(org, &h, tv, &t)) continue;
    if (!(t + t0 > 0 && t + t0 < t1)) continue;
    double e1[3] = {tv[3] - tv[0], tv[4] - tv[1], tv[5] - tv[2]};
    double e2[3] = {tv[6] - tv[0], tv[7] - tv[1], tv[8] - tv[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double dn = n[0] * w[0] + n[1] * w[1] + n[2] * w[2];
    Lb[c->tri_body[k]] += dn > 0 ? t + t0 : -(t + t0);
    ++ncross;
  }
  for (int b = 0; b < c->n_body; ++b) {
    if (Lb[b] == 0) continue;
    rhoL[c->body_mat[b]] += c->body_rho[b] * Lb[b];
    const int pb = c->body_parent[b];
    if (pb >= 0) rhoL[c->body_mat[pb]] -= c->body_rho[pb] * Lb[b];
  }
  return ncross;
}

/* One surface crossing of a half-line: its parameter and triangle. */
typedef struct {
  double t;
  int tri;
} crossing_t;
static int cmp_crossing(const void *pa, const void *pb) {
  const crossing_t *a = pa, *b = pb;
  if (a->t != b->t) return a->t < b->t ? -1 : 1;
  return a->tri < b->tri ? -1 : (a->tri > b->tri);
}

/* Free flight through the mesh with exact path lengths (the CAD model's ray
 * tracing, Sec. II-A).  Every crossing of the half-line x + t w, t > 0, is
 * collected (buf holds n_tri entries) and sorted by t.  Body b contains x when
 * the half-line crosses its closed surface an odd number of times, so the
 * start medium follows from the crossings themselves; each crossing then
 * toggles its body, and the medium is the deepest body containing the point
 * (a parent precedes its children: the highest index present).  Inside body
 * b the optical depth grows by rho_b mu/rho(m_b, E) per unit length.  Returns
 * 1 with the interaction distance *tint and material *mint when the depth
 * reaches tau_star, 0 after the last crossing (escape: outside every closed
 * surface); *nseg += the segments walked. */
static int mesh_flight(const orc_ctx *c, crossing_t *buf, const double x[3], const double w[3], double E,
                       double tau_star, double *tint, int *mint, long *nseg) {
  double t0 = -(x[0] * w[0] + x[1] * w[1] + x[2] * w[2]);
  double org[3] = {x[0] + t0 * w[0], x[1] + t0 * w[1], x[2] + t0 * w[2]};
  shear_t h;
  shear_of(w, &h);
  int n = 0;
  uint64_t inside = 0;
  for (int k = 0; k < c->n_tri; ++k) {
    double t;
    if (!ray_tri(org, &h, c->tri + 9 * k, &t)) continue;
    t += t0;
    if (!(t > 0)) continue;
    buf[n].t = t;
    buf[n].tri = k;
    ++n;
    inside ^= 1ull << c->tri_body[k];
  }
  qsort(buf, n, sizeof(crossing_t), cmp_crossing);
  double tau = 0, tprev = 0;
  for (int i = 0; i <= n; ++i) {
    *nseg += 1;
    if (i == n) break;
    if (inside) {
      int b = 63;
      while (!(inside >> b & 1)) --b;
      const double mu = c->body_rho[b] * mu_rho_tot(c, c->body_mat[b], E) * 0.1;
      const double len = buf[i].t - tprev;
      if (mu > 0 && tau + mu * len >= tau_star) {
        *tint = tprev + (tau_star - tau) / mu;
        *mint = c->body_mat[b];
        return 1;
      }
      tau += mu * len;
    }
    tprev = buf[i].t;
    inside ^= 1ull << c->tri_body[buf[i].tri];
  }
  return 0;
}

/* Optical depth at energy E from x to x + t1 w: the fixed-step march through
 * the volume, or the exact column masses through the mesh. */
static double path_tau(const orc_ctx *c, const double x[3], const double w[3], double t1, double step, double E,
                       long *nsteps) {
  if (!c->mesh_active) return march_tau(c, x, w, 0.0, t1, step, E, nsteps);
  double rhoL[ORC_MAXMAT] = {0};
  *nsteps += mesh_rhoL(c, x, w, t1, rhoL);
  double tau = 0;
  for (int m = 0; m < c->n_mat; ++m)
    if (rhoL[m] != 0) tau += mu_rho_tot(c, m, E) * 0.1 * rhoL[m];
  return tau;
}

/* Primary image of the mesh geometry, eq. (Ip) with exact path lengths. */
int orc_mesh_primary(const orc_ctx *c, double beta, double *Ip) {
  if (!(c->have_tables && c->have_mesh && c->have_spectrum && c->have_geometry)) return ORC_ESTATE;
  pose_t P;
  pose(c, beta, &P);
  for (int j = 0; j < c->nv; ++j)
    for (int i = 0; i < c->nu; ++i) {
      double X[3];
      det_point(c, &P, i + 0.5, j + 0.5, X);
      double D[3] = {X[0] - P.s[0], X[1] - P.s[1], X[2] - P.s[2]};
      double d = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
      double w[3] = {D[0] / d, D[1] / d, D[2] / d};
      double rhoL[ORC_MAXMAT] = {0};
      mesh_rhoL(c, P.s, w, d, rhoL);
      double sum = primary_sum(c, rhoL, NULL);
      Ip[(size_t)j * c->nu + i] = sum * c->pu * c->pv * (c->sdd / d) / (4.0 * PI * d * d);
    }
  return ORC_OK;
}

int orc_primary(const orc_ctx *c, double beta, double step, double *Ip, double *bound) {
  if (!(c->have_tables && c->have_volume && c->have_spectrum && c->have_geometry)) return ORC_ESTATE;
  if (!(step > 0)) return ORC_EINVAL;
  pose_t P;
  pose(c, beta, &P);
  double Emin = 1e30;
  for (int n = 0; n < c->n_bins; ++n)
    if (c->S[n] > 0 && c->Ebin[n] < Emin) Emin = c->Ebin[n];
  for (int j = 0; j < c->nv; ++j) {
    for (int i = 0; i < c->nu; ++i) {
      double X[3];
      det_point(c, &P, i + 0.5, j + 0.5, X);
      double D[3] = {X[0] - P.s[0], X[1] - P.s[1], X[2] - P.s[2]};
      double d = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
      double w[3] = {D[0] / d, D[1] / d, D[2] / d};
      double rhoL[ORC_MAXMAT] = {0};
      double b = 0;
      int namb = 0;
      long n = march_rhoL(c, P.s, w, 0.0, d, step, rhoL, &b, Emin, &namb);
      double sum = primary_sum(c, rhoL, NULL);
      double cosg = c->sdd / d;
      Ip[(size_t)j * c->nu + i] = sum * c->pu * c->pv * cosg / (4.0 * PI * d * d);
      if (bound) {
        /* Allowance for an FP32 re-evaluation of this pixel: the midpoints
         * flagged within eps_face of a face between different voxels (b), and,
         * where ceil(L/step) is within rounding of an integer, the change the
         * neighbouring step count produces.  Nothing is allowed for the chord's
         * own rounding: an evaluation that parameterises the ray from its point
         * nearest the isocentre carries an error of the volume's size there,
         * far below the 1e-5 target. */
        double extra = 0;
        if (namb) {
          for (long dn = -1; dn <= 1; dn += 2) {
            if (n + dn < 1) continue;
            double r2[ORC_MAXMAT] = {0}, b2 = 0;
            march_rhoL_n(c, P.s, w, 0.0, d, step, r2, &b2, Emin, NULL, n + dn);
            double s2 = primary_sum(c, r2, NULL);
            double lr = fabs(log(s2 / sum)) + b2;
            if (lr > extra) extra = lr;
          }
        }
        bound[(size_t)j * c->nu + i] = b + extra;
      }
    }
  }
  return ORC_OK;
}

/* Stratified photon counts per energy bin: M_n = max(1, floor(N S_n)) for
 * S_n > 0, the remainder handed out one by one by largest fractional part
 * (ties to the lower index) among bins not raised to one. */
int orc_stratify(int n_bins, const double *S, uint64_t N, uint64_t *M) {
  uint64_t sum = 0;
  int *elig = malloc(n_bins * sizeof(int));
  double *fr = malloc(n_bins * 8);
  for (int n = 0; n < n_bins; ++n) {
    double x = (double)N * S[n];
    double fl = floor(x);
    elig[n] = 0;
    fr[n] = 0;
    if (S[n] <= 0) {
      M[n] = 0;
    } else if (fl < 1.0) {
      M[n] = 1;
    } else {
      M[n] = (uint64_t)fl;
      elig[n] = 1;
      fr[n] = x - fl;
    }
    sum += M[n];
  }
  if (sum > N) {
    free(elig); free(fr);
    return ORC_EINVAL;
  }
  uint64_t rem = N - sum;
  while (rem > 0) {
    int best = -1;
    for (int n = 0; n < n_bins; ++n)
      if (elig[n] == 1 && (best < 0 || fr[n] > fr[best])) best = n;
    if (best < 0) break;
    M[best] += 1;
    elig[best] = 2;
    --rem;
  }
  free(elig); free(fr);
  return rem == 0 ? ORC_OK : ORC_EINVAL;
}

/* Statistics slots */
enum {
  ST_HIST = 0, ST_FLIGHT_STEPS, ST_NEE_STEPS, ST_NEE_RAYS, ST_PHOTO, ST_COMPTON, ST_RAYLEIGH, ST_ESCAPE,
  ST_MAX_EERR, ST_LIMIT, ST_SAMPLER_FAIL, ST_E_SOURCE, ST_E_DEPOSIT, ST_E_ESCAPE, ST_RR_KILLED, ST_N
};

/* Scatter image by eq. (Is): histories h in [h_begin, h_end) of an N-photon
 * run at angle beta (angle_index keys the random counter).
 *   Is[P]          sum of NEE scores (keV per pixel per source photon);
 *   Is_order[3][P] the same split by scatter order 1, 2, >=3 (nullable);
 *   analog[P]      detector hits of escaping scattered photons (nullable);
 *   analog0[P]     detector hits of unscattered photons (nullable);
 *   stats[ST_N]    counters (see enum). */
int orc_scatter(const orc_ctx *c, double beta, uint32_t angle_index, uint64_t N, uint64_t h_begin, uint64_t h_end,
                double step, uint64_t seed, double *Is, double *Is_order, double *analog, double *analog0,
                double *stats) {
  const int mesh = c->mesh_active;
  if (!(c->have_tables && (mesh || c->have_volume) && c->have_spectrum && c->have_geometry)) return ORC_ESTATE;
  if (!(step > 0) || h_end > N || h_begin > h_end) return ORC_EINVAL;
  /* the object must lie between source and detector */
  double rmax = mesh ? c->mesh_rxy : 0.5 * sqrt(pow(c->nx * c->dx, 2) + pow(c->ny * c->dy, 2));
  if (!(rmax < c->sod) || !(rmax < c->sdd - c->sod)) return ORC_EINVAL;
  crossing_t *xbuf = mesh ? malloc((size_t)c->n_tri * sizeof(crossing_t)) : NULL;
  uint64_t *M = malloc(c->n_bins * sizeof(uint64_t));
  uint64_t *pre = malloc((c->n_bins + 1) * sizeof(uint64_t));
  if (orc_stratify(c->n_bins, c->S, N, M) != ORC_OK) {
    free(M); free(pre); free(xbuf);
    return ORC_EINVAL;
  }
  pre[0] = 0;
  for (int n = 0; n < c->n_bins; ++n) pre[n + 1] = pre[n] + M[n];
  const int tiled = c->tile_u > 0;
  const int ntu = tiled ? (c->nu + c->tile_u - 1) / c->tile_u : 1;
  const int ntv = tiled ? (c->nv + c->tile_v - 1) / c->tile_v : 1;
  const uint64_t T = (uint64_t)ntu * ntv;
  uint64_t tile_off = 0;
  if (tiled) {
    const uint32_t ctr[4] = {0xFFFFFFFFu, angle_index, 0xFFFFFFFFu, 0xFFFFFFFFu};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox(ctr, key, out);
    tile_off = ((uint64_t)out[0] * T) >> 32;
  }
  pose_t P;
  pose(c, beta, &P);
  const size_t npix = (size_t)c->nu * c->nv;
  const double A_det = c->nu * c->pu * c->nv * c->pv;
  const double A_px = c->pu * c->pv;
  double st[ST_N] = {0};
  long nsteps = 0;
  for (uint64_t h = h_begin; h < h_end; ++h) {
    int bin = 0;
    while (bin < c->n_bins - 1 && !(h < pre[bin + 1])) ++bin;
    double E = c->Ebin[bin];
    rng_t g;
    rng_init(&g, h, angle_index, seed);
    /* source: a uniform point on the detector rectangle, weighted by the solid-angle Jacobian */
    double ua = rng_u(&g), ub = rng_u(&g);
    double Q[3];
    det_point(c, &P, ua * c->nu, ub * c->nv, Q);
    double D[3] = {Q[0] - P.s[0], Q[1] - P.s[1], Q[2] - P.s[2]};
    double d = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    double w[3] = {D[0] / d, D[1] / d, D[2] / d};
    double W = c->S[bin] / (double)M[bin] * A_det * (c->sdd / d) / (4.0 * PI * d * d);
    /* the pixels this history's pseudo-particles aim at: the whole panel, or its tile */
    int u0 = 0, v0 = 0, wt = c->nu, ht = c->nv;
    double tile_w = 1.0;
    if (tiled) {
      const uint64_t t = (h % T + tile_off) % T;
      u0 = (int)(t % ntu) * c->tile_u;
      v0 = (int)(t / ntu) * c->tile_v;
      wt = c->nu - u0 < c->tile_u ? c->nu - u0 : c->tile_u;
      ht = c->nv - v0 < c->tile_v ? c->nv - v0 : c->tile_v;
      tile_w = (double)T;
    }
    const uint64_t Pt = (uint64_t)wt * ht;
    double x[3] = {P.s[0], P.s[1], P.s[2]};
    double e_src = E * W, e_dep = 0, e_esc = 0;
    int order = 0;
    st[ST_HIST] += 1;
    for (;;) {
      /* free flight: march until the accumulated optical depth reaches -ln u */
      double tau_star = -log(rng_u(&g));
      double ta, tb;
      int hit = 0;
      double tint = 0;
      int mint = 0;
      if (mesh) {
        long nseg = 0;
        hit = mesh_flight(c, xbuf, x, w, E, tau_star, &tint, &mint, &nseg);
        st[ST_FLIGHT_STEPS] += nseg;
      } else if (clip_box(c, x, w, 0.0, INFINITY, &ta, &tb)) {
        double L = tb - ta;
        long n = (long)ceil(L / step);
        if (n < 1) n = 1;
        double hh = L / n, tau = 0;
        for (long k = 0; k < n; ++k) {
          double t = ta + (k + 0.5) * hh;
          double p[3] = {x[0] + t * w[0], x[1] + t * w[1], x[2] + t * w[2]};
          int ijk[3];
          size_t v = voxel_of(c, p, ijk);
          double mu = c->rho[v] * mu_rho_tot(c, c->mat[v], E) * 0.1;
          st[ST_FLIGHT_STEPS] += 1;
          if (tau + mu * hh >= tau_star) {
            tint = ta + k * hh + (tau_star - tau) / mu;
            mint = c->mat[v];
            hit = 1;
            break;
          }
          tau += mu * hh;
        }
      }
      if (!hit) {
        /* escape; the analog tally records where it meets the detector */
        e_esc += E * W;
        st[ST_ESCAPE] += 1;
        double wn = w[0] * P.n[0] + w[1] * P.n[1] + w[2] * P.n[2];
        double *img = order == 0 ? analog0 : analog;
        if (img && wn < 0) {
          double cx[3] = {P.c[0] - x[0], P.c[1] - x[1], P.c[2] - x[2]};
          double t = (cx[0] * P.n[0] + cx[1] * P.n[1] + cx[2] * P.n[2]) / wn;
          if (t > 0) {
            double y[3] = {x[0] + t * w[0] - P.c[0], x[1] + t * w[1] - P.c[1], x[2] + t * w[2] - P.c[2]};
            double a = (y[0] * P.eu[0] + y[1] * P.eu[1] + y[2] * P.eu[2]) / c->pu + 0.5 * c->nu;
            double b = (y[0] * P.ev[0] + y[1] * P.ev[1] + y[2] * P.ev[2]) / c->pv + 0.5 * c->nv;
            if (a >= 0 && a < c->nu && b >= 0 && b < c->nv)
              img[(size_t)floor(b) * c->nu + (size_t)floor(a)] += det_eta(c, E) * W;
          }
        }
        break;
      }
      for (int k = 0; k < 3; ++k) x[k] += tint * w[k];
      /* interaction type */
      double pe = tab(c, c->mu_pe, mint, E), in = tab(c, c->mu_in, mint, E), co = tab(c, c->mu_co, mint, E);
      double ut = rng_u(&g) * (pe + in + co);
      int type = ut < pe ? 0 : (ut < pe + in ? 1 : 2);
      if (type == 0 && c->nee_mode == 0) {
        st[ST_PHOTO] += 1;
        e_dep += E * W;
        break;
      }
      if (type != 0) st[type == 1 ? ST_COMPTON : ST_RAYLEIGH] += 1;
      /* point-detector scoring, split into n_split pseudo-particles, eq. (Th) */
      rng_align(&g);
      const uint32_t k0 = g.ctr[0];
      const int n_pp = c->forced ? (int)Pt : c->n_split;
      for (int s = 0; s < n_pp; ++s) {
        uint32_t r = rng_next(&g);
        double va = rng_u(&g), vb = rng_u(&g), vr = rng_u(&g);
        uint64_t pt = c->forced ? (uint64_t)s : ((uint64_t)r * Pt) >> 32;
        int pi = u0 + (int)(pt % wt), pj = v0 + (int)(pt / wt);
        uint64_t pix = (uint64_t)pj * c->nu + pi;
        double Pp[3];
        det_point(c, &P, pi + va, pj + vb, Pp);
        double DD[3] = {Pp[0] - x[0], Pp[1] - x[1], Pp[2] - x[2]};
        double dd = sqrt(DD[0] * DD[0] + DD[1] * DD[1] + DD[2] * DD[2]);
        double dir[3] = {DD[0] / dd, DD[1] / dd, DD[2] / dd};
        /* the scattering cosine of two unit vectors, kept within [-1, 1] against rounding */
        double lam = fmin(fmax(w[0] * dir[0] + w[1] * dir[1] + w[2] * dir[2], -1.0), 1.0);
        double cosg = -(dir[0] * P.n[0] + dir[1] * P.n[1] + dir[2] * P.n[2]);
        const double geo = tile_w * A_px * cosg * ((double)Pt / n_pp) / (2.0 * PI * dd * dd);
        double sc;
        st[ST_NEE_RAYS] += 1;
        rng_t side;
        rng_side(&side, &g, k0 + (uint32_t)s);
        int dfail = 0;
        if (c->nee_mode == 0) {
          double Ep;
          double p = orc_nee_pdf(c, type, mint, E, lam, &Ep);
          if (type == 1 && c->doppler) Ep = E * sample_doppler(c, &side, mint, E, lam, &dfail);
          st[ST_SAMPLER_FAIL] += dfail;
          double x0 = W * det_eta(c, Ep) * p * geo;
          if (c->rr_threshold > 0 && x0 < c->rr_threshold) {
            if (vr >= x0 / c->rr_threshold) {
              st[ST_RR_KILLED] += 1;
              continue;
            }
            x0 = c->rr_threshold;
          }
          long ns = 0;
          double tp = path_tau(c, x, dir, dd, step, Ep, &ns);
          st[ST_NEE_STEPS] += ns;
          sc = x0 * exp(-tp);
        } else {
          /* expected value over the interaction type */
          double Ep;
          const double mu = pe + in + co;
          double pc = orc_nee_pdf(c, 1, mint, E, lam, &Ep);
          double pr = orc_nee_pdf(c, 2, mint, E, lam, NULL);
          if (c->doppler) Ep = E * sample_doppler(c, &side, mint, E, lam, &dfail);
          st[ST_SAMPLER_FAIL] += dfail;
          double xc = W * (in / mu) * det_eta(c, Ep) * pc * geo;
          double xr = W * (co / mu) * det_eta(c, E) * pr * geo;
          const double x0 = xc + xr;
          if (c->rr_threshold > 0 && x0 < c->rr_threshold) {
            if (vr >= x0 / c->rr_threshold) {
              st[ST_RR_KILLED] += 1;
              continue;
            }
            xc *= c->rr_threshold / x0;
            xr *= c->rr_threshold / x0;
          }
          long ns = 0, ns2 = 0;
          double tc = path_tau(c, x, dir, dd, step, Ep, &ns);
          double tr = path_tau(c, x, dir, dd, step, E, &ns2);
          st[ST_NEE_STEPS] += ns; /* one march's steps: both walk the same midpoints (or crossings) */
          sc = xc * exp(-tc) + xr * exp(-tr);
        }
        Is[pix] += sc;
        if (Is_order) Is_order[(size_t)(order < 2 ? order : 2) * npix + pix] += sc;
      }
      if (type == 0) { /* expected-value mode scored the absorption site; the photon ends */
        st[ST_PHOTO] += 1;
        e_dep += E * W;
        break;
      }
      /* new direction */
      int fail = 0;
      double ct, Enew = E;
      if (type == 1) {
        double rr;
        ct = sample_incoherent(c, &g, mint, E, &rr, &fail);
        Enew = c->doppler ? E * sample_doppler(c, &g, mint, E, ct, &fail) : E / rr;
      } else {
        ct = sample_rayleigh(c, &g, mint, E, &fail);
      }
      double phi = 2.0 * PI * rng_u(&g);
      if (fail) st[ST_SAMPLER_FAIL] += 1;
      rotate(w, ct, phi);
      e_dep += (E - Enew) * W;
      E = Enew;
      order += 1;
      if (E < 1.0) {
        e_dep += E * W;
        break;
      }
      if (order >= c->max_order) {
        e_dep += E * W;
        st[ST_LIMIT] += 1;
        break;
      }
    }
    double err = fabs(e_src - e_dep - e_esc) / e_src;
    if (err > st[ST_MAX_EERR]) st[ST_MAX_EERR] = err;
    st[ST_E_SOURCE] += e_src;
    st[ST_E_DEPOSIT] += e_dep;
    st[ST_E_ESCAPE] += e_esc;
  }
  (void)nsteps;
  if (stats)
    for (int k = 0; k < ST_N; ++k) stats[k] += st[k];
  free(M); free(pre); free(xbuf);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Sampler access for the chi-square tests: n independent draws, stream h = i. */
int orc_sample_compton(double E, double mec2, uint64_t n, uint64_t seed, double *cos_out, double *ratio_out) {
  for (uint64_t i = 0; i < n; ++i) {
    rng_t g;
    rng_init(&g, i, 0, seed);
    int fail = 0;
    double r;
    cos_out[i] = sample_compton(&g, E, mec2, &r, &fail);
    if (ratio_out) ratio_out[i] = r;
    if (fail) return ORC_EINVAL;
  }
  return ORC_OK;
}

int orc_sample_incoherent(const orc_ctx *c, int m, double E, uint64_t n, uint64_t seed, double *cos_out) {
  if (!c->have_tables || m < 0 || m >= c->n_mat) return ORC_ESTATE;
  for (uint64_t i = 0; i < n; ++i) {
    rng_t g;
    rng_init(&g, i, 0, seed);
    int fail = 0;
    double r;
    cos_out[i] = sample_incoherent(c, &g, m, E, &r, &fail);
    if (fail) return ORC_EINVAL;
  }
  return ORC_OK;
}

int orc_sample_rayleigh(const orc_ctx *c, int m, double E, uint64_t n, uint64_t seed, double *cos_out) {
  if (!c->have_tables || m < 0 || m >= c->n_mat) return ORC_ESTATE;
  for (uint64_t i = 0; i < n; ++i) {
    rng_t g;
    rng_init(&g, i, 0, seed);
    int fail = 0;
    cos_out[i] = sample_rayleigh(c, &g, m, E, &fail);
    if (fail) return ORC_EINVAL;
  }
  return ORC_OK;
}

/* Uniforms of one history's stream, for cross-checking the generator. */
int orc_stream(uint64_t h, uint32_t angle_index, uint64_t seed, int n, uint32_t *out) {
  rng_t g;
  rng_init(&g, h, angle_index, seed);
  for (int i = 0; i < n; ++i) out[i] = rng_next(&g);
  return ORC_OK;
}

double orc_table(const orc_ctx *c, int which, int m, double E) {
  const double *a = which == 0 ? c->mu_pe : which == 1 ? c->mu_in : which == 2 ? c->mu_co : c->icoh;
  return tab(c, a, m, E);
}
