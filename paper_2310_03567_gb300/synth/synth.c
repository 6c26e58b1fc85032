/*
 * Seeded synthetic point clouds for the octree-update workloads.
 *
 * Records are 16 bytes: int32 x, y, z in millimetres and RGBA8, the point
 * layout of the paper's SIM format (Section 7.1) with the float xyz replaced
 * by 1 mm integers. This file holds only input generation: no octree, voxel
 * or chunk arithmetic lives here, so that the CPU oracle and the CUDA path can
 * both consume the same bytes without sharing any of the method.
 *
 * Random numbers: every draw is one output of a SplitMix64 generator
 * (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014), addressed by position: the n-th output of the generator
 * seeded with s is mix(s + n * gamma). Addressing by position makes the
 * output independent of the thread count. Gaussians use the Box-Muller
 * transform. Every stream derives its own seed from the workload seed.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t x, y, z;
  uint8_t r, g, b, a;
} sy_point;

#define SY_GAMMA 0x9E3779B97F4A7C15ull

static inline uint64_t sy_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* n-th output (n >= 1) of SplitMix64 seeded with s. */
static inline uint64_t sy_at(uint64_t s, uint64_t n) { return sy_mix(s + n * SY_GAMMA); }

/* Seed of sub-stream k of a workload seed. */
static inline uint64_t sy_stream(uint64_t seed, uint64_t k) { return sy_at(seed, k); }

/* Uniform integer in [0, m) by the multiply-shift map. */
static inline uint64_t sy_below(uint64_t r, uint64_t m) {
  return (uint64_t)(((unsigned __int128)r * m) >> 64);
}

/* Uniform double in [0, 1). */
static inline double sy_u01(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }

/* Uniform double in (0, 1]. */
static inline double sy_u01_open0(uint64_t r) { return (double)((r >> 11) + 1) * 0x1.0p-53; }

static void sy_box_muller(uint64_t r1, uint64_t r2, double* z0, double* z1) {
  double u1 = sy_u01_open0(r1), u2 = sy_u01(r2);
  double rad = sqrt(-2.0 * log(u1));
  double ang = 6.283185307179586 * u2;
  *z0 = rad * cos(ang);
  *z1 = rad * sin(ang);
}

static inline int32_t sy_quantize(double metres, int64_t hi) {
  double v = floor(metres * 1000.0 + 0.5);
  if (v < 0.0) v = 0.0;
  if (v > (double)hi) v = (double)hi;
  return (int32_t)v;
}

static inline uint8_t sy_clamp_u8(double v) {
  if (v < 0.0) return 0;
  if (v > 255.0) return 255;
  return (uint8_t)v;
}

/* ---------------------------------------------------------------- threads */

typedef void (*sy_range_fn)(void* ctx, uint64_t lo, uint64_t hi);
typedef struct {
  sy_range_fn fn;
  void* ctx;
  uint64_t lo, hi;
} sy_job;

static void* sy_job_main(void* p) {
  sy_job* j = (sy_job*)p;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

static void sy_parallel(uint64_t n, int nthreads, sy_range_fn fn, void* ctx) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((uint64_t)nthreads > n / 4096 + 1) nthreads = (int)(n / 4096 + 1);
  if (nthreads == 1) {
    fn(ctx, 0, n);
    return;
  }
  pthread_t th[256];
  sy_job jobs[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = fn;
    jobs[t].ctx = ctx;
    jobs[t].lo = n * (uint64_t)t / (uint64_t)nthreads;
    jobs[t].hi = n * (uint64_t)(t + 1) / (uint64_t)nthreads;
    pthread_create(&th[t], NULL, sy_job_main, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------- uniform in a cube */

typedef struct {
  uint64_t s, i0;
  int64_t extent;
  sy_point* out;
} sy_uniform_ctx;

static void sy_uniform_range(void* p, uint64_t lo, uint64_t hi) {
  sy_uniform_ctx* c = (sy_uniform_ctx*)p;
  for (uint64_t k = lo; k < hi; ++k) {
    uint64_t i = c->i0 + k, n = i * 4;
    sy_point q;
    q.x = (int32_t)sy_below(sy_at(c->s, n + 1), (uint64_t)c->extent);
    q.y = (int32_t)sy_below(sy_at(c->s, n + 2), (uint64_t)c->extent);
    q.z = (int32_t)sy_below(sy_at(c->s, n + 3), (uint64_t)c->extent);
    uint64_t col = sy_at(c->s, n + 4);
    q.r = (uint8_t)col;
    q.g = (uint8_t)(col >> 8);
    q.b = (uint8_t)(col >> 16);
    q.a = (uint8_t)(col >> 24);
    c->out[k] = q;
  }
}

/* Points i0 .. i0+n-1 of the stream: x, y, z uniform integers in
 * [0, extent) drawn in that order, then four uniform colour bytes. */
void synth_uniform(uint64_t seed, int64_t extent, uint64_t i0, uint64_t n, sy_point* out,
                   int nthreads) {
  sy_uniform_ctx c = {sy_stream(seed, 1), i0, extent, out};
  sy_parallel(n, nthreads, sy_uniform_range, &c);
}

/* ------------------------------------------------ aerial terrain scan lines */

typedef struct {
  uint64_t seed;
  double extent_m;      /* square side in metres */
  uint32_t row_len;     /* points per scan line */
  double wavelength_m;  /* wavelength of the coarsest octave */
  uint32_t octaves;
  double relief_m;      /* height range */
  double jitter_m;      /* standard deviation of the xyz jitter */
  double offset_x_m, offset_y_m; /* where the square starts */
  int64_t coord_max;    /* clamp bound in mm (2^root_log2 - 1) */
} sy_terrain_params;

static double sy_lattice(uint64_t s, uint32_t octave, int64_t i, int64_t j) {
  uint64_t key = ((uint64_t)octave << 42) + ((uint64_t)(i + 1) << 21) + (uint64_t)(j + 1);
  return sy_u01(sy_at(s, key + 1));
}

static double sy_value_noise(uint64_t s, uint32_t octave, double x, double y) {
  double fx0 = floor(x), fy0 = floor(y);
  int64_t ix = (int64_t)fx0, iy = (int64_t)fy0;
  double fx = x - fx0, fy = y - fy0;
  double sx = fx * fx * (3.0 - 2.0 * fx), sy = fy * fy * (3.0 - 2.0 * fy);
  double v00 = sy_lattice(s, octave, ix, iy), v10 = sy_lattice(s, octave, ix + 1, iy);
  double v01 = sy_lattice(s, octave, ix, iy + 1), v11 = sy_lattice(s, octave, ix + 1, iy + 1);
  double a = v00 + (v10 - v00) * sx, b = v01 + (v11 - v01) * sx;
  return a + (b - a) * sy;
}

/* Fractional Brownian motion of value noise, normalised to [0, 1]. */
double synth_terrain_height01(const sy_terrain_params* P, double x_m, double y_m) {
  uint64_t s = sy_stream(P->seed, 2);
  double sum = 0.0, norm = 0.0, amp = 1.0, freq = 1.0 / P->wavelength_m;
  for (uint32_t o = 0; o < P->octaves; ++o) {
    sum += amp * sy_value_noise(s, o, x_m * freq, y_m * freq);
    norm += amp;
    amp *= 0.5;
    freq *= 2.0;
  }
  return sum / norm;
}

static void sy_ramp(double h, uint8_t* r, uint8_t* g, uint8_t* b) {
  static const double stop[4] = {0.0, 0.33, 0.66, 1.0};
  static const double col[4][3] = {
      {34, 85, 34}, {107, 142, 35}, {139, 115, 85}, {245, 245, 245}};
  if (h < 0.0) h = 0.0;
  if (h > 1.0) h = 1.0;
  int k = 0;
  while (k < 2 && h > stop[k + 1]) ++k;
  double t = (h - stop[k]) / (stop[k + 1] - stop[k]);
  *r = sy_clamp_u8(col[k][0] + t * (col[k + 1][0] - col[k][0]) + 0.5);
  *g = sy_clamp_u8(col[k][1] + t * (col[k + 1][1] - col[k][1]) + 0.5);
  *b = sy_clamp_u8(col[k][2] + t * (col[k + 1][2] - col[k][2]) + 0.5);
}

typedef struct {
  const sy_terrain_params* P;
  uint64_t i0;
  sy_point* out;
} sy_terrain_ctx;

static void sy_terrain_range(void* p, uint64_t lo, uint64_t hi) {
  sy_terrain_ctx* c = (sy_terrain_ctx*)p;
  const sy_terrain_params* P = c->P;
  uint64_t s = sy_stream(P->seed, 1);
  double spacing = P->extent_m / (double)P->row_len;
  for (uint64_t k = lo; k < hi; ++k) {
    uint64_t i = c->i0 + k, n = i * 4;
    double x = P->offset_x_m + (double)(i % P->row_len) * spacing;
    double y = P->offset_y_m + (double)(i / P->row_len) * spacing;
    double h01 = synth_terrain_height01(P, x - P->offset_x_m, y - P->offset_y_m);
    double z = h01 * P->relief_m;
    double j0, j1, j2, j3;
    sy_box_muller(sy_at(s, n + 1), sy_at(s, n + 2), &j0, &j1);
    sy_box_muller(sy_at(s, n + 3), sy_at(s, n + 4), &j2, &j3);
    (void)j3;
    sy_point q;
    q.x = sy_quantize(x + P->jitter_m * j0, P->coord_max);
    q.y = sy_quantize(y + P->jitter_m * j1, P->coord_max);
    q.z = sy_quantize(z + P->jitter_m * j2, P->coord_max);
    sy_ramp(h01, &q.r, &q.g, &q.b);
    q.a = 255;
    c->out[k] = q;
  }
}

/* Points i0 .. i0+n-1 of the scan-line stream: point i sits at column
 * i mod row_len and row i div row_len of a regular grid over the square,
 * its height is the fBm terrain, and x, y, z each get Gaussian jitter. */
void synth_terrain(const sy_terrain_params* P, uint64_t i0, uint64_t n, sy_point* out,
                   int nthreads) {
  sy_terrain_ctx c = {P, i0, out};
  sy_parallel(n, nthreads, sy_terrain_range, &c);
}

/* ----------------------------------------------- clustered planar quads */

typedef struct {
  uint64_t seed;
  uint32_t n_quads;
  uint64_t n_points;
  double lo_m[3], hi_m[3];   /* range of quad centres */
  double side_min_m, side_max_m;
  double density_sigma;      /* log-normal sigma of the per-quad density */
  double noise_m;            /* isotropic Gaussian noise */
  int64_t coord_max;         /* clamp bound in mm */
} sy_cluster_params;

typedef struct {
  double c[3], t1[3], t2[3];
  double a, b;
  double weight;
  uint8_t col[3];
} sy_quad;

static void sy_make_quad(const sy_cluster_params* P, uint32_t q, sy_quad* Q) {
  uint64_t s = sy_stream(P->seed, 3), n = (uint64_t)q * 16;
  for (int k = 0; k < 3; ++k)
    Q->c[k] = P->lo_m[k] + (P->hi_m[k] - P->lo_m[k]) * sy_u01(sy_at(s, n + 1 + k));
  double nrm[3];
  if (sy_u01(sy_at(s, n + 4)) < 0.5) {
    int axis = (int)sy_below(sy_at(s, n + 5), 3);
    nrm[0] = nrm[1] = nrm[2] = 0.0;
    nrm[axis] = 1.0;
  } else {
    double zz = 2.0 * sy_u01(sy_at(s, n + 5)) - 1.0;
    double phi = 6.283185307179586 * sy_u01(sy_at(s, n + 6));
    double rr = sqrt(1.0 - zz * zz);
    nrm[0] = rr * cos(phi);
    nrm[1] = rr * sin(phi);
    nrm[2] = zz;
  }
  /* tangent basis: Gram-Schmidt against the least aligned axis */
  double h[3] = {0, 0, 0};
  int m = 0;
  for (int k = 1; k < 3; ++k)
    if (fabs(nrm[k]) < fabs(nrm[m])) m = k;
  h[m] = 1.0;
  double d = h[0] * nrm[0] + h[1] * nrm[1] + h[2] * nrm[2];
  double u[3] = {h[0] - d * nrm[0], h[1] - d * nrm[1], h[2] - d * nrm[2]};
  double ul = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  for (int k = 0; k < 3; ++k) u[k] /= ul;
  double v[3] = {nrm[1] * u[2] - nrm[2] * u[1], nrm[2] * u[0] - nrm[0] * u[2],
                 nrm[0] * u[1] - nrm[1] * u[0]};
  double th = 6.283185307179586 * sy_u01(sy_at(s, n + 7));
  double ct = cos(th), st = sin(th);
  for (int k = 0; k < 3; ++k) {
    Q->t1[k] = ct * u[k] + st * v[k];
    Q->t2[k] = -st * u[k] + ct * v[k];
  }
  double la = log(P->side_min_m), lb = log(P->side_max_m);
  Q->a = exp(la + (lb - la) * sy_u01(sy_at(s, n + 8)));
  Q->b = exp(la + (lb - la) * sy_u01(sy_at(s, n + 9)));
  double g0, g1;
  sy_box_muller(sy_at(s, n + 10), sy_at(s, n + 11), &g0, &g1);
  Q->weight = Q->a * Q->b * exp(P->density_sigma * g0);
  uint64_t col = sy_at(s, n + 12);
  Q->col[0] = (uint8_t)col;
  Q->col[1] = (uint8_t)(col >> 8);
  Q->col[2] = (uint8_t)(col >> 16);
}

typedef struct {
  double frac;
  uint32_t q;
} sy_rem;

static int sy_rem_cmp(const void* pa, const void* pb) {
  const sy_rem *a = (const sy_rem*)pa, *b = (const sy_rem*)pb;
  if (a->frac > b->frac) return -1;
  if (a->frac < b->frac) return 1;
  return a->q < b->q ? -1 : (a->q > b->q ? 1 : 0);
}

/* Points per quad, proportional to area x density, summing to exactly
 * n_points by the largest-remainder rule (ties by quad index). */
int synth_cluster_counts(const sy_cluster_params* P, uint64_t* counts) {
  uint32_t nq = P->n_quads;
  double* w = (double*)malloc(sizeof(double) * nq);
  sy_rem* rem = (sy_rem*)malloc(sizeof(sy_rem) * nq);
  if (!w || !rem) {
    free(w);
    free(rem);
    return -1;
  }
  double tot = 0.0;
  for (uint32_t q = 0; q < nq; ++q) {
    sy_quad Q;
    sy_make_quad(P, q, &Q);
    w[q] = Q.weight;
    tot += Q.weight;
  }
  uint64_t assigned = 0;
  for (uint32_t q = 0; q < nq; ++q) {
    double share = (double)P->n_points * w[q] / tot;
    double fl = floor(share);
    counts[q] = (uint64_t)fl;
    assigned += counts[q];
    rem[q].frac = share - fl;
    rem[q].q = q;
  }
  qsort(rem, nq, sizeof(sy_rem), sy_rem_cmp);
  uint64_t left = P->n_points > assigned ? P->n_points - assigned : 0;
  for (uint64_t k = 0; k < left; ++k) counts[rem[k % nq].q] += 1;
  free(w);
  free(rem);
  return 0;
}

typedef struct {
  const sy_cluster_params* P;
  const uint64_t* offsets; /* n_quads + 1 prefix sums */
  sy_point* out;
} sy_cluster_ctx;

static void sy_cluster_range(void* p, uint64_t lo, uint64_t hi) {
  sy_cluster_ctx* c = (sy_cluster_ctx*)p;
  const sy_cluster_params* P = c->P;
  uint64_t s = sy_stream(P->seed, 4);
  for (uint64_t q = lo; q < hi; ++q) {
    sy_quad Q;
    sy_make_quad(P, (uint32_t)q, &Q);
    for (uint64_t i = c->offsets[q]; i < c->offsets[q + 1]; ++i) {
      uint64_t n = i * 8;
      double u = (sy_u01(sy_at(s, n + 1)) - 0.5) * Q.a;
      double v = (sy_u01(sy_at(s, n + 2)) - 0.5) * Q.b;
      double e0, e1, e2, e3;
      sy_box_muller(sy_at(s, n + 3), sy_at(s, n + 4), &e0, &e1);
      sy_box_muller(sy_at(s, n + 5), sy_at(s, n + 6), &e2, &e3);
      uint64_t cn = sy_at(s, n + 7);
      sy_point pt;
      pt.x = sy_quantize(Q.c[0] + u * Q.t1[0] + v * Q.t2[0] + P->noise_m * e0, P->coord_max);
      pt.y = sy_quantize(Q.c[1] + u * Q.t1[1] + v * Q.t2[1] + P->noise_m * e1, P->coord_max);
      pt.z = sy_quantize(Q.c[2] + u * Q.t1[2] + v * Q.t2[2] + P->noise_m * e2, P->coord_max);
      pt.r = sy_clamp_u8((double)Q.col[0] + (double)((int)(cn & 15) - 8));
      pt.g = sy_clamp_u8((double)Q.col[1] + (double)((int)((cn >> 8) & 15) - 8));
      pt.b = sy_clamp_u8((double)Q.col[2] + (double)((int)((cn >> 16) & 15) - 8));
      pt.a = 255;
      c->out[i] = pt;
    }
  }
}

/* All points of the quad set, quad by quad (offsets from the counts). */
void synth_cluster_points(const sy_cluster_params* P, const uint64_t* offsets, sy_point* out,
                          int nthreads) {
  sy_cluster_ctx c = {P, offsets, out};
  sy_parallel(P->n_quads, nthreads, sy_cluster_range, &c);
}

/* Batch cut of an n-point stream: sizes uniform integers in [lo, hi] until
 * the points run out (the last batch takes the remainder), then the batch
 * order is shuffled by Fisher-Yates when permute != 0. Writes (offset,
 * count) pairs in insertion order; returns the batch count, or -1 when
 * max_batches is too small. */
int64_t synth_batches(uint64_t seed, uint64_t n, uint64_t lo, uint64_t hi, int permute,
                      uint64_t* offsets, uint64_t* counts, uint64_t max_batches) {
  uint64_t s = sy_stream(seed, 5), off = 0, k = 0;
  while (off < n) {
    if (k >= max_batches) return -1;
    uint64_t sz = lo + sy_below(sy_at(s, k + 1), hi - lo + 1);
    if (sz > n - off) sz = n - off;
    offsets[k] = off;
    counts[k] = sz;
    off += sz;
    ++k;
  }
  if (permute) {
    uint64_t sp = sy_stream(seed, 6);
    for (uint64_t i = k; i > 1; --i) {
      uint64_t j = sy_below(sy_at(sp, i), i);
      uint64_t to = offsets[i - 1], tc = counts[i - 1];
      offsets[i - 1] = offsets[j];
      counts[i - 1] = counts[j];
      offsets[j] = to;
      counts[j] = tc;
    }
  }
  return (int64_t)k;
}

/* Log-uniform batch sizes in [lo, hi] (no shuffle). Same return rules. */
int64_t synth_batches_loguniform(uint64_t seed, uint64_t n, uint64_t lo, uint64_t hi,
                                 uint64_t* offsets, uint64_t* counts, uint64_t max_batches) {
  uint64_t s = sy_stream(seed, 7), off = 0, k = 0;
  double la = log((double)lo), lb = log((double)hi);
  while (off < n) {
    if (k >= max_batches) return -1;
    uint64_t sz = (uint64_t)floor(exp(la + (lb - la) * sy_u01(sy_at(s, k + 1))));
    if (sz < lo) sz = lo;
    if (sz > hi) sz = hi;
    if (sz > n - off) sz = n - off;
    offsets[k] = off;
    counts[k] = sz;
    off += sz;
    ++k;
  }
  return (int64_t)k;
}
